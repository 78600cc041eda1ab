// ops.h - host launch wrappers for the templated MAC kernels (FP64 / FP32).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"
#include "state.cuh"

namespace gkb {

struct RedBuf;

template <typename T>
struct Ops {
  // y = W x (mode 0) or M x (mode 1)
  static void apply(const Lvl& L, int mode, const T* x, T* y, cudaStream_t s);
  // same, and reduce x.y through finaliser `fin` on state `st`
  static void apply_dot(const Lvl& L, int mode, const T* x, T* y, const RedBuf& red, int fin, void* st,
                        cudaStream_t s);
  // r = b - M x (x null: r = b); pred: device flag, launch is a no-op when 0
  static void residual(const Lvl& L, const T* x, const T* b, T* r, cudaStream_t s, const int* pred = nullptr);
  // one Chebyshev step of the patch smoother
  // (fold_in: the constant-viscosity class stencils of the interior class,
  // 2 or 3 x 16 values of the table at fold_interior_offset, read back at
  // setup; null: the general kernel)
  static void cheb(const Lvl& L, const T* r, T* x, T* d, T ca, T cb, int x_zero, const T* table,
                   cudaStream_t s, const double* fold_in = nullptr);
  // z = C r (additive patch preconditioner)
  static void patch(const Lvl& L, const T* r, T* z, const T* table, cudaStream_t s);
  // length of the smoother's inverse table of level L: the patch classes
  // (3*75*16 entries) for constant viscosity, every patch for variable
  static long long patch_table_len(const Lvl& L);
  // where the table holds the interior class's 2D or 3D stencils (-1: no
  // such stencils on this level)
  static long long fold_interior_offset(const Lvl& L);
  static void patch_table(const Lvl& L, T* table, cudaStream_t s);
  // node (2D) / edge (3D) viscosity table of a variable-viscosity level
  static long long edge_table_len(const Lvl& L);
  static void edge_table(const Lvl& L, T* em, cudaStream_t s);
  // y = scale * A p (faces from cells)
  static void grad(const Lvl& L, const T* p, T* y, T scale, cudaStream_t s);
  // y = scale * A^T x (cells from faces)
  static void negdiv(const Lvl& L, const T* x, T* y, T scale, cudaStream_t s);
  // xf += P xc
  // (slopes: 2 x the coarse level's velocity length of scratch, 3D only)
  static void prolong(const Lvl& Lf, const Lvl& Lc, const T* xc, T* xf, T* slopes, cudaStream_t s);
  // bc = P^T rf (tmp, tmp2: coarse-sized scratch; tmp2 only in 3D)
  static void restrict_(const Lvl& Lf, const Lvl& Lc, const T* rf, T* bc, T* tmp, T* tmp2, cudaStream_t s);
  // coarsest level dense solve through the stored inverse
  static void coarse(int m, const T* Minv, const int* idx, const T* b, T* x, cudaStream_t s);
  // reductions and vector updates on flat padded arrays
  static void dot(long long len, const T* a, const T* b, const RedBuf& red, int fin, void* st, cudaStream_t s,
                  const int* pred = nullptr);
  // sums a.b and b.c (flexible CG: r.z and z.q)
  static void dot2(long long len, const T* a, const T* b, const T* c, const RedBuf& red, int fin, void* st,
                   cudaStream_t s);
  static void cg_update(long long len, T* x, const T* p, T* r, const T* q, const CgState* cg,
                        const RedBuf& red, void* st, cudaStream_t s, int fin = FIN_CG_RR);
  static void cg_dir(long long len, T* p, const T* z, const CgState* cg, int first, cudaStream_t s);
  static void axpby(long long len, T a, const T* x, T b, T* y, cudaStream_t s);
  // blocks used by the stencil launches of level L (reduction partial sizing)
  static long long face_blocks(const Lvl& L);
};

long long blas_blocks(long long len);

}  // namespace gkb
