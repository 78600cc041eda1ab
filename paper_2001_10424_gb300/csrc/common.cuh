// common.cuh - level descriptor, padded MAC layout and stencil device code.
//
// Padded layout of one grid level (2D uses nz = 1):
//   every array is indexed  k * S + j * P + i  with row pitch P >= nx + 1
//   (a multiple of 32 elements) and plane stride S = (ny + 1) * P.
//   velocity: component blocks u | v | w at offsets off[c]; u has nz planes of
//   ny rows of nx+1 faces, v nz planes of ny+1 rows of nx faces, w nz+1 planes
//   of ny rows of nx faces. pressure / cell arrays: nz planes of ny rows of nx.
//   Entries outside the active faces (Dirichlet boundary faces and padding)
//   are kept exactly zero by every kernel, so flat BLAS-1 over the whole
//   array equals BLAS-1 over the unknowns.
#pragma once

// Read-only loads and pointer qualifiers of the kernel bodies. By default the
// bodies read their inputs through the read-only (non-coherent) path, which
// is valid because no launch writes what it reads that way. A translation
// unit that runs several dependent steps inside one kernel (writing arrays
// that later steps read) defines both before including the headers, to plain
// coherent loads and no restrict.
#ifndef GKB_LDG
#define GKB_LDG(p) __ldg(p)
#endif
#ifndef GKB_RESTRICT
#define GKB_RESTRICT __restrict__
#endif
#include <cuda_runtime.h>
#include <stdint.h>

namespace gkb {

struct Lvl {
  int dim;            // 2 or 3
  int n[3];           // cells per axis (n[2] = 1 in 2D)
  int nat[6];         // 1 where the side is natural (outflow)
  int P;              // row pitch in elements
  long long S;        // plane stride
  long long off[3];   // velocity component offsets
  long long nvel;     // padded velocity length
  long long ncell;    // padded cell length (n[2] * S)
  double h;
  double wscale;      // h^(d-2): link conductance factor
  double ascale;      // h^(d-1): gradient entry
  double gc;          // gamma / n_scale
  double mu0;         // constant viscosity when mu == null
  const double* mu64; // cell viscosity in the padded cell layout, or null
  const float* mu32;
  // diagonal N: relative grad-div weight n_ref / N_cell of every cell (the
  // level's gc holds gamma / n_ref), or null for N = n_ref * I; only set on
  // variable-viscosity levels
  const double* nw64;
  const float* nw32;
  // node (2D) / edge (3D) viscosities of variable-viscosity levels: one
  // plane of em_plane() values per edge orientation E (the axis the edge
  // runs along; 2D has only E = 2), indexed by the padded index of the edge's
  // (node, node, cell) coordinates; null: computed from the cells on the fly
  const double* em64;
  const float* em32;
  // 1: W is -div(2 mu eps(u)) (normal links doubled, cross couplings at the
  // interior nodes / edges); only on variable-viscosity levels, all sides
  // Dirichlet
  int sym;
  // derived constants (set by finish_level), in both precisions so that FP32
  // kernels never convert from double on the FP64 pipe
  int has_gd;         // gc != 0
  int fast;           // deep-interior fast paths enabled
  double g2;          // gc * ascale^2: grad-div coupling of two faces of a cell
  double wmu;         // wscale * mu0
  double wkd;         // 2d * wmu: the diagonal of a regular constant-viscosity W row
  float mu0f, wscalef, ascalef, g2f, wmuf, wkdf;
};

// Coordinates of a thread block in the grid of one problem's launch and that
// grid's extent. A kernel launched for one problem takes its own blockIdx /
// gridDim; a lock-step batched launch (several problems in one grid) maps its
// blocks to (problem, block of that problem's grid) and hands the body the
// coordinates the problem's own launch would have had.
struct Blk {
  unsigned x, y, z, nx, ny, nz;
};

#ifdef __CUDACC__
__device__ __forceinline__ Blk native_blk() {
  return Blk{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}
#endif

inline void finish_level(Lvl& L) {
  L.has_gd = (L.gc != 0.0) ? 1 : 0;
  L.g2 = L.gc * L.ascale * L.ascale;
  L.wmu = L.wscale * L.mu0;
  L.wkd = (L.dim == 3 ? 6.0 : 4.0) * L.wmu;
  L.mu0f = (float)L.mu0;
  L.wscalef = (float)L.wscale;
  L.ascalef = (float)L.ascale;
  L.g2f = (float)L.g2;
  L.wmuf = (float)L.wmu;
  L.wkdf = (float)L.wkd;
}

// per-precision level constants
template <typename T> struct Kc;
template <> struct Kc<double> {
  static __host__ __device__ __forceinline__ double mu0(const Lvl& L) { return L.mu0; }
  static __host__ __device__ __forceinline__ double ws(const Lvl& L) { return L.wscale; }
  static __host__ __device__ __forceinline__ double as(const Lvl& L) { return L.ascale; }
  static __host__ __device__ __forceinline__ double g2(const Lvl& L) { return L.g2; }
  static __host__ __device__ __forceinline__ double wmu(const Lvl& L) { return L.wmu; }
  static __host__ __device__ __forceinline__ double wkd(const Lvl& L) { return L.wkd; }
};
template <> struct Kc<float> {
  static __host__ __device__ __forceinline__ float mu0(const Lvl& L) { return L.mu0f; }
  static __host__ __device__ __forceinline__ float ws(const Lvl& L) { return L.wscalef; }
  static __host__ __device__ __forceinline__ float as(const Lvl& L) { return L.ascalef; }
  static __host__ __device__ __forceinline__ float g2(const Lvl& L) { return L.g2f; }
  static __host__ __device__ __forceinline__ float wmu(const Lvl& L) { return L.wmuf; }
  static __host__ __device__ __forceinline__ float wkd(const Lvl& L) { return L.wkdf; }
};

// number of velocity unknowns (active faces) of a level
inline long long lvl_unknowns(const Lvl& L) {
  long long m = 0;
  for (int c = 0; c < L.dim; ++c) {
    long long k = L.n[c] + 1 - (L.nat[2 * c] ? 0 : 1) - (L.nat[2 * c + 1] ? 0 : 1);
    for (int a = 0; a < L.dim; ++a)
      if (a != c) k *= L.n[a];
    m += k;
  }
  return m;
}

__host__ __device__ __forceinline__ long long cix(const Lvl& L, int i, int j, int k) {
  return (long long)k * L.S + (long long)j * L.P + i;
}

// active face test for component C at (i, j, k)
template <int C>
__host__ __device__ __forceinline__ bool face_active(const Lvl& L, int i, int j, int k) {
  const int p[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (a >= L.dim) { if (p[a] != 0) return false; continue; }
    if (a == C) {
      if (p[a] < 0 || p[a] > L.n[a]) return false;
      if (p[a] == 0 && !L.nat[2 * a]) return false;
      if (p[a] == L.n[a] && !L.nat[2 * a + 1]) return false;
    } else {
      if (p[a] < 0 || p[a] >= L.n[a]) return false;
    }
  }
  return true;
}

__host__ __device__ __forceinline__ bool cell_in(const Lvl& L, int i, int j, int k) {
  return i >= 0 && i < L.n[0] && j >= 0 && j < L.n[1] && k >= 0 && k < L.n[2];
}

template <typename T> struct MuPtr;
template <> struct MuPtr<double> { static __device__ __forceinline__ const double* get(const Lvl& L) { return L.mu64; } };
template <> struct MuPtr<float>  { static __device__ __forceinline__ const float*  get(const Lvl& L) { return L.mu32; } };

template <typename T, bool VarMu>
__device__ __forceinline__ T cell_mu(const Lvl& L, int i, int j, int k) {
  if (!VarMu) return Kc<T>::mu0(L);
  return GKB_LDG(MuPtr<T>::get(L) + cix(L, i, j, k));
}

template <typename T> struct NwPtr;
template <> struct NwPtr<double> { static __device__ __forceinline__ const double* get(const Lvl& L) { return L.nw64; } };
template <> struct NwPtr<float>  { static __device__ __forceinline__ const float*  get(const Lvl& L) { return L.nw32; } };

// grad-div weight of an in-domain cell (1 unless N is a non-uniform diagonal)
template <typename T, bool VarMu>
__device__ __forceinline__ T cell_nw(const Lvl& L, long long cb) {
  if (!VarMu) return (T)1;
  const T* w = NwPtr<T>::get(L);
  return w ? GKB_LDG(w + cb) : (T)1;
}

__host__ __device__ __forceinline__ long long em_plane(const Lvl& L) {
  return (L.dim == 3 ? (long long)(L.n[2] + 1) : 1LL) * L.S;
}

template <typename T> struct EmPtr;
template <> struct EmPtr<double> { static __device__ __forceinline__ const double* get(const Lvl& L) { return L.em64; } };
template <> struct EmPtr<float>  { static __device__ __forceinline__ const float*  get(const Lvl& L) { return L.em32; } };

// mean viscosity of the in-domain cells around the node/edge crossed by a
// tangential link of component C along axis A; the cells have C-coordinate
// p[C]-1 and p[C], A-coordinate af-1 and af, other coordinates from p.
// Summed in the order (C-1, A-1), (C-1, A), (C, A-1), (C, A).
template <typename T, int C, int A>
__device__ __forceinline__ T edge_mu_cells(const Lvl& L, const int p[3], int af) {
  T s = 0;
  int cnt = 0;
#pragma unroll
  for (int dc = -1; dc <= 0; ++dc)
#pragma unroll
    for (int da = -1; da <= 0; ++da) {
      int q[3] = {p[0], p[1], p[2]};
      q[C] = p[C] + dc;
      q[A] = af + da;
      if (cell_in(L, q[0], q[1], q[2])) { s += cell_mu<T, true>(L, q[0], q[1], q[2]); ++cnt; }
    }
  return s / (T)cnt;
}

// the same from the level's node/edge table when it has one (one value per
// node/edge whichever component asks, so every path reads the same bits)
template <typename T, bool VarMu, int C, int A>
__device__ __forceinline__ T edge_mu(const Lvl& L, const int p[3], int af) {
  if (!VarMu) return Kc<T>::mu0(L);
  const T* em = EmPtr<T>::get(L);
  if (em) {
    constexpr int E = 3 - C - A;
    int q[3] = {p[0], p[1], p[2]};
    q[A] = af;
    return GKB_LDG(em + (L.dim == 3 ? E : 0) * em_plane(L) + cix(L, q[0], q[1], q[2]));
  }
  return edge_mu_cells<T, C, A>(L, p, af);
}

// velocity loads: through the read-only path (NC, the default: the array is
// not written during the kernel) or plain coherent loads (kernels that
// update the array they read between their own barriers)
template <typename T, bool NC = true>
__device__ __forceinline__ T ldv(const T* x, long long idx) {
  if (NC) return GKB_LDG(x + idx);
  return x[idx];
}

// rounded product that the compiler may not fuse into a neighbouring add:
// with the explicit fma() of the link sums it fixes every rounding of a W
// row, so that differently structured paths give bitwise equal rows
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Velocity value of component C at face position p; positions outside the
// face grid read as 0 (callers only ask for in-grid or wall-adjacent ones).
template <typename T, int C, bool NC = true>
__device__ __forceinline__ T face_val(const Lvl& L, const T* x, int i, int j, int k) {
  return ldv<T, NC>(x, L.off[C] + cix(L, i, j, k));
}

// index stride of axis A in the padded layout
template <int A>
__host__ __device__ __forceinline__ long long strd(const Lvl& L) {
  return A == 0 ? 1LL : (A == 1 ? (long long)L.P : L.S);
}
__host__ __device__ __forceinline__ long long strd_rt(const Lvl& L, int a) {
  return a == 0 ? 1LL : (a == 1 ? (long long)L.P : L.S);
}

// (A^T x)_cell / ascale = sum over components of (low face - high face),
// for the in-domain cell with padded index cb
template <typename T, bool NC = true>
__device__ __forceinline__ T neg_div_at(const Lvl& L, const T* x, long long cb) {
  const long long u = L.off[0] + cb, v = L.off[1] + cb;
  T s = ldv<T, NC>(x, u) - ldv<T, NC>(x, u + 1) + ldv<T, NC>(x, v) - ldv<T, NC>(x, v + L.P);
  if (L.dim == 3) {
    const long long w = L.off[2] + cb;
    s += ldv<T, NC>(x, w) - ldv<T, NC>(x, w + L.S);
  }
  return s;
}

template <typename T, bool NC = true>
__device__ __forceinline__ T neg_div(const Lvl& L, const T* x, int i, int j, int k) {
  if (!cell_in(L, i, j, k)) return (T)0;
  return neg_div_at<T, NC>(L, x, cix(L, i, j, k));
}

// Row of W at an active face of component C, position p (FV links, see
// include/gkb.h). Returns sum_links kappa (x_f - x_nb) with x_nb = 0 for
// mirror links, divided by wscale (the caller scales).
template <typename T, bool VarMu, int C, bool NC = true>
__device__ __forceinline__ T w_row(const Lvl& L, const T* x, const int p[3], T xf) {
  T acc = 0;
  const bool sym = VarMu && L.sym;
  // normal links across the cells p[C]-1 and p[C] (conductance 2 mu in the
  // symmetric-gradient form)
  {
    int q[3] = {p[0], p[1], p[2]};
    if (p[C] < L.n[C]) {
      q[C] = p[C] + 1;
      T mu = cell_mu<T, VarMu>(L, p[0], p[1], p[2]);
      if (sym) mu += mu;
      acc = fma(mu, xf - face_val<T, C, NC>(L, x, q[0], q[1], q[2]), acc);
    }
    if (p[C] > 0) {
      q[C] = p[C] - 1;
      T mu = cell_mu<T, VarMu>(L, q[0], q[1], q[2]);
      if (sym) mu += mu;
      acc = fma(mu, xf - face_val<T, C, NC>(L, x, q[0], q[1], q[2]), acc);
    }
  }
  const bool half = (p[C] == 0 && L.nat[2 * C]) || (p[C] == L.n[C] && L.nat[2 * C + 1]);
  const T area = half ? (T)0.5 : (T)1;
  // tangential links
#pragma unroll
  for (int A = 0; A < 3; ++A) {
    if (A == C || A >= L.dim) continue;
    int q[3] = {p[0], p[1], p[2]};
    // + direction: crosses A-face coordinate p[A]+1
    {
      T mu;
      if (A == 0) mu = edge_mu<T, VarMu, C, 0>(L, p, p[A] + 1);
      else if (A == 1) mu = edge_mu<T, VarMu, C, 1>(L, p, p[A] + 1);
      else mu = edge_mu<T, VarMu, C, 2>(L, p, p[A] + 1);
      if (p[A] + 1 < L.n[A]) {
        q[A] = p[A] + 1;
        acc = fma(area * mu, xf - face_val<T, C, NC>(L, x, q[0], q[1], q[2]), acc);
        if (sym) {
          // cross coupling at the interior node / edge (A-node p[A]+1,
          // C-node p[C]): -mu (u_A(p + e_A) - u_A(p + e_A - e_C))
          int s[3] = {p[0], p[1], p[2]};
          s[A] = p[A] + 1;
          const T ap = ldv<T, NC>(x, L.off[A] + cix(L, s[0], s[1], s[2]));
          s[C] = p[C] - 1;
          const T am = ldv<T, NC>(x, L.off[A] + cix(L, s[0], s[1], s[2]));
          acc = fma(-mu, ap - am, acc);
        }
      } else if (!L.nat[2 * A + 1]) {
        acc = fma((T)2 * area * mu, xf, acc);
      }
    }
    // - direction: crosses A-face coordinate p[A]
    {
      T mu;
      if (A == 0) mu = edge_mu<T, VarMu, C, 0>(L, p, p[A]);
      else if (A == 1) mu = edge_mu<T, VarMu, C, 1>(L, p, p[A]);
      else mu = edge_mu<T, VarMu, C, 2>(L, p, p[A]);
      if (p[A] > 0) {
        q[A] = p[A] - 1;
        acc = fma(area * mu, xf - face_val<T, C, NC>(L, x, q[0], q[1], q[2]), acc);
        if (sym) {
          // cross coupling at (A-node p[A], C-node p[C]): +mu (u_A(p) - u_A(p - e_C))
          int s[3] = {p[0], p[1], p[2]};
          const T ap = ldv<T, NC>(x, L.off[A] + cix(L, s[0], s[1], s[2]));
          s[C] = p[C] - 1;
          const T am = ldv<T, NC>(x, L.off[A] + cix(L, s[0], s[1], s[2]));
          acc = fma(mu, ap - am, acc);
        }
      } else if (!L.nat[2 * A]) {
        acc = fma((T)2 * area * mu, xf, acc);
      }
    }
  }
  return acc;
}

// Diagonal of W at an active face (divided by wscale).
template <typename T, bool VarMu, int C>
__device__ __forceinline__ T w_diag(const Lvl& L, const int p[3]) {
  T acc = 0;
  if (p[C] < L.n[C]) acc += cell_mu<T, VarMu>(L, p[0], p[1], p[2]);
  if (p[C] > 0) {
    int q[3] = {p[0], p[1], p[2]};
    q[C] = p[C] - 1;
    acc += cell_mu<T, VarMu>(L, q[0], q[1], q[2]);
  }
  if (VarMu && L.sym) acc += acc;  // normal conductance 2 mu
  const bool half = (p[C] == 0 && L.nat[2 * C]) || (p[C] == L.n[C] && L.nat[2 * C + 1]);
  const T area = half ? (T)0.5 : (T)1;
#pragma unroll
  for (int A = 0; A < 3; ++A) {
    if (A == C || A >= L.dim) continue;
    T mup, mum;
    if (A == 0) { mup = edge_mu<T, VarMu, C, 0>(L, p, p[A] + 1); mum = edge_mu<T, VarMu, C, 0>(L, p, p[A]); }
    else if (A == 1) { mup = edge_mu<T, VarMu, C, 1>(L, p, p[A] + 1); mum = edge_mu<T, VarMu, C, 1>(L, p, p[A]); }
    else { mup = edge_mu<T, VarMu, C, 2>(L, p, p[A] + 1); mum = edge_mu<T, VarMu, C, 2>(L, p, p[A]); }
    if (p[A] + 1 < L.n[A]) acc += area * mup; else if (!L.nat[2 * A + 1]) acc += (T)2 * area * mup;
    if (p[A] > 0) acc += area * mum; else if (!L.nat[2 * A]) acc += (T)2 * area * mum;
  }
  return acc;
}

// number of in-domain cells adjacent to a face of component C (1 or 2)
template <int C>
__device__ __forceinline__ int face_cells(const Lvl& L, const int p[3]) {
  return (p[C] < L.n[C] ? 1 : 0) + (p[C] > 0 ? 1 : 0);
}

// sum of the grad-div weights of the in-domain cells adjacent to a face
// (face_cells when N is a multiple of the identity)
template <typename T, bool VarMu, int C>
__device__ __forceinline__ T face_nw(const Lvl& L, const int p[3]) {
  if (!VarMu || !NwPtr<T>::get(L)) return (T)face_cells<C>(L, p);
  T s = 0;
  if (p[C] < L.n[C]) s += cell_nw<T, true>(L, cix(L, p[0], p[1], p[2]));
  if (p[C] > 0) {
    int q[3] = {p[0], p[1], p[2]};
    q[C] -= 1;
    s += cell_nw<T, true>(L, cix(L, q[0], q[1], q[2]));
  }
  return s;
}

// (M x)_f at an active face of component C: W row + gc * ascale^2 * grad(nw negdiv)
template <typename T, bool VarMu, int C, bool NC = true>
__device__ __forceinline__ T m_row(const Lvl& L, const T* x, const int p[3]) {
  const T xf = face_val<T, C, NC>(L, x, p[0], p[1], p[2]);
  T wv = w_row<T, VarMu, C, NC>(L, x, p, xf) * Kc<T>::ws(L);
  if (!L.has_gd) return wv;
  int q[3] = {p[0], p[1], p[2]};
  T dplus = neg_div<T, NC>(L, x, q[0], q[1], q[2]);
  if (cell_in(L, q[0], q[1], q[2])) dplus *= cell_nw<T, VarMu>(L, cix(L, q[0], q[1], q[2]));
  q[C] -= 1;
  T dminus = neg_div<T, NC>(L, x, q[0], q[1], q[2]);
  if (cell_in(L, q[0], q[1], q[2])) dminus *= cell_nw<T, VarMu>(L, cix(L, q[0], q[1], q[2]));
  return wv + Kc<T>::g2(L) * (dplus - dminus);
}

}  // namespace gkb
