// kernels_impl.cuh - templated MAC stencil, multigrid and BLAS-1 kernels.
// Included by kernels_f64.cu / kernels_f32.cu with KT = double / float.
#pragma once
#include "common.cuh"
#include "ops.h"
#include "reduce.cuh"

namespace gkb {

constexpr int BX = 32, BY = 8;

inline dim3 face_grid(const Lvl& L) {
  const int nz = (L.dim == 3) ? L.n[2] + 1 : 1;
  return dim3((L.n[0] + 1 + BX - 1) / BX, (L.n[1] + 1 + BY - 1) / BY, nz);
}
inline dim3 cell_grid(const Lvl& L) {
  return dim3((L.n[0] + BX - 1) / BX, (L.n[1] + BY - 1) / BY, L.n[2]);
}

// storage box of component C: may the padded array hold position (i,j,k)?
template <int C>
__device__ __forceinline__ bool in_store(const Lvl& L, int i, int j, int k) {
  if (i > L.n[0] || j > L.n[1]) return false;
  if (L.dim == 2) return k == 0;
  return C == 2 ? (k <= L.n[2]) : (k < L.n[2]);
}

// ---------------------------------------------------------------------------
// velocity -> velocity stencils
// ---------------------------------------------------------------------------

// y = W x (mode 0) or y = M x (mode 1); optionally sum x.y into a reduction.
template <typename T, bool VarMu, bool DOT>
__global__ void __launch_bounds__(BX* BY) k_apply(Lvl L, int mode, const T* __restrict__ x,
                                                   T* __restrict__ y, RedBuf red, int fin, void* st) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  double dot = 0.0;
  const int p[3] = {i, j, k};
#define GKB_APPLY_COMP(C)                                                        \
  if (in_store<C>(L, i, j, k)) {                                                 \
    const long long id = L.off[C] + cix(L, i, j, k);                             \
    T val = 0;                                                                   \
    if (face_active<C>(L, i, j, k)) {                                            \
      if (mode == 1) val = m_row<T, VarMu, C>(L, x, p);                          \
      else val = w_row<T, VarMu, C>(L, x, p, x[id]) * (T)L.wscale;               \
      if (DOT) dot += (double)x[id] * (double)val;                               \
    }                                                                            \
    y[id] = val;                                                                 \
  }
  GKB_APPLY_COMP(0)
  GKB_APPLY_COMP(1)
  if (L.dim == 3) { GKB_APPLY_COMP(2) }
#undef GKB_APPLY_COMP
  if (DOT) {
    double v[1] = {dot};
    grid_reduce<1>(v, red, fin, st);
  }
}

// r = b - M x  (x may be null: r = b)
template <typename T, bool VarMu>
__global__ void __launch_bounds__(BX* BY) k_residual(Lvl L, const T* __restrict__ x,
                                                      const T* __restrict__ b, T* __restrict__ r) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p[3] = {i, j, k};
#define GKB_RES_COMP(C)                                                          \
  if (in_store<C>(L, i, j, k)) {                                                 \
    const long long id = L.off[C] + cix(L, i, j, k);                             \
    T val = 0;                                                                   \
    if (face_active<C>(L, i, j, k)) {                                            \
      val = b[id];                                                               \
      if (x) val -= m_row<T, VarMu, C>(L, x, p);                                 \
    }                                                                            \
    r[id] = val;                                                                 \
  }
  GKB_RES_COMP(0)
  GKB_RES_COMP(1)
  if (L.dim == 3) { GKB_RES_COMP(2) }
#undef GKB_RES_COMP
}

// ---------------------------------------------------------------------------
// vertex (2D) / edge (3D) patch smoother: additive Schwarz over the patches
// of faces around each node (2D) or edge (3D); the faces of one patch carry
// the discrete curl of that node's / edge's hat function, i.e. a local
// divergence-free field, which makes the smoother robust in gamma.
// ---------------------------------------------------------------------------

template <int E> struct EAx;
template <> struct EAx<0> { static constexpr int a = 1, b = 2; };
template <> struct EAx<1> { static constexpr int a = 0, b = 2; };
template <> struct EAx<2> { static constexpr int a = 0, b = 1; };

__host__ __device__ __forceinline__ int cls5(int e, int n) {
  return e == 0 ? 0 : e == 1 ? 1 : e == n ? 4 : e == n - 1 ? 3 : 2;
}
__host__ __device__ __forceinline__ int cls3(int e, int n) {
  return e == 0 ? 0 : e == n - 1 ? 2 : 1;
}

template <int E>
__device__ __forceinline__ int patch_class(const Lvl& L, const int e[3]) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  const int nE = (E < L.dim) ? L.n[E] : 1;
  return (cls5(e[a], L.n[a]) * 5 + cls5(e[b], L.n[b])) * 3 + cls3(e[E], nE);
}

template <int C>
__device__ __forceinline__ bool face_half(const Lvl& L, const int p[3]) {
  return (p[C] == 0 && L.nat[2 * C]) || (p[C] == L.n[C] && L.nat[2 * C + 1]);
}

// Local matrix of M on the 4 faces of the patch of edge e (orientation E):
//   f0 = comp a at (b-1), f1 = comp a at e, f2 = comp b at (a-1), f3 = comp b at e.
// Inactive faces get an identity row/column.
template <typename T, bool VarMu, int E>
__device__ void patch_matrix(const Lvl& L, const int e[3], T Mp[4][4], bool act[4]) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  int q0[3] = {e[0], e[1], e[2]}; q0[b] -= 1;
  int q2[3] = {e[0], e[1], e[2]}; q2[a] -= 1;
  act[0] = face_active<a>(L, q0[0], q0[1], q0[2]);
  act[1] = face_active<a>(L, e[0], e[1], e[2]);
  act[2] = face_active<b>(L, q2[0], q2[1], q2[2]);
  act[3] = face_active<b>(L, e[0], e[1], e[2]);
  const T g = (T)(L.gc * L.ascale * L.ascale);
  const T ws = (T)L.wscale;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) Mp[r][c] = 0;
  Mp[0][0] = act[0] ? ws * w_diag<T, VarMu, a>(L, q0) + g * (T)face_cells<a>(L, q0) : (T)1;
  Mp[1][1] = act[1] ? ws * w_diag<T, VarMu, a>(L, e) + g * (T)face_cells<a>(L, e) : (T)1;
  Mp[2][2] = act[2] ? ws * w_diag<T, VarMu, b>(L, q2) + g * (T)face_cells<b>(L, q2) : (T)1;
  Mp[3][3] = act[3] ? ws * w_diag<T, VarMu, b>(L, e) + g * (T)face_cells<b>(L, e) : (T)1;
  if (act[0] && act[1]) {
    const T area = face_half<a>(L, e) ? (T)0.5 : (T)1;
    Mp[0][1] = Mp[1][0] = -ws * area * edge_mu<T, VarMu, a, b>(L, e, e[b]);
  }
  if (act[2] && act[3]) {
    const T area = face_half<b>(L, e) ? (T)0.5 : (T)1;
    Mp[2][3] = Mp[3][2] = -ws * area * edge_mu<T, VarMu, b, a>(L, e, e[a]);
  }
  if (L.gc != 0.0) {
    int cc[3] = {e[0], e[1], e[2]};
    cc[a] = e[a] - 1; cc[b] = e[b] - 1;
    if (act[0] && act[2] && cell_in(L, cc[0], cc[1], cc[2])) Mp[0][2] = Mp[2][0] = g;
    cc[a] = e[a]; cc[b] = e[b] - 1;
    if (act[0] && act[3] && cell_in(L, cc[0], cc[1], cc[2])) Mp[0][3] = Mp[3][0] = -g;
    cc[a] = e[a] - 1; cc[b] = e[b];
    if (act[1] && act[2] && cell_in(L, cc[0], cc[1], cc[2])) Mp[1][2] = Mp[2][1] = -g;
    cc[a] = e[a]; cc[b] = e[b];
    if (act[1] && act[3] && cell_in(L, cc[0], cc[1], cc[2])) Mp[1][3] = Mp[3][1] = g;
  }
}

// In-place Cholesky solve of the SPD 4x4 system Mp z = rhs.
template <typename T>
__device__ __forceinline__ void chol4_solve(T Mp[4][4], T rhs[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    T s = Mp[c][c];
#pragma unroll
    for (int k2 = 0; k2 < c; ++k2) s -= Mp[c][k2] * Mp[c][k2];
    const T d = sqrt(s);
    const T inv = (T)1 / d;
    Mp[c][c] = d;
#pragma unroll
    for (int r = c + 1; r < 4; ++r) {
      T t = Mp[r][c];
#pragma unroll
      for (int k2 = 0; k2 < c; ++k2) t -= Mp[r][k2] * Mp[c][k2];
      Mp[r][c] = t * inv;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    T t = rhs[r];
#pragma unroll
    for (int k2 = 0; k2 < r; ++k2) t -= Mp[r][k2] * rhs[k2];
    rhs[r] = t / Mp[r][r];
  }
#pragma unroll
  for (int r = 3; r >= 0; --r) {
    T t = rhs[r];
#pragma unroll
    for (int k2 = r + 1; k2 < 4; ++k2) t -= Mp[k2][r] * rhs[k2];
    rhs[r] = t / Mp[r][r];
  }
}

// residual of the patch faces (0 for inactive ones)
template <typename T, int E>
__device__ __forceinline__ void patch_rhs(const Lvl& L, const T* r, const int e[3], const bool act[4], T out[4]) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  int q0[3] = {e[0], e[1], e[2]}; q0[b] -= 1;
  int q2[3] = {e[0], e[1], e[2]}; q2[a] -= 1;
  out[0] = act[0] ? __ldg(r + L.off[a] + cix(L, q0[0], q0[1], q0[2])) : (T)0;
  out[1] = act[1] ? __ldg(r + L.off[a] + cix(L, e[0], e[1], e[2])) : (T)0;
  out[2] = act[2] ? __ldg(r + L.off[b] + cix(L, q2[0], q2[1], q2[2])) : (T)0;
  out[3] = act[3] ? __ldg(r + L.off[b] + cix(L, e[0], e[1], e[2])) : (T)0;
}

template <int E>
__device__ __forceinline__ void patch_active(const Lvl& L, const int e[3], bool act[4]) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  int q0[3] = {e[0], e[1], e[2]}; q0[b] -= 1;
  int q2[3] = {e[0], e[1], e[2]}; q2[a] -= 1;
  act[0] = face_active<a>(L, q0[0], q0[1], q0[2]);
  act[1] = face_active<a>(L, e[0], e[1], e[2]);
  act[2] = face_active<b>(L, q2[0], q2[1], q2[2]);
  act[3] = face_active<b>(L, e[0], e[1], e[2]);
}

// contribution of the patch of edge e to slot `slot` of z = C r
template <typename T, bool VarMu, int E>
__device__ __forceinline__ T patch_contrib(const Lvl& L, const T* r, const int e[3], int slot,
                                           const T* __restrict__ table) {
  bool act[4];
  T rp[4];
  if (VarMu || table == nullptr) {
    T Mp[4][4];
    patch_matrix<T, VarMu, E>(L, e, Mp, act);
    patch_rhs<T, E>(L, r, e, act, rp);
    chol4_solve<T>(Mp, rp);
    return rp[slot];
  }
  patch_active<E>(L, e, act);
  patch_rhs<T, E>(L, r, e, act, rp);
  const T* row = table + (size_t)(E * 75 + patch_class<E>(L, e)) * 16 + slot * 4;
  return __ldg(row + 0) * rp[0] + __ldg(row + 1) * rp[1] + __ldg(row + 2) * rp[2] + __ldg(row + 3) * rp[3];
}

// (C r) at an active face of component C, position p
template <typename T, bool VarMu, int C>
__device__ __forceinline__ T patch_apply(const Lvl& L, const T* r, const int p[3], const T* table) {
  T acc = 0;
#pragma unroll
  for (int E = 0; E < 3; ++E) {
    if (E == C) continue;
    if (L.dim == 2 && E != 2) continue;
    int e[3] = {p[0], p[1], p[2]};
    if (E == 0) {
      constexpr int a = EAx<0>::a, b = EAx<0>::b;
      if (C == a) { acc += patch_contrib<T, VarMu, 0>(L, r, e, 1, table); e[b] += 1; acc += patch_contrib<T, VarMu, 0>(L, r, e, 0, table); }
      else        { acc += patch_contrib<T, VarMu, 0>(L, r, e, 3, table); e[a] += 1; acc += patch_contrib<T, VarMu, 0>(L, r, e, 2, table); }
    } else if (E == 1) {
      constexpr int a = EAx<1>::a, b = EAx<1>::b;
      if (C == a) { acc += patch_contrib<T, VarMu, 1>(L, r, e, 1, table); e[b] += 1; acc += patch_contrib<T, VarMu, 1>(L, r, e, 0, table); }
      else        { acc += patch_contrib<T, VarMu, 1>(L, r, e, 3, table); e[a] += 1; acc += patch_contrib<T, VarMu, 1>(L, r, e, 2, table); }
    } else {
      constexpr int a = EAx<2>::a, b = EAx<2>::b;
      if (C == a) { acc += patch_contrib<T, VarMu, 2>(L, r, e, 1, table); e[b] += 1; acc += patch_contrib<T, VarMu, 2>(L, r, e, 0, table); }
      else        { acc += patch_contrib<T, VarMu, 2>(L, r, e, 3, table); e[a] += 1; acc += patch_contrib<T, VarMu, 2>(L, r, e, 2, table); }
    }
  }
  return acc;
}

// One Chebyshev step of the patch-preconditioned smoother:
//   z = C r;  d = ca * z + cb * d;  x = (x_zero ? 0 : x) + d
template <typename T, bool VarMu>
__global__ void __launch_bounds__(BX* BY) k_cheb(Lvl L, const T* __restrict__ r, T* __restrict__ x,
                                                  T* __restrict__ d, T ca, T cb, int x_zero, const T* table) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p[3] = {i, j, k};
#define GKB_CHEB_COMP(C)                                                         \
  if (in_store<C>(L, i, j, k) && face_active<C>(L, i, j, k)) {                   \
    const long long id = L.off[C] + cix(L, i, j, k);                             \
    const T z = patch_apply<T, VarMu, C>(L, r, p, table);                        \
    const T dn = (cb != (T)0) ? ca * z + cb * d[id] : ca * z;                    \
    d[id] = dn;                                                                  \
    x[id] = x_zero ? dn : x[id] + dn;                                            \
  }
  GKB_CHEB_COMP(0)
  GKB_CHEB_COMP(1)
  if (L.dim == 3) { GKB_CHEB_COMP(2) }
#undef GKB_CHEB_COMP
}

// z = C r (power iteration, tests)
template <typename T, bool VarMu>
__global__ void __launch_bounds__(BX* BY) k_patch(Lvl L, const T* __restrict__ r, T* __restrict__ z, const T* table) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p[3] = {i, j, k};
#define GKB_PATCH_COMP(C)                                                        \
  if (in_store<C>(L, i, j, k)) {                                                 \
    const long long id = L.off[C] + cix(L, i, j, k);                             \
    z[id] = face_active<C>(L, i, j, k) ? patch_apply<T, VarMu, C>(L, r, p, table) : (T)0; \
  }
  GKB_PATCH_COMP(0)
  GKB_PATCH_COMP(1)
  if (L.dim == 3) { GKB_PATCH_COMP(2) }
#undef GKB_PATCH_COMP
}

// Inverse of the local patch matrix of every class (constant coefficients):
// one thread per (orientation E, class). Gauss-Jordan in FP64.
template <typename T>
__global__ void k_patch_table(Lvl L, T* table) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * 75) return;
  const int E = t / 75, cl = t % 75;
  if (E >= L.dim && !(L.dim == 2 && E == 2)) return;
  if (L.dim == 2 && E != 2) return;
  const int ca = cl / 15, cb = (cl / 3) % 5, cE = cl % 3;
  int a, b;
  if (E == 0) { a = 1; b = 2; } else if (E == 1) { a = 0; b = 2; } else { a = 0; b = 1; }
  const int nE = (E < L.dim) ? L.n[E] : 1;
  auto rep5 = [](int c, int n) { return c == 0 ? 0 : c == 1 ? 1 : c == 2 ? 2 : c == 3 ? n - 1 : n; };
  auto rep3 = [](int c, int n) { return c == 0 ? 0 : c == 1 ? (n > 2 ? 1 : 0) : n - 1; };
  int e[3] = {0, 0, 0};
  e[a] = rep5(ca, L.n[a]);
  e[b] = rep5(cb, L.n[b]);
  e[E] = rep3(cE, nE);
  double Mp[4][4];
  bool act[4];
  if (E == 0) patch_matrix<double, false, 0>(L, e, Mp, act);
  else if (E == 1) patch_matrix<double, false, 1>(L, e, Mp, act);
  else patch_matrix<double, false, 2>(L, e, Mp, act);
  double inv[4][4];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) inv[r][c] = (r == c) ? 1.0 : 0.0;
  for (int c = 0; c < 4; ++c) {
    const double piv = 1.0 / Mp[c][c];
    for (int k2 = 0; k2 < 4; ++k2) { Mp[c][k2] *= piv; inv[c][k2] *= piv; }
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const double f = Mp[r][c];
      for (int k2 = 0; k2 < 4; ++k2) { Mp[r][k2] -= f * Mp[c][k2]; inv[r][k2] -= f * inv[c][k2]; }
    }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c)
      table[(size_t)t * 16 + r * 4 + c] = (act[r] && act[c]) ? (T)inv[r][c] : (T)0;
}

// ---------------------------------------------------------------------------
// gradient / divergence
// ---------------------------------------------------------------------------

// y = s * A p  (faces from cells): y_f = s * ascale * (p_plus - p_minus)
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_grad(Lvl L, const T* __restrict__ pc, T* __restrict__ y, T s) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const T sc = s * (T)L.ascale;
#define GKB_GRAD_COMP(C, DI, DJ, DK)                                             \
  if (in_store<C>(L, i, j, k)) {                                                 \
    const long long id = L.off[C] + cix(L, i, j, k);                             \
    T val = 0;                                                                   \
    if (face_active<C>(L, i, j, k)) {                                            \
      const T pp = cell_in(L, i, j, k) ? __ldg(pc + cix(L, i, j, k)) : (T)0;     \
      const T pm = cell_in(L, i - DI, j - DJ, k - DK) ? __ldg(pc + cix(L, i - DI, j - DJ, k - DK)) : (T)0; \
      val = sc * (pp - pm);                                                      \
    }                                                                            \
    y[id] = val;                                                                 \
  }
  GKB_GRAD_COMP(0, 1, 0, 0)
  GKB_GRAD_COMP(1, 0, 1, 0)
  if (L.dim == 3) { GKB_GRAD_COMP(2, 0, 0, 1) }
#undef GKB_GRAD_COMP
}

// y = s * A^T x  (cells from faces) = s * ascale * negdiv(x); padding untouched
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_negdiv(Lvl L, const T* __restrict__ x, T* __restrict__ y, T s) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= L.n[0] || j >= L.n[1]) return;
  y[cix(L, i, j, k)] = s * (T)L.ascale * neg_div<T>(L, x, i, j, k);
}

// ---------------------------------------------------------------------------
// grid transfer: divergence-preserving prolongation (normal-linear,
// tangential-constant embedding of the coarse face field) and its transpose
// ---------------------------------------------------------------------------

template <typename T, int C>
__device__ __forceinline__ T coarse_face(const Lvl& Lc, const T* xc, int I, int J, int K) {
  if (!face_active<C>(Lc, I, J, K)) return (T)0;
  return __ldg(xc + Lc.off[C] + cix(Lc, I, J, K));
}

// xf += P xc
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_prolong(Lvl Lf, Lvl Lc, const T* __restrict__ xc, T* __restrict__ xf) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p[3] = {i, j, k};
#define GKB_PROL_COMP(C)                                                         \
  if (in_store<C>(Lf, i, j, k) && face_active<C>(Lf, i, j, k)) {                 \
    int q[3] = {p[0] >> 1, p[1] >> 1, p[2] >> 1};                                \
    T val;                                                                       \
    if ((p[C] & 1) == 0) {                                                       \
      val = coarse_face<T, C>(Lc, xc, q[0], q[1], q[2]);                         \
    } else {                                                                     \
      T v0 = coarse_face<T, C>(Lc, xc, q[0], q[1], q[2]);                        \
      q[C] += 1;                                                                 \
      T v1 = coarse_face<T, C>(Lc, xc, q[0], q[1], q[2]);                        \
      val = (T)0.5 * (v0 + v1);                                                  \
    }                                                                            \
    xf[Lf.off[C] + cix(Lf, i, j, k)] += val;                                     \
  }
  GKB_PROL_COMP(0)
  GKB_PROL_COMP(1)
  if (Lf.dim == 3) { GKB_PROL_COMP(2) }
#undef GKB_PROL_COMP
}

template <typename T, int C>
__device__ __forceinline__ T fine_face(const Lvl& Lf, const T* rf, int i, int j, int k) {
  if (!face_active<C>(Lf, i, j, k)) return (T)0;
  return __ldg(rf + Lf.off[C] + cix(Lf, i, j, k));
}

// bc = P^T rf  (launched over the coarse face grid)
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_restrict(Lvl Lf, Lvl Lc, const T* __restrict__ rf, T* __restrict__ bc) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  const int K = blockIdx.z;
  const int P3[3] = {I, J, K};
#define GKB_REST_COMP(C)                                                         \
  if (in_store<C>(Lc, I, J, K)) {                                                \
    T acc = 0;                                                                   \
    if (face_active<C>(Lc, I, J, K)) {                                           \
      const int t1 = (C == 0) ? 1 : 0, t2 = (C == 2) ? 1 : 2;                    \
      const int nt2 = (Lf.dim == 3) ? 2 : 1;                                     \
      for (int s1 = 0; s1 < 2; ++s1)                                             \
        for (int s2 = 0; s2 < nt2; ++s2) {                                       \
          int q[3] = {2 * P3[0], 2 * P3[1], 2 * P3[2]};                          \
          q[t1] += s1;                                                           \
          if (Lf.dim == 3) q[t2] += s2;                                          \
          acc += fine_face<T, C>(Lf, rf, q[0], q[1], q[2]);                      \
          q[C] += 1;                                                             \
          acc += (T)0.5 * fine_face<T, C>(Lf, rf, q[0], q[1], q[2]);             \
          q[C] -= 2;                                                             \
          if (q[C] >= 0) acc += (T)0.5 * fine_face<T, C>(Lf, rf, q[0], q[1], q[2]); \
        }                                                                        \
    }                                                                            \
    bc[Lc.off[C] + cix(Lc, I, J, K)] = acc;                                      \
  }
  GKB_REST_COMP(0)
  GKB_REST_COMP(1)
  if (Lc.dim == 3) { GKB_REST_COMP(2) }
#undef GKB_REST_COMP
}

// coarsest level: x[idx[r]] = sum_c Minv[r][c] b[idx[c]]; one warp per row
template <typename T>
__global__ void k_coarse_solve(int m, const T* __restrict__ Minv, const int* __restrict__ idx,
                               const T* __restrict__ b, T* __restrict__ x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  double acc = 0.0;
  const T* row = Minv + (size_t)warp * m;
  for (int c = lane; c < m; c += 32) acc += (double)row[c] * (double)__ldg(b + idx[c]);
  acc = warp_sum(acc);
  if (lane == 0) x[idx[warp]] = (T)acc;
}

// ---------------------------------------------------------------------------
// BLAS-1 on flat padded arrays (len multiple of 4), fused reductions
// ---------------------------------------------------------------------------

constexpr int RB = 256;

// sum a.b (and b.b when NV == 2)
template <typename T>
__global__ void __launch_bounds__(RB) k_dot(long long len, const T* __restrict__ a, const T* __restrict__ b,
                                             RedBuf red, int fin, void* st) {
  T acc = 0;
  const long long stride = (long long)gridDim.x * RB;
  for (long long t = (long long)blockIdx.x * RB + threadIdx.x; t < len; t += stride)
    acc += a[t] * b[t];
  double v[1] = {(double)acc};
  grid_reduce<1>(v, red, fin, st);
}

// x += alpha p ; r -= alpha q ; sum r.r      (alpha from CgState)
template <typename T>
__global__ void __launch_bounds__(RB) k_cg_update(long long len, T* __restrict__ x, const T* __restrict__ p,
                                                   T* __restrict__ r, const T* __restrict__ q,
                                                   const CgState* cg, RedBuf red, void* st) {
  const T alpha = (T)cg->alpha;
  T acc = 0;
  const long long stride = (long long)gridDim.x * RB;
  for (long long t = (long long)blockIdx.x * RB + threadIdx.x; t < len; t += stride) {
    x[t] += alpha * p[t];
    const T rn = r[t] - alpha * q[t];
    r[t] = rn;
    acc += rn * rn;
  }
  double v[1] = {(double)acc};
  grid_reduce<1>(v, red, FIN_CG_RR, st);
}

// p = z + beta p   (beta from CgState; first: p = z)
template <typename T>
__global__ void __launch_bounds__(RB) k_cg_dir(long long len, T* __restrict__ p, const T* __restrict__ z,
                                                const CgState* cg, int first) {
  const T beta = first ? (T)0 : (T)cg->beta;
  const long long stride = (long long)gridDim.x * RB;
  for (long long t = (long long)blockIdx.x * RB + threadIdx.x; t < len; t += stride)
    p[t] = z[t] + beta * p[t];
}

// y = a x + b y (host scalars)
template <typename T>
__global__ void __launch_bounds__(RB) k_axpby(long long len, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  const long long stride = (long long)gridDim.x * RB;
  for (long long t = (long long)blockIdx.x * RB + threadIdx.x; t < len; t += stride)
    y[t] = a * x[t] + b * y[t];
}

}  // namespace gkb
