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

// Position of a thread in its 32 x 8 block. 3D levels give every warp an
// 8 x 4 patch of the block instead of a 32-wide row: on the short x rows of
// 3D levels (a few warps per row) a row warp nearly always mixes the two
// boundary cells of the row with interior ones, so it runs both the general
// and the deep-interior path; an 8 x 4 warp meets a boundary 4x less often.
__device__ __forceinline__ void block_xy(const Lvl& L, int& tx, int& ty) {
  if (L.dim != 3) {
    tx = threadIdx.x;
    ty = threadIdx.y;
    return;
  }
  const int t = threadIdx.y * BX + threadIdx.x, w = t >> 5, l = t & 31;
  tx = ((w & 3) << 3) | (l & 7);
  ty = ((w >> 2) << 2) | (l >> 3);
}

// A position whose coordinates lie in [2, n-3] on every axis: all its faces
// are active, all their links regular and every patch containing one of its
// faces is in the interior class. L.fast = 0 disables the fast paths (the
// general paths compute bitwise the same values).
__device__ __forceinline__ bool deep_interior(const Lvl& L, int i, int j, int k) {
  bool d = L.fast && i >= 2 && i <= L.n[0] - 3 && j >= 2 && j <= L.n[1] - 3;
  if (L.dim == 3) d = d && k >= 2 && k <= L.n[2] - 3;
  return d;
}

// ---------------------------------------------------------------------------
// velocity -> velocity stencils
// ---------------------------------------------------------------------------

// A constant-viscosity face whose links are all regular (no wall, no
// natural side): its W row is wmu * (2d x_f - sum of the 2d neighbours).
template <int C>
__device__ __forceinline__ bool const_regular(const Lvl& L, const int p[3]) {
  bool interior = p[C] >= 1 && p[C] <= L.n[C] - 1;
#pragma unroll
  for (int A = 0; A < 3; ++A)
    if (A != C && A < L.dim) interior = interior && p[A] >= 1 && p[A] <= L.n[A] - 2;
  return interior;
}

// sum of the 2d neighbours of the face xc points at (+-1 in x, +-P in y,
// +-S in z), in the order every path uses
template <typename T>
__device__ __forceinline__ T nb_sum(const Lvl& L, const T* xc) {
  T acc = GKB_LDG(xc + 1) + GKB_LDG(xc - 1) + GKB_LDG(xc + L.P) + GKB_LDG(xc - L.P);
  if (L.dim == 3) acc += GKB_LDG(xc + L.S) + GKB_LDG(xc - L.S);
  return acc;
}

// M row of a regular constant-viscosity face, wmu (2d x_f - acc) +
// g2 (dp - dm) (acc: nb_sum; dp, dm: the negative divergences of the cells
// after and before the face; gd: with the grad-div term), as b - row (MODE 0)
// or the row (MODE 1), in multiply-adds in one fixed order: every path that
// forms this row (shared-memory tile, deep interior, general) computes it bit
// for bit alike, with one FP64-pipe operation fewer than the factored form.
template <typename T, int MODE>
__device__ __forceinline__ T const_row(const Lvl& L, T b, T xf, T acc, bool gd, T dp, T dm) {
  const T wmu = Kc<T>::wmu(L), wkd = Kc<T>::wkd(L), g2 = Kc<T>::g2(L);
  if (MODE == 0) {
    T t = gd ? fma(-g2, dp - dm, b) : b;
    t = fma(wmu, acc, t);
    return fma(-wkd, xf, t);
  }
  T t = gd ? g2 * (dp - dm) : (T)0;
  t = fma(-wmu, acc, t);
  return fma(wkd, xf, t);
}

// W row for variable viscosity at a deep-interior face (all links regular,
// all cells in the domain): the same operations in the same order as the
// general link-by-link row, without its bookkeeping. xc points at the face,
// mc at the viscosity of the cell with the face's padded index.
template <typename T, int C>
__device__ __forceinline__ T w_row_var_deep(const Lvl& L, const T* xc, const T* mc, T xf) {
  const long long sc = strd<C>(L);
  const bool sym = L.sym;
  T acc = 0;
  T m0 = GKB_LDG(mc), m1 = GKB_LDG(mc - sc);
  if (sym) { m0 += m0; m1 += m1; }
  acc = fma(m0, xf - GKB_LDG(xc + sc), acc);
  acc = fma(m1, xf - GKB_LDG(xc - sc), acc);
#pragma unroll
  for (int A = 0; A < 3; ++A) {
    if (A == C || A >= L.dim) continue;
    const long long sa = A == 0 ? 1LL : (A == 1 ? (long long)L.P : L.S);
    // u_A at the face's padded index (cross couplings of the symmetric form)
    const T* xa = xc - L.off[C] + L.off[A];
    // node/edge means: from the level's table (the node/edge of the + link
    // has the padded index of the face plus sa, that of the - link the
    // face's), else from the cells at C-offsets -1, 0 and A-offsets (0, +1) /
    // (-1, 0) in the order of edge_mu_cells
    const T* em = EmPtr<T>::get(L);
    const T* emp = em ? em + (L.dim == 3 ? 3 - C - A : 0) * em_plane(L) + (mc - MuPtr<T>::get(L)) : nullptr;
    const T mup = em ? GKB_LDG(emp + sa)
                     : (((GKB_LDG(mc - sc) + GKB_LDG(mc - sc + sa)) + GKB_LDG(mc)) + GKB_LDG(mc + sa)) / (T)4;
    acc = fma(mup, xf - GKB_LDG(xc + sa), acc);
    if (sym) acc = fma(-mup, GKB_LDG(xa + sa) - GKB_LDG(xa + sa - sc), acc);
    const T mum = em ? GKB_LDG(emp)
                     : (((GKB_LDG(mc - sc - sa) + GKB_LDG(mc - sc)) + GKB_LDG(mc - sa)) + GKB_LDG(mc)) / (T)4;
    acc = fma(mum, xf - GKB_LDG(xc - sa), acc);
    if (sym) acc = fma(mum, GKB_LDG(xa) - GKB_LDG(xa - sc), acc);
  }
  return acc;
}

// Tiled MAC operator: the block first stores the (negative) divergence of
// its cells plus a one-cell halo (and the plane below in 3D) in shared
// memory, then every thread forms the W row of its faces and adds the
// grad-div term from the stored divergences.
//   mode 0: y = b - M x   (x null: y = b)
//   mode 1: y = M x       (wonly: y = W x), DOT: reduce x.y
template <typename T, bool VarMu, int MODE, bool DOT>
__device__ __forceinline__ void mac_tile_body(const Blk& B, const Lvl& L, int wonly, const T* GKB_RESTRICT x, const T* GKB_RESTRICT b,
                                                     T* GKB_RESTRICT y, RedBuf red, int fin, void* st, const int* pred) {
  // row stride 40 (>= BX + 1): conflict-free for the 8 x 4 warps of 3D levels
  // (8r + c covers the 32 banks) as well as for 32-wide rows
  __shared__ T Dt[2][BY + 1][40];
  // 2D blocks wholly in the deep interior: u, v (and mu) tiles with a
  // one-cell halo (u, v faces and cells i0-1 .. i0+BX, j0-1 .. j0+BY)
  __shared__ T Tl[VarMu ? 3 : 2][BY + 2][BX + 2];
  if (pred && !*pred) return;  // predicated launch (uniform over the grid)
  const int tid = threadIdx.y * BX + threadIdx.x;
  int tx, ty;
  block_xy(L, tx, ty);
  const int i0 = B.x * BX, j0 = B.y * BY, k = B.z;
  const int i = i0 + tx, j = j0 + ty;
  const bool gd = L.has_gd && !wonly && x != nullptr;
  const int cur = (L.dim == 3) ? 1 : 0;
  const bool tile2d = L.dim == 2 && L.fast && x != nullptr && (!VarMu || EmPtr<T>::get(L) == nullptr) && i0 >= 2 &&
                      i0 + BX + 2 <= L.n[0] && j0 >= 2 && j0 + BY + 2 <= L.n[1];
  if (tile2d) {
    constexpr int TW = BX + 2, TN = (BY + 2) * (BX + 2);
    const T* mu = MuPtr<T>::get(L);
    for (int t = tid; t < TN; t += BX * BY) {
      const int r = t / TW, c = t - r * TW;
      const long long g = cix(L, i0 - 1 + c, j0 - 1 + r, 0);
      Tl[0][r][c] = GKB_LDG(x + L.off[0] + g);
      Tl[1][r][c] = GKB_LDG(x + L.off[1] + g);
      if (VarMu) Tl[VarMu ? 2 : 0][r][c] = GKB_LDG(mu + g);
    }
    __syncthreads();
    if (gd) {
      // the divergences as neg_div_at forms them, from the tiles
      const T* nw = NwPtr<T>::get(L);
      for (int t = tid; t < (BY + 1) * (BX + 1); t += BX * BY) {
        const int cj = t / (BX + 1), ci = t - cj * (BX + 1);
        T dv = Tl[0][cj][ci] - Tl[0][cj][ci + 1] + Tl[1][cj][ci] - Tl[1][cj + 1][ci];
        if (nw) dv *= GKB_LDG(nw + cix(L, i0 - 1 + ci, j0 - 1 + cj, 0));
        Dt[0][cj][ci] = dv;
      }
      __syncthreads();
    }
  } else if (gd) {
    const int nplanes = (L.dim == 3) ? 2 : 1;
    constexpr int TS = (BX + 1) * (BY + 1);
    for (int t = tid; t < nplanes * TS; t += BX * BY) {
      const int pl = t / TS, rem = t - pl * TS;
      const int cj = rem / (BX + 1), ci = rem - cj * (BX + 1);
      const int gk = (L.dim == 3) ? k - 1 + pl : 0;
      const int gi = i0 - 1 + ci, gj = j0 - 1 + cj;
      if (cell_in(L, gi, gj, gk)) {
        const long long cc = cix(L, gi, gj, gk);
        T dv = neg_div_at<T>(L, x, cc);
        if (VarMu && NwPtr<T>::get(L)) dv *= GKB_LDG(NwPtr<T>::get(L) + cc);
        Dt[pl][cj][ci] = dv;
      } else {
        Dt[pl][cj][ci] = (T)0;
      }
    }
    __syncthreads();
  }
  const int p[3] = {i, j, k};
  const T g2 = Kc<T>::g2(L);
  const long long cb = cix(L, i, j, k);
  double dot = 0.0;
  if (tile2d && !VarMu) {
    // GKB_TILE_DEEP with every operand from the tiles
    const int c = tx + 1, r = ty + 1;
#define GKB_TILE_SMEM(C, DPLUS, DMINUS)                                          \
    {                                                                            \
      const long long id = L.off[C] + cb;                                        \
      const T xf = Tl[C][r][c];                                                  \
      T acc = Tl[C][r][c + 1] + Tl[C][r][c - 1] + Tl[C][r + 1][c] + Tl[C][r - 1][c]; \
      const T val = const_row<T, MODE>(L, (MODE == 0) ? b[id] : (T)0, xf, acc, gd, DPLUS, DMINUS); \
      if (DOT) dot += (double)xf * (double)val;                                  \
      y[id] = val;                                                               \
    }
    GKB_TILE_SMEM(0, Dt[0][ty + 1][tx + 1], Dt[0][ty + 1][tx])
    GKB_TILE_SMEM(1, Dt[0][ty + 1][tx + 1], Dt[0][ty][tx + 1])
#undef GKB_TILE_SMEM
  } else if (tile2d) {
    // the operations and roundings of w_row_var_deep + GKB_TILE_VDEEP, with
    // every operand from the tiles (bitwise equal to the general row)
    const T ws = Kc<T>::ws(L);
    const bool sym = L.sym;
    const int c = tx + 1, r = ty + 1;
    constexpr int MU = VarMu ? 2 : 0;
    {  // u face (C = 0, A = 1)
      const long long id = L.off[0] + cb;
      const T xf = Tl[0][r][c];
      T m0 = Tl[MU][r][c], m1 = Tl[MU][r][c - 1];
      if (sym) { m0 += m0; m1 += m1; }
      T acc = 0;
      acc = fma(m0, xf - Tl[0][r][c + 1], acc);
      acc = fma(m1, xf - Tl[0][r][c - 1], acc);
      const T mup = (((Tl[MU][r][c - 1] + Tl[MU][r + 1][c - 1]) + Tl[MU][r][c]) + Tl[MU][r + 1][c]) / (T)4;
      acc = fma(mup, xf - Tl[0][r + 1][c], acc);
      if (sym) acc = fma(-mup, Tl[1][r + 1][c] - Tl[1][r + 1][c - 1], acc);
      const T mum = (((Tl[MU][r - 1][c - 1] + Tl[MU][r][c - 1]) + Tl[MU][r - 1][c]) + Tl[MU][r][c]) / (T)4;
      acc = fma(mum, xf - Tl[0][r - 1][c], acc);
      if (sym) acc = fma(mum, Tl[1][r][c] - Tl[1][r][c - 1], acc);
      T m = mul_rn(acc, ws);
      if (gd) m = fma(g2, Dt[0][ty + 1][tx + 1] - Dt[0][ty + 1][tx], m);
      const T val = (MODE == 0) ? b[id] - m : m;
      if (DOT) dot += (double)xf * (double)val;
      y[id] = val;
    }
    {  // v face (C = 1, A = 0)
      const long long id = L.off[1] + cb;
      const T xf = Tl[1][r][c];
      T m0 = Tl[MU][r][c], m1 = Tl[MU][r - 1][c];
      if (sym) { m0 += m0; m1 += m1; }
      T acc = 0;
      acc = fma(m0, xf - Tl[1][r + 1][c], acc);
      acc = fma(m1, xf - Tl[1][r - 1][c], acc);
      const T mup = (((Tl[MU][r - 1][c] + Tl[MU][r - 1][c + 1]) + Tl[MU][r][c]) + Tl[MU][r][c + 1]) / (T)4;
      acc = fma(mup, xf - Tl[1][r][c + 1], acc);
      if (sym) acc = fma(-mup, Tl[0][r][c + 1] - Tl[0][r - 1][c + 1], acc);
      const T mum = (((Tl[MU][r - 1][c - 1] + Tl[MU][r - 1][c]) + Tl[MU][r][c - 1]) + Tl[MU][r][c]) / (T)4;
      acc = fma(mum, xf - Tl[1][r][c - 1], acc);
      if (sym) acc = fma(mum, Tl[0][r][c] - Tl[0][r - 1][c], acc);
      T m = mul_rn(acc, ws);
      if (gd) m = fma(g2, Dt[0][ty + 1][tx + 1] - Dt[0][ty][tx + 1], m);
      const T val = (MODE == 0) ? b[id] - m : m;
      if (DOT) dot += (double)xf * (double)val;
      y[id] = val;
    }
  } else if (!VarMu && x != nullptr && deep_interior(L, i, j, k)) {
#define GKB_TILE_DEEP(C, DPLUS, DMINUS)                                          \
    {                                                                            \
      const long long id = L.off[C] + cb;                                        \
      const T* xc = x + id;                                                      \
      const T xf = GKB_LDG(xc);                                                    \
      const T acc = nb_sum<T>(L, xc);                                            \
      const T val = const_row<T, MODE>(L, (MODE == 0) ? b[id] : (T)0, xf, acc, gd, DPLUS, DMINUS); \
      if (DOT) dot += (double)xf * (double)val;                                  \
      y[id] = val;                                                               \
    }
    GKB_TILE_DEEP(0, Dt[cur][ty + 1][tx + 1], Dt[cur][ty + 1][tx])
    GKB_TILE_DEEP(1, Dt[cur][ty + 1][tx + 1], Dt[cur][ty][tx + 1])
    if (L.dim == 3) { GKB_TILE_DEEP(2, Dt[1][ty + 1][tx + 1], Dt[0][ty + 1][tx + 1]) }
#undef GKB_TILE_DEEP
  } else if (VarMu && x != nullptr && deep_interior(L, i, j, k)) {
    const T ws = Kc<T>::ws(L);
    const T* mc = MuPtr<T>::get(L) + cb;
#define GKB_TILE_VDEEP(C, DPLUS, DMINUS)                                         \
    {                                                                            \
      const long long id = L.off[C] + cb;                                        \
      const T xf = GKB_LDG(x + id);                                                \
      T m = mul_rn(w_row_var_deep<T, C>(L, x + id, mc, xf), ws);                 \
      if (gd) m = fma(g2, (DPLUS) - (DMINUS), m);                                \
      const T val = (MODE == 0) ? b[id] - m : m;                                 \
      if (DOT) dot += (double)xf * (double)val;                                  \
      y[id] = val;                                                               \
    }
    GKB_TILE_VDEEP(0, Dt[cur][ty + 1][tx + 1], Dt[cur][ty + 1][tx])
    GKB_TILE_VDEEP(1, Dt[cur][ty + 1][tx + 1], Dt[cur][ty][tx + 1])
    if (L.dim == 3) { GKB_TILE_VDEEP(2, Dt[1][ty + 1][tx + 1], Dt[0][ty + 1][tx + 1]) }
#undef GKB_TILE_VDEEP
  } else {
#define GKB_TILE_COMP(C, DPLUS, DMINUS)                                          \
  if (in_store<C>(L, i, j, k)) {                                                 \
    const long long id = L.off[C] + cb;                                          \
    T val = 0;                                                                   \
    if (face_active<C>(L, i, j, k)) {                                            \
      T m = 0, xf = 0;                                                           \
      bool fused = false;                                                        \
      if (x) {                                                                   \
        xf = x[id];                                                              \
        if (VarMu) {                                                             \
          m = mul_rn(w_row<T, VarMu, C>(L, x, p, xf), Kc<T>::ws(L));             \
          if (gd) m = fma(g2, (DPLUS) - (DMINUS), m);                            \
        } else if (const_regular<C>(L, p)) {                                     \
          fused = true;                                                          \
          m = const_row<T, MODE>(L, (MODE == 0) ? b[id] : (T)0, xf, nb_sum<T>(L, x + id), gd, DPLUS, DMINUS); \
        } else {                                                                 \
          m = w_row<T, false, C>(L, x, p, xf) * Kc<T>::ws(L);                    \
          if (gd) m += g2 * ((DPLUS) - (DMINUS));                                \
        }                                                                        \
      }                                                                          \
      val = (MODE == 0 && !fused) ? b[id] - m : m;                               \
      if (DOT) dot += (double)xf * (double)val;                                  \
    }                                                                            \
    y[id] = val;                                                                 \
  }
  GKB_TILE_COMP(0, Dt[cur][ty + 1][tx + 1], Dt[cur][ty + 1][tx])
  GKB_TILE_COMP(1, Dt[cur][ty + 1][tx + 1], Dt[cur][ty][tx + 1])
  if (L.dim == 3) { GKB_TILE_COMP(2, Dt[1][ty + 1][tx + 1], Dt[0][ty + 1][tx + 1]) }
#undef GKB_TILE_COMP
  }
  if (DOT) {
    double v[1] = {dot};
    grid_reduce<1>(v, red, fin, st, B);
  }
}

template <typename T, bool VarMu, int MODE, bool DOT>
__global__ void __launch_bounds__(BX* BY) k_mac_tile(Lvl L, int wonly, const T* GKB_RESTRICT x, const T* GKB_RESTRICT b,
                                                     T* GKB_RESTRICT y, RedBuf red, int fin, void* st, const int* pred) {
  mac_tile_body<T, VarMu, MODE, DOT>(native_blk(), L, wonly, x, b, y, red, fin, st, pred);
}

// ---------------------------------------------------------------------------
// 3D constant-viscosity operator (mode 0: b - M x; mode 1: M x; DOT: with
// the fused x . y), one launch split by geometry. Box blocks take the
// positions [1, n-2] on every axis, where every face of every component is
// active and all its links are regular: a block of 32 x 8 threads walks
// MAC3_KZ planes of a 32 x 8 column, keeping x of three planes (u, v, w with a
// one-position halo) and the negative cell divergences of two cell planes in
// shared memory as rings, with x and b of the next plane fetched into
// registers while the current one is computed; every face forms the fused
// row (const_row) without tests. Shell blocks (the extra z slices of the
// grid) take the other positions, one thread each, with the general
// link-by-link row. Both use the operations and roundings of k_mac_tile, so
// the values are bit for bit its (the dot sums in another order).
// ---------------------------------------------------------------------------
constexpr int MAC3_KZ = 16;

// levels that take the split kernels (smaller ones stay with k_mac_tile)
inline bool mac3_level(const Lvl& L) {
  return L.dim == 3 && L.n[0] >= 16 && L.n[1] >= 16 && L.n[2] >= 16;
}
// The shell of positions around the box [lo, n - hi] (every axis) of a 3D
// level, in a fixed order: the lo + hi outer planes whole, then on every
// other plane the lo + hi outer rows whole and the lo + hi outer positions
// of the other rows.
__host__ __device__ __forceinline__ long long shell_count(const Lvl& L, int lo, int hi) {
  const long long nx = L.n[0] + 1, ny = L.n[1] + 1, w = lo + hi;
  return w * nx * ny + (L.n[2] + 1 - w) * (w * nx + w * (ny - w));
}
__device__ __forceinline__ void shell_ijk(const Lvl& L, int lo, int hi, long long t, int& i, int& j, int& k) {
  const int nx = L.n[0] + 1, ny = L.n[1] + 1, w = lo + hi;
  const long long full = (long long)nx * ny, ring = (long long)w * nx + (long long)w * (ny - w);
  if (t < w * full) {
    const int pl = (int)(t / full);
    const long long r = t - pl * full;
    k = pl < lo ? pl : L.n[2] - hi + 1 + (pl - lo);
    j = (int)(r / nx);
    i = (int)(r - (long long)j * nx);
  } else {
    const long long u = t - w * full;
    k = lo + (int)(u / ring);
    const long long r = u - (long long)(k - lo) * ring;
    if (r < (long long)w * nx) {
      const int rw = (int)(r / nx);
      j = rw < lo ? rw : L.n[1] - hi + 1 + (rw - lo);
      i = (int)(r - (long long)rw * nx);
    } else {
      const int e = (int)(r - (long long)w * nx);
      j = lo + e / w;
      const int c = e - (j - lo) * w;
      i = c < lo ? c : L.n[0] - hi + 1 + (c - lo);
    }
  }
}
// the shell of the operator's box [1, n-2]
__host__ __device__ __forceinline__ long long mac3_shell_count(const Lvl& L) { return shell_count(L, 1, 2); }
// z extent of the box part of the launch; z slices beyond it are the shell's
__host__ __device__ __forceinline__ int mac3_box_z(const Lvl& L) { return (L.n[2] - 2 + MAC3_KZ - 1) / MAC3_KZ; }
// one launch: the box's blocks, then enough z slices of blocks for one
// thread per shell position
inline dim3 mac3_grid(const Lvl& L) {
  const unsigned gx = (L.n[0] - 2 + BX - 1) / BX, gy = (L.n[1] - 2 + BY - 1) / BY;
  const long long per_slice = (long long)gx * gy * BX * BY;
  return dim3(gx, gy, mac3_box_z(L) + (unsigned)((mac3_shell_count(L) + per_slice - 1) / per_slice));
}

template <typename T, int MODE, bool DOT>
__device__ __forceinline__ double mac3_box_body(const Blk& B, const Lvl& L, int wonly, const T* GKB_RESTRICT x,
                                                const T* GKB_RESTRICT b, T* GKB_RESTRICT y) {
  constexpr int TW = BX + 2, TH = BY + 2;
  __shared__ T Xt[3][3][TH][TW];      // [plane slot][component][row][col]: position (i0-1+col, j0-1+row)
  __shared__ T Dv[2][BY + 1][BX + 1];  // [cell plane parity][row][col]: cell (i0-1+col, j0-1+row)
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int i0 = 1 + (int)B.x * BX, j0 = 1 + (int)B.y * BY, k0 = 1 + (int)B.z * MAC3_KZ;
  const int i = i0 + tx, j = j0 + ty;
  const int kend = min(k0 + MAC3_KZ, L.n[2] - 1);  // planes k0 .. kend-1 (uniform over the block)
  const bool mine = i <= L.n[0] - 2 && j <= L.n[1] - 2;
  const bool gd = L.has_gd && !wonly;
  auto slot = [](int k) { return k % 3; };   // k >= 0
  // this thread's tile entries: (col, row) = (tx, ty) of every component,
  // and for tid < 3 * HALO one entry of the halo (rows BY, BY+1 and columns
  // BX, BX+1 of component tid / HALO); the planes k0-1 .. kend lie in
  // [0, n-1], held by every component's box, so only x and y are tested
  // (once). xp[c] points at this thread's main entry of component c in the
  // plane to fetch next, xh at its halo entry; both advance by S per plane.
  constexpr int HALO = 2 * TW + 2 * BY;
  const bool tin0 = i0 - 1 + tx <= L.n[0] && j0 - 1 + ty <= L.n[1];
  int hc = 0, hr = 0, hq = 0;
  bool hin = false;
  if (tid < 3 * HALO) {
    hc = tid / HALO;
    const int h = tid - hc * HALO;
    if (h < 2 * TW) { hr = BY + h / TW; hq = h - (hr - BY) * TW; }
    else { hr = (h - 2 * TW) >> 1; hq = BX + ((h - 2 * TW) & 1); }
    hin = i0 - 1 + hq <= L.n[0] && j0 - 1 + hr <= L.n[1];
  }
  const T* xp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) xp[c] = x + L.off[c] + cix(L, i0 - 1 + tx, j0 - 1 + ty, k0 - 1);
  const T* xh = x + L.off[hc] + cix(L, i0 - 1 + hq, j0 - 1 + hr, k0 - 1);
  T pre[3], preh = (T)0;
  auto fetch = [&]() {  // the next plane in order (k0-1, k0, ...)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pre[c] = tin0 ? *xp[c] : (T)0;
      xp[c] += L.S;
    }
    if (tid < 3 * HALO) {
      preh = hin ? *xh : (T)0;
      xh += L.S;
    }
  };
  auto commit = [&](int k) {
    const int sl = slot(k);
#pragma unroll
    for (int c = 0; c < 3; ++c) Xt[sl][c][ty][tx] = pre[c];
    if (tid < 3 * HALO) Xt[sl][hc][hr][hq] = preh;
  };
  // the cells this thread forms divergences for: (tx, ty); row BY for tid <
  // BX; column BX for BX <= tid < BX + BY + 1 (cell planes k0-1 .. kend-1 lie
  // in [0, n-2]; x and y tested once)
  const int dci1 = (tid < BX) ? tid : BX, dcj1 = (tid < BX) ? BY : tid - BX;
  const bool has1 = tid < BX + BY + 1;
  const bool cin0 = i0 - 1 + tx < L.n[0] && j0 - 1 + ty < L.n[1];
  const bool cin1 = has1 && i0 - 1 + dci1 < L.n[0] && j0 - 1 + dcj1 < L.n[1];
  auto div_cell = [&](int kc, int ci, int cj, bool in) {
    const int s0 = slot(kc), s1 = slot(kc + 1);
    T dv = (T)0;
    if (in) {
      // the cell's low faces sit at tile [cj][ci] (neg_div_at's order)
      dv = Xt[s0][0][cj][ci] - Xt[s0][0][cj][ci + 1] + Xt[s0][1][cj][ci] - Xt[s0][1][cj + 1][ci];
      dv += Xt[s0][2][cj][ci] - Xt[s1][2][cj][ci];
    }
    Dv[kc & 1][cj][ci] = dv;
  };
  auto div_plane = [&](int kc) {
    div_cell(kc, tx, ty, cin0);
    if (has1) div_cell(kc, dci1, dcj1, cin1);
  };
  fetch();
  commit(k0 - 1);
  fetch();
  commit(k0);
  fetch();
  if (gd) {
    __syncthreads();
    div_plane(k0 - 1);
  }
  // this thread's faces of plane k: index cb in every component's block;
  // b of plane k+1 is fetched while plane k is computed
  long long cb = cix(L, i, j, k0);
  double dot = 0.0;
  T bnx[3] = {(T)0, (T)0, (T)0};
  auto fetch_b = [&](long long at) {
    if (MODE == 0 && mine) {
#pragma unroll
      for (int c = 0; c < 3; ++c) bnx[c] = b[L.off[c] + at];
    }
  };
  fetch_b(cb);
  for (int k = k0; k < kend; ++k, cb += L.S) {
    T bv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) bv[c] = bnx[c];
    commit(k + 1);
    if (k + 1 < kend) {
      fetch();
      fetch_b(cb + L.S);
    }
    __syncthreads();
    if (gd) {
      div_plane(k);
      __syncthreads();
    }
    if (mine) {
      const int sc = slot(k), su = slot(k + 1), sd = slot(k - 1);
#define GKB_MAC3_FACE(C, DPLUS, DMINUS)                                                        \
      {                                                                                        \
        const T xf = Xt[sc][C][ty + 1][tx + 1];                                                \
        T acc = Xt[sc][C][ty + 1][tx + 2] + Xt[sc][C][ty + 1][tx] + Xt[sc][C][ty + 2][tx + 1] + \
                Xt[sc][C][ty][tx + 1];                                                         \
        acc += Xt[su][C][ty + 1][tx + 1] + Xt[sd][C][ty + 1][tx + 1];                          \
        const T val = const_row<T, MODE>(L, bv[C], xf, acc, gd, gd ? (DPLUS) : (T)0,           \
                                         gd ? (DMINUS) : (T)0);                                \
        if (DOT) dot += (double)xf * (double)val;                                              \
        y[L.off[C] + cb] = val;                                                                \
      }
      GKB_MAC3_FACE(0, Dv[k & 1][ty + 1][tx + 1], Dv[k & 1][ty + 1][tx])
      GKB_MAC3_FACE(1, Dv[k & 1][ty + 1][tx + 1], Dv[k & 1][ty][tx + 1])
      GKB_MAC3_FACE(2, Dv[k & 1][ty + 1][tx + 1], Dv[(k - 1) & 1][ty + 1][tx + 1])
#undef GKB_MAC3_FACE
    }
    __syncthreads();  // the next plane's load and divergences overwrite slot k-1 and parity k-1
  }
  return dot;
}

// the shell: one thread per position (t = its index in the shell's order),
// the three faces as k_mac_tile's general path forms them (divergences from
// neg_div)
template <typename T, int MODE, bool DOT>
__device__ __forceinline__ double mac3_shell_body(const Lvl& L, int wonly, const T* GKB_RESTRICT x,
                                                  const T* GKB_RESTRICT b, T* GKB_RESTRICT y, long long t) {
  if (t >= mac3_shell_count(L)) return 0.0;
  int i, j, k;
  shell_ijk(L, 1, 2, t, i, j, k);
  const bool gd = L.has_gd && !wonly;
  const T g2 = Kc<T>::g2(L);
  const int p[3] = {i, j, k};
  const long long cb = cix(L, i, j, k);
  const T d0 = gd ? neg_div<T>(L, x, i, j, k) : (T)0;
  double dot = 0.0;
#define GKB_MAC3_SHELL(C, DMINUS)                                                              \
  if (in_store<C>(L, i, j, k)) {                                                               \
    const long long id = L.off[C] + cb;                                                        \
    T val = 0;                                                                                 \
    if (face_active<C>(L, i, j, k)) {                                                          \
      const T xf = x[id];                                                                      \
      const T dm = gd ? (DMINUS) : (T)0;                                                       \
      const T bb = (MODE == 0) ? b[id] : (T)0;                                                 \
      if (const_regular<C>(L, p)) {                                                            \
        val = const_row<T, MODE>(L, bb, xf, nb_sum<T>(L, x + id), gd, d0, dm);                 \
      } else {                                                                                 \
        T m = w_row<T, false, C>(L, x, p, xf) * Kc<T>::ws(L);                                  \
        if (gd) m += g2 * (d0 - dm);                                                           \
        val = (MODE == 0) ? bb - m : m;                                                        \
      }                                                                                        \
      if (DOT) dot += (double)xf * (double)val;                                                \
    }                                                                                          \
    y[id] = val;                                                                               \
  }
  GKB_MAC3_SHELL(0, neg_div<T>(L, x, i - 1, j, k))
  GKB_MAC3_SHELL(1, neg_div<T>(L, x, i, j - 1, k))
  GKB_MAC3_SHELL(2, neg_div<T>(L, x, i, j, k - 1))
#undef GKB_MAC3_SHELL
  return dot;
}

// DOT: x . y over box and shell, reduced through finaliser fin on st
template <typename T, int MODE, bool DOT>
__global__ void __launch_bounds__(BX* BY, sizeof(T) == 8 ? 3 : 4) k_mac3(Lvl L, int wonly, const T* GKB_RESTRICT x,
                                                    const T* GKB_RESTRICT b, T* GKB_RESTRICT y, RedBuf red,
                                                    int fin, void* st) {
  const int bz = mac3_box_z(L);
  double dot;
  if ((int)blockIdx.z < bz) {
    dot = mac3_box_body<T, MODE, DOT>(native_blk(), L, wonly, x, b, y);
  } else {
    const long long blk = ((long long)(blockIdx.z - bz) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    dot = mac3_shell_body<T, MODE, DOT>(L, wonly, x, b, y, blk * (BX * BY) + threadIdx.y * BX + threadIdx.x);
  }
  if (DOT) {
    double v[1] = {dot};
    grid_reduce<1>(v, red, fin, st);
  }
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
  const T g = Kc<T>::g2(L);
  const T ws = Kc<T>::ws(L);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) Mp[r][c] = 0;
  Mp[0][0] = act[0] ? ws * w_diag<T, VarMu, a>(L, q0) + g * face_nw<T, VarMu, a>(L, q0) : (T)1;
  Mp[1][1] = act[1] ? ws * w_diag<T, VarMu, a>(L, e) + g * face_nw<T, VarMu, a>(L, e) : (T)1;
  Mp[2][2] = act[2] ? ws * w_diag<T, VarMu, b>(L, q2) + g * face_nw<T, VarMu, b>(L, q2) : (T)1;
  Mp[3][3] = act[3] ? ws * w_diag<T, VarMu, b>(L, e) + g * face_nw<T, VarMu, b>(L, e) : (T)1;
  if (act[0] && act[1]) {
    const T area = face_half<a>(L, e) ? (T)0.5 : (T)1;
    Mp[0][1] = Mp[1][0] = -ws * area * edge_mu<T, VarMu, a, b>(L, e, e[b]);
  }
  if (act[2] && act[3]) {
    const T area = face_half<b>(L, e) ? (T)0.5 : (T)1;
    Mp[2][3] = Mp[3][2] = -ws * area * edge_mu<T, VarMu, b, a>(L, e, e[a]);
  }
  if (L.has_gd) {
    int cc[3] = {e[0], e[1], e[2]};
    // the two faces share one cell: coupling +-g times its weight
    cc[a] = e[a] - 1; cc[b] = e[b] - 1;
    if (act[0] && act[2] && cell_in(L, cc[0], cc[1], cc[2]))
      Mp[0][2] = Mp[2][0] = g * cell_nw<T, VarMu>(L, cix(L, cc[0], cc[1], cc[2]));
    cc[a] = e[a]; cc[b] = e[b] - 1;
    if (act[0] && act[3] && cell_in(L, cc[0], cc[1], cc[2]))
      Mp[0][3] = Mp[3][0] = -g * cell_nw<T, VarMu>(L, cix(L, cc[0], cc[1], cc[2]));
    cc[a] = e[a] - 1; cc[b] = e[b];
    if (act[1] && act[2] && cell_in(L, cc[0], cc[1], cc[2]))
      Mp[1][2] = Mp[2][1] = -g * cell_nw<T, VarMu>(L, cix(L, cc[0], cc[1], cc[2]));
    cc[a] = e[a]; cc[b] = e[b];
    if (act[1] && act[3] && cell_in(L, cc[0], cc[1], cc[2]))
      Mp[1][3] = Mp[3][1] = g * cell_nw<T, VarMu>(L, cix(L, cc[0], cc[1], cc[2]));
  }
  if (VarMu && L.sym && e[a] >= 1 && e[a] < L.n[a] && e[b] >= 1 && e[b] < L.n[b]) {
    // symmetric form: the cross coupling of an interior node / edge, +-k
    // with the same signs as the grad-div couplings
    const T k = ws * edge_mu<T, VarMu, a, b>(L, e, e[b]);
    Mp[0][2] += k; Mp[2][0] += k;
    Mp[0][3] -= k; Mp[3][0] -= k;
    Mp[1][2] -= k; Mp[2][1] -= k;
    Mp[1][3] += k; Mp[3][1] += k;
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

// residual of the patch faces (0 for inactive ones); ce = padded index of e
template <typename T, int E>
__device__ __forceinline__ void patch_rhs(const Lvl& L, const T* r, long long ce, const bool act[4], T out[4]) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  const T* ra = r + L.off[a] + ce;
  const T* rb = r + L.off[b] + ce;
  out[0] = act[0] ? GKB_LDG(ra - strd<b>(L)) : (T)0;
  out[1] = act[1] ? GKB_LDG(ra) : (T)0;
  out[2] = act[2] ? GKB_LDG(rb - strd<a>(L)) : (T)0;
  out[3] = act[3] ? GKB_LDG(rb) : (T)0;
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

// local solve of the patch of edge e with the matrix assembled on the fly
template <typename T, bool VarMu, int E>
__device__ __forceinline__ T patch_solve_inl(const Lvl& L, const T* r, const int e[3], long long ce, int slot) {
  bool act[4];
  T rp[4];
  T Mp[4][4];
  patch_matrix<T, VarMu, E>(L, e, Mp, act);
  patch_rhs<T, E>(L, r, ce, act, rp);
  chol4_solve<T>(Mp, rp);
  return rp[slot];
}

// the same, out of line: used for the twelve patches of a 3D face, whose
// inlined copies multiply the compile time of the kernels twentyfold
template <typename T, bool VarMu, int E>
__device__ __noinline__ T patch_solve(const Lvl& L, const T* r, int e0, int e1, int e2, long long ce, int slot) {
  const int e[3] = {e0, e1, e2};
  return patch_solve_inl<T, VarMu, E>(L, r, e, ce, slot);
}

// Variable viscosity: the inverse of every patch matrix is stored once per
// level (symmetric, 10 entries, zero in the rows and columns of inactive
// faces), as planes of vtab_plane(L) values indexed by the padded index of
// the patch's edge (node in 2D); one group of 10 planes per orientation in 3D.
__host__ __device__ __forceinline__ long long vtab_plane(const Lvl& L) {
  return (L.dim == 3 ? (long long)(L.n[2] + 1) : 1LL) * L.S;
}

// packed index of entry (r, c) of a symmetric 4 x 4 matrix, r <= c
__host__ __device__ __forceinline__ int sym4(int r, int c) {
  return r <= c ? (r * (7 - r)) / 2 + c : (c * (7 - c)) / 2 + r;
}

// row `slot` of the stored inverse of patch e applied to the patch residual
template <typename T, int E>
__device__ __forceinline__ T patch_vtab_row(const Lvl& L, const T* r, const int e[3], long long ce, int slot,
                                            const T* GKB_RESTRICT vtab) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  const long long Q = vtab_plane(L);
  const T* t = vtab + (size_t)(L.dim == 3 ? E : 0) * 10 * Q + ce;
  const T* ra = r + L.off[a] + ce;
  const T* rb = r + L.off[b] + ce;
  // faces outside the store (below the first node) are inactive: coefficient 0
  const T r0 = e[b] > 0 ? GKB_LDG(ra - strd<b>(L)) : (T)0;
  const T r2 = e[a] > 0 ? GKB_LDG(rb - strd<a>(L)) : (T)0;
  return GKB_LDG(t + sym4(slot, 0) * Q) * r0 + GKB_LDG(t + sym4(slot, 1) * Q) * GKB_LDG(ra) +
         GKB_LDG(t + sym4(slot, 2) * Q) * r2 + GKB_LDG(t + sym4(slot, 3) * Q) * GKB_LDG(rb);
}

// contribution of the patch of edge e (padded index ce) to slot `slot` of z = C r
// (table: the class inverses for constant viscosity, the per-patch inverses
// for variable viscosity)
template <typename T, bool VarMu, int E>
__device__ __forceinline__ T patch_contrib(const Lvl& L, const T* r, const int e[3], long long ce, int slot,
                                           const T* GKB_RESTRICT table) {
  bool act[4];
  T rp[4];
  if (VarMu) return patch_vtab_row<T, E>(L, r, e, ce, slot, table);
  if (table == nullptr) {
    if (E == 2 && L.dim == 2) return patch_solve_inl<T, VarMu, E>(L, r, e, ce, slot);
    return patch_solve<T, VarMu, E>(L, r, e[0], e[1], e[2], ce, slot);
  }
  patch_active<E>(L, e, act);
  patch_rhs<T, E>(L, r, ce, act, rp);
  const T* row = table + (size_t)(E * 75 + patch_class<E>(L, e)) * 16 + slot * 4;
  return GKB_LDG(row + 0) * rp[0] + GKB_LDG(row + 1) * rp[1] + GKB_LDG(row + 2) * rp[2] + GKB_LDG(row + 3) * rp[3];
}

// the two patches of orientation E that contain a face of component C at
// position p (padded cell index cb)
template <typename T, bool VarMu, int C, int E>
__device__ __forceinline__ T patch_pair(const Lvl& L, const T* r, const int p[3], long long cb, const T* table) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  int e[3] = {p[0], p[1], p[2]};
  T acc;
  if (C == a) {
    acc = patch_contrib<T, VarMu, E>(L, r, e, cb, 1, table);
    e[b] += 1;
    acc += patch_contrib<T, VarMu, E>(L, r, e, cb + strd<b>(L), 0, table);
  } else {
    acc = patch_contrib<T, VarMu, E>(L, r, e, cb, 3, table);
    e[a] += 1;
    acc += patch_contrib<T, VarMu, E>(L, r, e, cb + strd<a>(L), 2, table);
  }
  return acc;
}

// (C r) at an active face of component C, position p (padded cell index cb)
template <typename T, bool VarMu, int C>
__device__ __forceinline__ T patch_apply(const Lvl& L, const T* r, const int p[3], long long cb, const T* table) {
  if (L.dim == 2) return patch_pair<T, VarMu, C, 2>(L, r, p, cb, table);
  T acc = 0;
  if (C != 0) acc += patch_pair<T, VarMu, C, 0>(L, r, p, cb, table);
  if (C != 1) acc += patch_pair<T, VarMu, C, 1>(L, r, p, cb, table);
  if (C != 2) acc += patch_pair<T, VarMu, C, 2>(L, r, p, cb, table);
  return acc;
}

// ---- deep-interior fast path ---------------------------------------------
// A position at least two cells away from every wall has all its faces
// active, all links regular and every patch in the interior class; kernels
// test this once per thread (warp-uniform almost everywhere) and then use
// plain offset loads instead of per-face activity and class logic.
// interior patch class of orientation E (cls5 = 2 on both node axes, cls3 = 1
// on the cell axis in 3D, 0 in 2D)
template <int E>
__device__ __forceinline__ int interior_class(const Lvl& L) {
  return (2 * 5 + 2) * 3 + (L.dim == 3 ? 1 : 0);
}

// patch rows of an interior patch: rhs faces at fixed offsets of ce
template <typename T, int E>
__device__ __forceinline__ T patch_deep(const Lvl& L, const T* r, long long ce, const T* row) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  const T* ra = r + L.off[a] + ce;
  const T* rb = r + L.off[b] + ce;
  return GKB_LDG(row + 0) * GKB_LDG(ra - strd<b>(L)) + GKB_LDG(row + 1) * GKB_LDG(ra) + GKB_LDG(row + 2) * GKB_LDG(rb - strd<a>(L)) +
         GKB_LDG(row + 3) * GKB_LDG(rb);
}

template <typename T, int C, int E>
__device__ __forceinline__ T patch_pair_deep(const Lvl& L, const T* r, long long cb, const T* table) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  const T* rows = table + (size_t)(E * 75 + interior_class<E>(L)) * 16;
  if (C == a) return patch_deep<T, E>(L, r, cb, rows + 4) + patch_deep<T, E>(L, r, cb + strd<b>(L), rows + 0);
  return patch_deep<T, E>(L, r, cb, rows + 12) + patch_deep<T, E>(L, r, cb + strd<a>(L), rows + 8);
}

template <typename T, int C>
__device__ __forceinline__ T patch_apply_deep(const Lvl& L, const T* r, long long cb, const T* table) {
  if (L.dim == 2) return patch_pair_deep<T, C, 2>(L, r, cb, table);
  T acc = 0;
  if (C != 0) acc += patch_pair_deep<T, C, 0>(L, r, cb, table);
  if (C != 1) acc += patch_pair_deep<T, C, 1>(L, r, cb, table);
  if (C != 2) acc += patch_pair_deep<T, C, 2>(L, r, cb, table);
  return acc;
}

// 3D interior faces, constant viscosity: the four interior patches through a
// face of component C (two orientations, two patches each) act as one fixed
// 13-point stencil on r, stored after the class table (PATCH_FOLD_OFF) as 16
// coefficients per component: [0] the face itself, then for each orientation
// E != C in increasing order six neighbour terms (see k_patch_fold).
constexpr int PATCH_FOLD_OFF = 3 * 75 * 16;

template <typename T, int C>
__device__ __forceinline__ T patch_apply_fold(const Lvl& L, const T* GKB_RESTRICT r, long long cb,
                                              const T* GKB_RESTRICT fold) {
  const T* f = fold + C * 16;
  const T* rc = r + L.off[C] + cb;
  T acc = GKB_LDG(f) * GKB_LDG(rc);
  int t = 1;
#pragma unroll
  for (int E = 0; E < 3; ++E) {
    if (E == C) continue;
    const int a = (E == 0) ? 1 : 0, b = (E == 2) ? 1 : 2;
    const long long sa = strd_rt(L, a), sb = strd_rt(L, b);
    const T* ra = r + L.off[a] + cb;
    const T* rb = r + L.off[b] + cb;
    if (C == a) {
      acc += GKB_LDG(f + t + 0) * GKB_LDG(ra - sb);
      acc += GKB_LDG(f + t + 1) * GKB_LDG(rb - sa);
      acc += GKB_LDG(f + t + 2) * GKB_LDG(rb);
      acc += GKB_LDG(f + t + 3) * GKB_LDG(ra + sb);
      acc += GKB_LDG(f + t + 4) * GKB_LDG(rb + sb - sa);
      acc += GKB_LDG(f + t + 5) * GKB_LDG(rb + sb);
    } else {
      acc += GKB_LDG(f + t + 0) * GKB_LDG(ra - sb);
      acc += GKB_LDG(f + t + 1) * GKB_LDG(ra);
      acc += GKB_LDG(f + t + 2) * GKB_LDG(rb - sa);
      acc += GKB_LDG(f + t + 3) * GKB_LDG(ra + sa - sb);
      acc += GKB_LDG(f + t + 4) * GKB_LDG(ra + sa);
      acc += GKB_LDG(f + t + 5) * GKB_LDG(rb + sa);
    }
    t += 6;
  }
  return acc;
}

// The folded interior stencils of the 3D constant-viscosity smoother, from the
// interior-class rows of the table (one thread per component): for a face of
// component C = a of orientation E the patches are e = p (row 1) and
// p + e_b (row 0); for C = b they are e = p (row 3) and p + e_a (row 2); the
// face's own residual collects one entry of each row.
template <typename T>
__global__ void k_patch_fold(Lvl L, T* table) {
  const int C = threadIdx.x;
  if (L.dim != 3 || C >= 3) return;
  T* f = table + PATCH_FOLD_OFF + C * 16;
  for (int k = 0; k < 16; ++k) f[k] = (T)0;
  double self = 0.0;
  int t = 1;
  for (int E = 0; E < 3; ++E) {
    if (E == C) continue;
    const int a = (E == 0) ? 1 : 0;
    const T* R = table + (size_t)(E * 75 + (2 * 5 + 2) * 3 + 1) * 16;  // interior class in 3D
    if (C == a) {
      self += (double)R[1 * 4 + 1] + (double)R[0 * 4 + 0];
      f[t + 0] = R[1 * 4 + 0];
      f[t + 1] = R[1 * 4 + 2];
      f[t + 2] = R[1 * 4 + 3];
      f[t + 3] = R[0 * 4 + 1];
      f[t + 4] = R[0 * 4 + 2];
      f[t + 5] = R[0 * 4 + 3];
    } else {
      self += (double)R[3 * 4 + 3] + (double)R[2 * 4 + 2];
      f[t + 0] = R[3 * 4 + 0];
      f[t + 1] = R[3 * 4 + 1];
      f[t + 2] = R[3 * 4 + 2];
      f[t + 3] = R[2 * 4 + 0];
      f[t + 4] = R[2 * 4 + 1];
      f[t + 5] = R[2 * 4 + 3];
    }
    t += 6;
  }
  f[0] = (T)self;
}

// ---- 3D constant viscosity: folded stencils for every position class ------
// Per axis a position (face index along the face's normal axis, cell index
// along the others) falls in one of seven classes: 0, 1, 2 (its distance
// from the low side), 3 (interior), 4, 5, 6 (n - 2, n - 1, n). With at least
// six cells on the axis, the classes of a position fix the classes and the
// activity of every patch through its faces (their edges lie within one
// cell of it), so (C r) at a face of component C is one 13-point stencil per
// (position class, C): the face itself and, for each orientation E != C, the
// six other faces of its two patches (the offsets of patch_apply_fold). The
// stencils follow the interior table after PATCH_FOLD_OFF.
constexpr int FOLD3_OFF = PATCH_FOLD_OFF + 3 * 16;
constexpr int FOLD3_CLASSES = 343;
constexpr int FOLD3_INTERIOR = (3 * 7 + 3) * 7 + 3;

__host__ __device__ __forceinline__ int cls7(int x, int n) {
  return x <= 2 ? x : (x >= n - 2 ? x - n + 6 : 3);
}
__host__ __device__ __forceinline__ int rep7(int c, int n) {
  return c <= 3 ? c : n + c - 6;
}

// the two patches of orientation E through a face of component C at p: their
// rows of the class inverses, scattered into the stencil slots t..t+5 and the
// face's own slot 0 (inactive faces contribute nothing)
template <typename T, int E>
__device__ void fold3_orient(const Lvl& L, const T* GKB_RESTRICT inv, const int p[3], int C, double acc[13], int t) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  int e0[3] = {p[0], p[1], p[2]};
  int e1[3] = {p[0], p[1], p[2]};
  bool act0[4], act1[4];
  if (C == a) {
    e1[b] += 1;
    patch_active<E>(L, e0, act0);
    patch_active<E>(L, e1, act1);
    const T* R0 = inv + (size_t)(E * 75 + patch_class<E>(L, e0)) * 16 + 1 * 4;  // slot 1 of patch p
    const T* R1 = inv + (size_t)(E * 75 + patch_class<E>(L, e1)) * 16 + 0 * 4;  // slot 0 of patch p + e_b
    if (act0[0]) acc[t + 0] += (double)R0[0];
    if (act0[1]) acc[0] += (double)R0[1];
    if (act0[2]) acc[t + 1] += (double)R0[2];
    if (act0[3]) acc[t + 2] += (double)R0[3];
    if (act1[0]) acc[0] += (double)R1[0];
    if (act1[1]) acc[t + 3] += (double)R1[1];
    if (act1[2]) acc[t + 4] += (double)R1[2];
    if (act1[3]) acc[t + 5] += (double)R1[3];
  } else {
    e1[a] += 1;
    patch_active<E>(L, e0, act0);
    patch_active<E>(L, e1, act1);
    const T* R0 = inv + (size_t)(E * 75 + patch_class<E>(L, e0)) * 16 + 3 * 4;  // slot 3 of patch p
    const T* R1 = inv + (size_t)(E * 75 + patch_class<E>(L, e1)) * 16 + 2 * 4;  // slot 2 of patch p + e_a
    if (act0[0]) acc[t + 0] += (double)R0[0];
    if (act0[1]) acc[t + 1] += (double)R0[1];
    if (act0[2]) acc[t + 2] += (double)R0[2];
    if (act0[3]) acc[0] += (double)R0[3];
    if (act1[0]) acc[t + 3] += (double)R1[0];
    if (act1[1]) acc[t + 4] += (double)R1[1];
    if (act1[2]) acc[0] += (double)R1[2];
    if (act1[3]) acc[t + 5] += (double)R1[3];
  }
}

// the stencils of all position classes (one thread per class and component),
// from the class inverses at the start of the same table (k_patch_table),
// summed in FP64
template <typename T>
__global__ void k_fold3_table(Lvl L, T* table) {
  const T* inv = table;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (L.dim != 3 || t >= FOLD3_CLASSES * 3) return;
  const int C = t % 3, pc = t / 3;
  const int p[3] = {rep7(pc / 49, L.n[0]), rep7((pc / 7) % 7, L.n[1]), rep7(pc % 7, L.n[2])};
  double acc[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) acc[q] = 0.0;
  int slot = 1;
  if (C != 0) { fold3_orient<T, 0>(L, inv, p, C, acc, slot); slot += 6; }
  if (C != 1) { fold3_orient<T, 1>(L, inv, p, C, acc, slot); slot += 6; }
  if (C != 2) { fold3_orient<T, 2>(L, inv, p, C, acc, slot); }
  T* f = table + FOLD3_OFF + (size_t)t * 16;
  for (int q = 0; q < 13; ++q) f[q] = (T)acc[q];
  f[13] = f[14] = f[15] = (T)0;
}

// the interior class's stencils as a kernel parameter (read from the
// constant bank, no load instructions)
template <typename T>
struct Fold3In {
  T c[3][13];
};

// (C r) at an active face of component C by the stencil f (13 entries);
// near a side (Inner == false) only faces with a nonzero coefficient are
// read, which are active faces inside the arrays. Offsets are 32-bit (the
// padded arrays hold fewer than 2^31 entries).
template <typename T, int C, bool Inner, class Coef>
__device__ __forceinline__ T fold3_apply(const Lvl& L, const T* GKB_RESTRICT r, int cb, Coef f) {
  const int P = L.P, S = (int)L.S;
  const T* rc = r + L.off[C] + cb;
  T acc = f(0) * GKB_LDG(rc);
  int t = 1;
#pragma unroll
  for (int E = 0; E < 3; ++E) {
    if (E == C) continue;
    const int a = (E == 0) ? 1 : 0, b = (E == 2) ? 1 : 2;
    const int sa = a == 0 ? 1 : (a == 1 ? P : S), sb = b == 1 ? P : S;
    const T* ra = r + L.off[a] + cb;
    const T* rb = r + L.off[b] + cb;
    int o[6];
    const T* base[6];
    if (C == a) {
      base[0] = ra; o[0] = -sb; base[1] = rb; o[1] = -sa; base[2] = rb; o[2] = 0;
      base[3] = ra; o[3] = sb; base[4] = rb; o[4] = sb - sa; base[5] = rb; o[5] = sb;
    } else {
      base[0] = ra; o[0] = -sb; base[1] = ra; o[1] = 0; base[2] = rb; o[2] = -sa;
      base[3] = ra; o[3] = sa - sb; base[4] = ra; o[4] = sa; base[5] = rb; o[5] = sa;
    }
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const T c = f(t + u);
      if (Inner || c != (T)0) acc += c * GKB_LDG(base[u] + o[u]);
    }
    t += 6;
  }
  return acc;
}

// one Chebyshev step at one position: d, x are read before the stencil so
// that their loads overlap it
template <typename T, int C, bool Inner, class Coef>
__device__ __forceinline__ void cheb3_face(const Lvl& L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                           T* GKB_RESTRICT d, T ca, T cb, int x_zero, int p0, Coef f) {
  const int id = (int)L.off[C] + p0;
  const T dold = (cb != (T)0) ? d[id] : (T)0;
  const T xold = x_zero ? (T)0 : x[id];
  const T z = fold3_apply<T, C, Inner>(L, r, p0, f);
  const T dn = (cb != (T)0) ? ca * z + cb * dold : ca * z;
  d[id] = dn;
  x[id] = x_zero ? dn : xold + dn;
}

// one Chebyshev step of the 3D constant-viscosity smoother through the class
// stencils (levels with at least six cells on every axis). Every thread
// walks CHEB3_KZ planes; blocks whose positions are all interior take the
// interior stencils from the kernel parameter (the constant bank) with no
// per-face checks, the others the table's stencil of each position's class.
constexpr int CHEB3_KZ = 4;

template <typename T>
__device__ __forceinline__ void cheb3_body(const Blk& B, const Lvl& L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                           T* GKB_RESTRICT d, T ca, T cb, int x_zero, const T* GKB_RESTRICT table,
                                           const Fold3In<T>& fin) {
  const int i0 = B.x * BX, j0 = B.y * BY, k0 = B.z * CHEB3_KZ;
  const int i = i0 + threadIdx.x;
  const int j = j0 + threadIdx.y;
  const bool inner = i0 >= 3 && i0 + BX - 1 <= L.n[0] - 3 && j0 >= 3 && j0 + BY - 1 <= L.n[1] - 3 && k0 >= 3 &&
                     k0 + CHEB3_KZ - 1 <= L.n[2] - 3;
  const int P = L.P, S = (int)L.S;
  if (inner) {
#pragma unroll
    for (int kk = 0; kk < CHEB3_KZ; ++kk) {
      const int p0 = (k0 + kk) * S + j * P + i;
      cheb3_face<T, 0, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[0][q]; });
      cheb3_face<T, 1, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[1][q]; });
      cheb3_face<T, 2, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[2][q]; });
    }
    return;
  }
  if (i > L.n[0] || j > L.n[1]) return;
  const int cxy = (cls7(i, L.n[0]) * 7 + cls7(j, L.n[1])) * 7;
  for (int kk = 0; kk < CHEB3_KZ; ++kk) {
    const int k = k0 + kk;
    if (k > L.n[2]) break;
    const int pc = cxy + cls7(k, L.n[2]);
    const int p0 = k * S + j * P + i;
    const T* fold = table + FOLD3_OFF + (size_t)pc * 48;
    if (pc == FOLD3_INTERIOR) {
      cheb3_face<T, 0, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[0][q]; });
      cheb3_face<T, 1, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[1][q]; });
      cheb3_face<T, 2, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[2][q]; });
      continue;
    }
    if (in_store<0>(L, i, j, k) && face_active<0>(L, i, j, k))
      cheb3_face<T, 0, false>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return GKB_LDG(fold + q); });
    if (in_store<1>(L, i, j, k) && face_active<1>(L, i, j, k))
      cheb3_face<T, 1, false>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return GKB_LDG(fold + 16 + q); });
    if (in_store<2>(L, i, j, k) && face_active<2>(L, i, j, k))
      cheb3_face<T, 2, false>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return GKB_LDG(fold + 32 + q); });
  }
}

// the launch grid of k_cheb3: 32 x 8 positions per block, CHEB3_KZ planes
inline dim3 cheb3_grid(const Lvl& L) {
  return dim3((L.n[0] + 1 + BX - 1) / BX, (L.n[1] + 1 + BY - 1) / BY, (L.n[2] + 1 + CHEB3_KZ - 1) / CHEB3_KZ);
}

// ---- 2D constant viscosity: folded stencils for every position class ------
// The same construction with one orientation (vertex patches, E = 2): per
// (position class, component) a 7-point stencil, the face itself and the six
// other faces of its two patches, after FOLD3_OFF with the 3D layout (48
// entries per class, 16 per component).
constexpr int FOLD2_CLASSES = 49;
constexpr int FOLD2_INTERIOR = 3 * 7 + 3;

template <typename T>
__global__ void k_fold2_table(Lvl L, T* table) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (L.dim != 2 || t >= FOLD2_CLASSES * 2) return;
  const int C = t % 2, pc = t / 2;
  const int p[3] = {rep7(pc / 7, L.n[0]), rep7(pc % 7, L.n[1]), 0};
  double acc[13];
#pragma unroll
  for (int q = 0; q < 13; ++q) acc[q] = 0.0;
  fold3_orient<T, 2>(L, table, p, C, acc, 1);
  T* f = table + FOLD3_OFF + (size_t)pc * 48 + C * 16;
  for (int q = 0; q < 16; ++q) f[q] = q < 7 ? (T)acc[q] : (T)0;
}

// the interior class's 2D stencils scaled by the Chebyshev step's ca, as a
// kernel parameter
template <typename T>
struct Fold2In {
  T c[2][7];
};

// (C r) at an active face of component C by the 7-point stencil f (2D);
// Inner == false reads only faces with nonzero coefficients
template <typename T, int C, bool Inner, class Coef>
__device__ __forceinline__ T fold2_apply(const Lvl& L, const T* GKB_RESTRICT r, int cb, Coef f) {
  const int P = L.P;
  const T* ra = r + L.off[0] + cb;
  const T* rb = r + L.off[1] + cb;
  T acc = f(0) * GKB_LDG(C == 0 ? ra : rb);
  const T* base[6];
  int o[6];
  if (C == 0) {
    base[0] = ra; o[0] = -P; base[1] = rb; o[1] = -1; base[2] = rb; o[2] = 0;
    base[3] = ra; o[3] = P; base[4] = rb; o[4] = P - 1; base[5] = rb; o[5] = P;
  } else {
    base[0] = ra; o[0] = -P; base[1] = ra; o[1] = 0; base[2] = rb; o[2] = -1;
    base[3] = ra; o[3] = 1 - P; base[4] = ra; o[4] = 1; base[5] = rb; o[5] = 1;
  }
#pragma unroll
  for (int u = 0; u < 6; ++u) {
    const T c = f(1 + u);
    if (Inner || c != (T)0) acc += c * GKB_LDG(base[u] + o[u]);
  }
  return acc;
}

// one Chebyshev step of the 2D constant-viscosity smoother through the class
// stencils (levels with at least six cells per axis). Blocks whose positions
// are all interior use the kernel parameter's stencils, already scaled by
// ca (d = z + cb d); the others each position's class stencil from the table.
template <typename T>
__device__ __forceinline__ void cheb2_body(const Blk& B, const Lvl& L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                           T* GKB_RESTRICT d, T ca, T cb, int x_zero, const T* GKB_RESTRICT table,
                                           const Fold2In<T>& fs) {
  const int i0 = B.x * BX, j0 = B.y * BY;
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const int P = L.P;
  if (i0 >= 3 && i0 + BX - 1 <= L.n[0] - 3 && j0 >= 3 && j0 + BY - 1 <= L.n[1] - 3) {
    const int p0 = j * P + i;
#define GKB_CHEB2_IN(C)                                                                  \
    {                                                                                    \
      const int id = (int)L.off[C] + p0;                                                 \
      const T dold = (cb != (T)0) ? d[id] : (T)0;                                        \
      const T xold = x_zero ? (T)0 : x[id];                                              \
      const T zs = fold2_apply<T, C, true>(L, r, p0, [&](int q) { return fs.c[C][q]; }); \
      const T dn = (cb != (T)0) ? fma(cb, dold, zs) : zs;                                \
      d[id] = dn;                                                                        \
      x[id] = x_zero ? dn : xold + dn;                                                   \
    }
    GKB_CHEB2_IN(0)
    GKB_CHEB2_IN(1)
#undef GKB_CHEB2_IN
    return;
  }
  if (i > L.n[0] || j > L.n[1]) return;
  const int pc = cls7(i, L.n[0]) * 7 + cls7(j, L.n[1]);
  const int p0 = j * P + i;
  const T* fold = table + FOLD3_OFF + (size_t)pc * 48;
#define GKB_CHEB2(C)                                                                              \
  if (in_store<C>(L, i, j, 0) && face_active<C>(L, i, j, 0)) {                                    \
    const int id = (int)L.off[C] + p0;                                                            \
    const T dold = (cb != (T)0) ? d[id] : (T)0;                                                   \
    const T xold = x_zero ? (T)0 : x[id];                                                         \
    const T z = fold2_apply<T, C, false>(L, r, p0, [&](int q) { return GKB_LDG(fold + C * 16 + q); }); \
    const T dn = (cb != (T)0) ? ca * z + cb * dold : ca * z;                                      \
    d[id] = dn;                                                                                   \
    x[id] = x_zero ? dn : xold + dn;                                                              \
  }
  GKB_CHEB2(0)
  GKB_CHEB2(1)
#undef GKB_CHEB2
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_cheb2(Lvl L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                                   T* GKB_RESTRICT d, T ca, T cb, int x_zero, const T* table,
                                                   const __grid_constant__ Fold2In<T> fs) {
  cheb2_body<T>(native_blk(), L, r, x, d, ca, cb, x_zero, table, fs);
}

inline bool cheb2_level(const Lvl& L) { return L.dim == 2 && L.fast && L.n[0] >= 6 && L.n[1] >= 6; }

// the interior stencils of a 2D level (host copy, 2 x 16 values) scaled by ca
template <typename T>
inline Fold2In<T> fold2_scaled(const double* fold_in, double ca) {
  Fold2In<T> f;
  for (int c = 0; c < 2; ++c)
    for (int q = 0; q < 7; ++q) f.c[c][q] = (T)(ca * fold_in[c * 16 + q]);
  return f;
}

// the class stencils serve 3D constant-viscosity levels with the fast paths
// on and at least six cells on every axis
inline bool cheb3_level(const Lvl& L) {
  return L.dim == 3 && L.fast && L.n[0] >= 6 && L.n[1] >= 6 && L.n[2] >= 6;
}
inline bool cheb3_applies(const Lvl& L, const void* table) { return table != nullptr && cheb3_level(L); }

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_cheb3(Lvl L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                                   T* GKB_RESTRICT d, T ca, T cb, int x_zero, const T* table,
                                                   const __grid_constant__ Fold3In<T> fin) {
  cheb3_body<T>(native_blk(), L, r, x, d, ca, cb, x_zero, table, fin);
}

// ---------------------------------------------------------------------------
// The same step split by geometry (levels of at least 16 cells per axis): the
// box [3, n-3]^3, where every position is of the interior class, walks planes
// like k_mac3's box (r of three planes with a one-position halo in shared
// memory; r, d and x of the next plane fetched into registers while the
// current one is computed) and applies the interior stencils in
// fold3_apply's order; the shell (three positions deep, the extra z slices of
// the same launch) takes the class table one thread per position. The same
// operations as k_cheb3 for every face.
// ---------------------------------------------------------------------------
constexpr int CHEB3S_KZ = 16;

inline bool cheb3s_level(const Lvl& L) {
  return L.dim == 3 && L.n[0] >= 16 && L.n[1] >= 16 && L.n[2] >= 16;
}
__host__ __device__ __forceinline__ int cheb3s_box_z(const Lvl& L) { return (L.n[2] - 5 + CHEB3S_KZ - 1) / CHEB3S_KZ; }
inline dim3 cheb3s_grid(const Lvl& L) {
  const unsigned gx = (L.n[0] - 5 + BX - 1) / BX, gy = (L.n[1] - 5 + BY - 1) / BY;
  const long long per_slice = (long long)gx * gy * BX * BY;
  return dim3(gx, gy, cheb3s_box_z(L) + (unsigned)((shell_count(L, 3, 3) + per_slice - 1) / per_slice));
}

// fold3_apply's interior stencil of component C at tile position (tx, ty)
// of plane slot s0 (planes below / above: sm, sp)
template <typename T, int C>
__device__ __forceinline__ T fold3_tile(const T (*Rt)[3][BY + 2][BX + 2], int sm, int s0, int sp, int tx, int ty,
                                        const T* f) {
  auto R = [&](int comp, const int dl[3]) -> T {
    return Rt[dl[2] < 0 ? sm : (dl[2] > 0 ? sp : s0)][comp][ty + 1 + dl[1]][tx + 1 + dl[0]];
  };
  const int z0[3] = {0, 0, 0};
  T acc = f[0] * R(C, z0);
  int t = 1;
#pragma unroll
  for (int E = 0; E < 3; ++E) {
    if (E == C) continue;
    const int a = (E == 0) ? 1 : 0, b = (E == 2) ? 1 : 2;
    int mb[3] = {0, 0, 0}, ma[3] = {0, 0, 0}, pb[3] = {0, 0, 0}, pa[3] = {0, 0, 0}, ba[3] = {0, 0, 0}, ab[3] = {0, 0, 0};
    mb[b] = -1; ma[a] = -1; pb[b] = 1; pa[a] = 1; ba[b] = 1; ba[a] = -1; ab[a] = 1; ab[b] = -1;
    if (C == a) {
      acc += f[t + 0] * R(a, mb);
      acc += f[t + 1] * R(b, ma);
      acc += f[t + 2] * R(b, z0);
      acc += f[t + 3] * R(a, pb);
      acc += f[t + 4] * R(b, ba);
      acc += f[t + 5] * R(b, pb);
    } else {
      acc += f[t + 0] * R(a, mb);
      acc += f[t + 1] * R(a, z0);
      acc += f[t + 2] * R(b, ma);
      acc += f[t + 3] * R(a, ab);
      acc += f[t + 4] * R(a, pa);
      acc += f[t + 5] * R(b, pa);
    }
    t += 6;
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ void cheb3s_box_body(const Blk& B, const Lvl& L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                                T* GKB_RESTRICT d, T ca, T cb, int x_zero, const Fold3In<T>& fin) {
  constexpr int TW = BX + 2, TH = BY + 2;
  __shared__ T Rt[3][3][TH][TW];   // [plane slot][component][row][col]: position (i0-1+col, j0-1+row)
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int i0 = 3 + (int)B.x * BX, j0 = 3 + (int)B.y * BY, k0 = 3 + (int)B.z * CHEB3S_KZ;
  const int i = i0 + tx, j = j0 + ty;
  const int kend = min(k0 + CHEB3S_KZ, L.n[2] - 2);  // planes k0 .. kend-1 (uniform over the block)
  const bool mine = i <= L.n[0] - 3 && j <= L.n[1] - 3;
  auto slot = [](int k) { return k % 3; };
  // tile entries as in k_mac3's box (planes k0-1 .. kend lie in [2, n-2])
  constexpr int HALO = 2 * TW + 2 * BY;
  const bool tin0 = i0 - 1 + tx <= L.n[0] && j0 - 1 + ty <= L.n[1];
  int hc = 0, hr = 0, hq = 0;
  bool hin = false;
  if (tid < 3 * HALO) {
    hc = tid / HALO;
    const int h = tid - hc * HALO;
    if (h < 2 * TW) { hr = BY + h / TW; hq = h - (hr - BY) * TW; }
    else { hr = (h - 2 * TW) >> 1; hq = BX + ((h - 2 * TW) & 1); }
    hin = i0 - 1 + hq <= L.n[0] && j0 - 1 + hr <= L.n[1];
  }
  const T* rp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) rp[c] = r + L.off[c] + cix(L, i0 - 1 + tx, j0 - 1 + ty, k0 - 1);
  const T* rh = r + L.off[hc] + cix(L, i0 - 1 + hq, j0 - 1 + hr, k0 - 1);
  T pre[3], preh = (T)0;
  auto fetch = [&]() {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pre[c] = tin0 ? *rp[c] : (T)0;
      rp[c] += L.S;
    }
    if (tid < 3 * HALO) {
      preh = hin ? *rh : (T)0;
      rh += L.S;
    }
  };
  auto commit = [&](int k) {
    const int sl = slot(k);
#pragma unroll
    for (int c = 0; c < 3; ++c) Rt[sl][c][ty][tx] = pre[c];
    if (tid < 3 * HALO) Rt[sl][hc][hr][hq] = preh;
  };
  fetch();
  commit(k0 - 1);
  fetch();
  commit(k0);
  fetch();
  long long cbk = cix(L, i, j, k0);
  // d and x of the faces: those of plane k+1 are fetched while plane k is
  // computed
  T dnx[3] = {(T)0, (T)0, (T)0}, xnx[3] = {(T)0, (T)0, (T)0};
  auto fetch_dx = [&](long long at) {
    if (mine) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (cb != (T)0) dnx[c] = d[L.off[c] + at];
        if (!x_zero) xnx[c] = x[L.off[c] + at];
      }
    }
  };
  fetch_dx(cbk);
  for (int k = k0; k < kend; ++k, cbk += L.S) {
    commit(k + 1);
    if (k + 1 < kend) fetch();
    T dold[3], xold[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dold[c] = dnx[c];
      xold[c] = xnx[c];
    }
    if (k + 1 < kend) fetch_dx(cbk + L.S);
    __syncthreads();
    if (mine) {
      const int sc = slot(k), su = slot(k + 1), sd = slot(k - 1);
#define GKB_CHEB3S_FACE(C)                                                                     \
      {                                                                                        \
        const T z = fold3_tile<T, C>(Rt, sd, sc, su, tx, ty, fin.c[C]);                         \
        const T dn = (cb != (T)0) ? ca * z + cb * dold[C] : ca * z;                            \
        d[L.off[C] + cbk] = dn;                                                                \
        x[L.off[C] + cbk] = x_zero ? dn : xold[C] + dn;                                        \
      }
      GKB_CHEB3S_FACE(0)
      GKB_CHEB3S_FACE(1)
      GKB_CHEB3S_FACE(2)
#undef GKB_CHEB3S_FACE
    }
    __syncthreads();  // the next plane's load overwrites slot k-1
  }
}

// one position of the shell [3, n-3]: the class path of cheb3_body
template <typename T>
__device__ __forceinline__ void cheb3s_shell_body(const Lvl& L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                                  T* GKB_RESTRICT d, T ca, T cb, int x_zero,
                                                  const T* GKB_RESTRICT table, const Fold3In<T>& fin, long long t) {
  if (t >= shell_count(L, 3, 3)) return;
  int i, j, k;
  shell_ijk(L, 3, 3, t, i, j, k);
  const int pc = (cls7(i, L.n[0]) * 7 + cls7(j, L.n[1])) * 7 + cls7(k, L.n[2]);
  const int p0 = k * (int)L.S + j * L.P + i;
  const T* fold = table + FOLD3_OFF + (size_t)pc * 48;
  if (pc == FOLD3_INTERIOR) {
    cheb3_face<T, 0, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[0][q]; });
    cheb3_face<T, 1, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[1][q]; });
    cheb3_face<T, 2, true>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return fin.c[2][q]; });
    return;
  }
  if (in_store<0>(L, i, j, k) && face_active<0>(L, i, j, k))
    cheb3_face<T, 0, false>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return GKB_LDG(fold + q); });
  if (in_store<1>(L, i, j, k) && face_active<1>(L, i, j, k))
    cheb3_face<T, 1, false>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return GKB_LDG(fold + 16 + q); });
  if (in_store<2>(L, i, j, k) && face_active<2>(L, i, j, k))
    cheb3_face<T, 2, false>(L, r, x, d, ca, cb, x_zero, p0, [&](int q) { return GKB_LDG(fold + 32 + q); });
}

template <typename T>
__global__ void __launch_bounds__(BX* BY, sizeof(T) == 8 ? 2 : 4) k_cheb3s(Lvl L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                                      T* GKB_RESTRICT d, T ca, T cb, int x_zero, const T* table,
                                                      const __grid_constant__ Fold3In<T> fin) {
  const int bz = cheb3s_box_z(L);
  if ((int)blockIdx.z < bz) {
    cheb3s_box_body<T>(native_blk(), L, r, x, d, ca, cb, x_zero, fin);
  } else {
    const long long blk = ((long long)(blockIdx.z - bz) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    cheb3s_shell_body<T>(L, r, x, d, ca, cb, x_zero, table, fin, blk * (BX * BY) + threadIdx.y * BX + threadIdx.x);
  }
}

// One Chebyshev step of the patch-preconditioned smoother:
//   z = C r;  d = ca * z + cb * d;  x = (x_zero ? 0 : x) + d
template <typename T, bool VarMu>
__device__ __forceinline__ void cheb_body(const Blk& B, const Lvl& L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                                  T* GKB_RESTRICT d, T ca, T cb, int x_zero, const T* table) {
  int tx, ty;
  block_xy(L, tx, ty);
  const int i = B.x * BX + tx;
  const int j = B.y * BY + ty;
  const int k = B.z;
  const int p[3] = {i, j, k};
  const long long pc = cix(L, i, j, k);
  if (!VarMu && table != nullptr && deep_interior(L, i, j, k)) {
#define GKB_CHEB_DEEP(C)                                                         \
    {                                                                            \
      const long long id = L.off[C] + pc;                                        \
      const T z = (L.dim == 3) ? patch_apply_fold<T, C>(L, r, pc, table + PATCH_FOLD_OFF) \
                               : patch_apply_deep<T, C>(L, r, pc, table);        \
      const T dn = (cb != (T)0) ? ca * z + cb * d[id] : ca * z;                  \
      d[id] = dn;                                                                \
      x[id] = x_zero ? dn : x[id] + dn;                                          \
    }
    GKB_CHEB_DEEP(0)
    GKB_CHEB_DEEP(1)
    if (L.dim == 3) { GKB_CHEB_DEEP(2) }
#undef GKB_CHEB_DEEP
    return;
  }
#define GKB_CHEB_COMP(C)                                                         \
  if (in_store<C>(L, i, j, k) && face_active<C>(L, i, j, k)) {                   \
    const long long id = L.off[C] + pc;                                          \
    const T z = patch_apply<T, VarMu, C>(L, r, p, pc, table);                    \
    const T dn = (cb != (T)0) ? ca * z + cb * d[id] : ca * z;                    \
    d[id] = dn;                                                                  \
    x[id] = x_zero ? dn : x[id] + dn;                                            \
  }
  GKB_CHEB_COMP(0)
  GKB_CHEB_COMP(1)
  if (L.dim == 3) { GKB_CHEB_COMP(2) }
#undef GKB_CHEB_COMP
}

template <typename T, bool VarMu>
__global__ void __launch_bounds__(BX* BY) k_cheb(Lvl L, const T* GKB_RESTRICT r, T* GKB_RESTRICT x,
                                                  T* GKB_RESTRICT d, T ca, T cb, int x_zero, const T* table) {
  cheb_body<T, VarMu>(native_blk(), L, r, x, d, ca, cb, x_zero, table);
}

// z = C r (power iteration, tests)
template <typename T, bool VarMu>
__global__ void __launch_bounds__(BX* BY) k_patch(Lvl L, const T* GKB_RESTRICT r, T* GKB_RESTRICT z, const T* table) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p[3] = {i, j, k};
  const long long cb = cix(L, i, j, k);
#define GKB_PATCH_COMP(C)                                                        \
  if (in_store<C>(L, i, j, k)) {                                                 \
    const long long id = L.off[C] + cb;                                          \
    z[id] = face_active<C>(L, i, j, k) ? patch_apply<T, VarMu, C>(L, r, p, cb, table) : (T)0; \
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

// Node (2D) / edge (3D) viscosity table of a variable-viscosity level: one
// thread per position (e0, e1, e2) with e0 <= n0, e1 <= n1, e2 <= n2 (3D);
// orientation E takes the positions with node coordinates along its two
// other axes and a cell coordinate along E.
template <typename T>
__global__ void k_edge_mu(Lvl L, T* GKB_RESTRICT em) {
  const int e[3] = {(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(blockIdx.y * blockDim.y + threadIdx.y),
                    (int)blockIdx.z};
  if (e[0] > L.n[0] || e[1] > L.n[1]) return;
  const long long Q = em_plane(L), id = cix(L, e[0], e[1], e[2]);
  if (L.dim == 2) {
    em[id] = edge_mu_cells<T, 0, 1>(L, e, e[1]);
    return;
  }
  if (e[2] < L.n[2]) em[2 * Q + id] = edge_mu_cells<T, 0, 1>(L, e, e[1]);
  if (e[0] < L.n[0]) em[0 * Q + id] = edge_mu_cells<T, 1, 2>(L, e, e[2]);
  if (e[1] < L.n[1]) em[1 * Q + id] = edge_mu_cells<T, 0, 2>(L, e, e[2]);
}

// Per-patch inverses for variable viscosity (one thread per edge of
// orientation E; e[a] in [0, n_a], e[b] in [0, n_b], e[E] in [0, n_E - 1]):
// the patch matrix in the level's precision, Gauss-Jordan in FP64.
template <typename T, int E>
__global__ void k_patch_vtab(Lvl L, T* GKB_RESTRICT vtab) {
  constexpr int a = EAx<E>::a, b = EAx<E>::b;
  const int e[3] = {(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(blockIdx.y * blockDim.y + threadIdx.y),
                    (int)blockIdx.z};
  if (e[a] > L.n[a] || e[b] > L.n[b]) return;
  if (L.dim == 3 && e[E] >= L.n[E]) return;
  T Mt[4][4];
  bool act[4];
  patch_matrix<T, true, E>(L, e, Mt, act);
  double Mp[4][4], inv[4][4];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      Mp[r][c] = (double)Mt[r][c];
      inv[r][c] = (r == c) ? 1.0 : 0.0;
    }
  for (int c = 0; c < 4; ++c) {
    const double piv = 1.0 / Mp[c][c];
    for (int k2 = 0; k2 < 4; ++k2) { Mp[c][k2] *= piv; inv[c][k2] *= piv; }
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const double f = Mp[r][c];
      for (int k2 = 0; k2 < 4; ++k2) { Mp[r][k2] -= f * Mp[c][k2]; inv[r][k2] -= f * inv[c][k2]; }
    }
  }
  const long long Q = vtab_plane(L);
  T* t = vtab + (size_t)(L.dim == 3 ? E : 0) * 10 * Q + cix(L, e[0], e[1], e[2]);
  for (int r = 0; r < 4; ++r)
    for (int c = r; c < 4; ++c)
      t[(long long)sym4(r, c) * Q] = (act[r] && act[c]) ? (T)(0.5 * (inv[r][c] + inv[c][r])) : (T)0;
}

// ---------------------------------------------------------------------------
// gradient / divergence
// ---------------------------------------------------------------------------

// y = s * A p  (faces from cells): y_f = s * ascale * (p_plus - p_minus)
template <typename T>
__device__ __forceinline__ void grad_body(const Blk& B, const Lvl& L, const T* GKB_RESTRICT pc, T* GKB_RESTRICT y, T s) {
  const int i = B.x * BX + threadIdx.x;
  const int j = B.y * BY + threadIdx.y;
  const int k = B.z;
  const T sc = s * Kc<T>::as(L);
#define GKB_GRAD_COMP(C, DI, DJ, DK)                                             \
  if (in_store<C>(L, i, j, k)) {                                                 \
    const long long id = L.off[C] + cix(L, i, j, k);                             \
    T val = 0;                                                                   \
    if (face_active<C>(L, i, j, k)) {                                            \
      const T pp = cell_in(L, i, j, k) ? GKB_LDG(pc + cix(L, i, j, k)) : (T)0;     \
      const T pm = cell_in(L, i - DI, j - DJ, k - DK) ? GKB_LDG(pc + cix(L, i - DI, j - DJ, k - DK)) : (T)0; \
      val = sc * (pp - pm);                                                      \
    }                                                                            \
    y[id] = val;                                                                 \
  }
  GKB_GRAD_COMP(0, 1, 0, 0)
  GKB_GRAD_COMP(1, 0, 1, 0)
  if (L.dim == 3) { GKB_GRAD_COMP(2, 0, 0, 1) }
#undef GKB_GRAD_COMP
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_grad(Lvl L, const T* GKB_RESTRICT pc, T* GKB_RESTRICT y, T s) {
  grad_body<T>(native_blk(), L, pc, y, s);
}

// y = s * A^T x  (cells from faces) = s * ascale * negdiv(x); padding untouched
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_negdiv(Lvl L, const T* GKB_RESTRICT x, T* GKB_RESTRICT y, T s) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= L.n[0] || j >= L.n[1]) return;
  y[cix(L, i, j, k)] = s * Kc<T>::as(L) * neg_div<T>(L, x, i, j, k);
}

// ---------------------------------------------------------------------------
// grid transfer helpers
// ---------------------------------------------------------------------------

template <typename T, int C>
__device__ __forceinline__ T coarse_face(const Lvl& Lc, const T* xc, int I, int J, int K) {
  if (!face_active<C>(Lc, I, J, K)) return (T)0;
  return GKB_LDG(xc + Lc.off[C] + cix(Lc, I, J, K));
}

template <typename T, int C>
__device__ __forceinline__ T fine_face(const Lvl& Lf, const T* rf, int i, int j, int k) {
  if (!face_active<C>(Lf, i, j, k)) return (T)0;
  return GKB_LDG(rf + Lf.off[C] + cix(Lf, i, j, k));
}

// ---- 2D flux-conserving, divergence-preserving transfers -----------------
// Prolongation of a coarse face field U (component C, tangential axis t):
//   fine faces on a coarse face line (normal index 2I):  U(I,q) + s D(I,q),
//     q = tangential fine index / 2, s = -1 / +1 for the lower / upper fine
//     face, D(I,q) = (U(I,q+1) - U(I,q-1)) / 8 (tangential slope; no-slip
//     mirror U(ghost) = -U(inside) across walls), so both fine faces carry
//     the coarse flux;
//   fine faces inside a coarse cell (normal index 2I+1): the mean of the two
//     line values above plus (D'(line q+1) - D'(line q)) / 2, D' the slopes
//     of the other component on the two faces of that coarse cell. The last
//     term is the minimal-norm correction that makes the divergence of every
//     fine cell equal to that of its coarse cell.
// Restriction is the exact transpose, in two passes: a gather of the fine
// residual into (rU, rD) per coarse face, then rU + G^T rD.

template <typename T, int C>
__device__ __forceinline__ T coarse_slope(const Lvl& Lc, const T* xc, int I, int J) {
  constexpr int t = 1 - C;
  int P[3] = {I, J, 0};
  if (!face_active<C>(Lc, P[0], P[1], 0)) return (T)0;
  const T u0 = GKB_LDG(xc + Lc.off[C] + cix(Lc, P[0], P[1], 0));
  int Pp[3] = {P[0], P[1], 0}, Pm[3] = {P[0], P[1], 0};
  Pp[t] += 1;
  Pm[t] -= 1;
  const T up = (Pp[t] < Lc.n[t]) ? coarse_face<T, C>(Lc, xc, Pp[0], Pp[1], 0) : -u0;
  const T um = (Pm[t] >= 0) ? coarse_face<T, C>(Lc, xc, Pm[0], Pm[1], 0) : -u0;
  return (up - um) * (T)0.125;
}

template <typename T, int C>
__device__ __forceinline__ T prolong_flux_val(const Lvl& Lc, const T* xc, int pc, int pt) {
  constexpr int t = 1 - C, Co = 1 - C;
  const int q = pt >> 1;
  const T s = (pt & 1) ? (T)1 : (T)-1;
  auto line_val = [&](int I) -> T {
    int P[3] = {0, 0, 0};
    P[C] = I;
    P[t] = q;
    return coarse_face<T, C>(Lc, xc, P[0], P[1], 0) + s * coarse_slope<T, C>(Lc, xc, P[0], P[1]);
  };
  if ((pc & 1) == 0) return line_val(pc >> 1);
  const int I = pc >> 1;
  int P0[3] = {0, 0, 0}, P1[3] = {0, 0, 0};
  P0[C] = I; P0[t] = q;        // other component's face on tangential line q
  P1[C] = I; P1[t] = q + 1;    // ... and on line q + 1
  const T fix = (T)0.5 * (coarse_slope<T, Co>(Lc, xc, P1[0], P1[1]) - coarse_slope<T, Co>(Lc, xc, P0[0], P0[1]));
  return (T)0.5 * (line_val(I) + line_val(I + 1)) + fix;
}

// xf += P xc (2D), one thread per coarse cell (I, J): the cell's left and
// bottom coarse faces and their tangential slopes are formed once and give
// its 2 x 2 fine u faces (fine columns 2I, 2I+1) and v faces (fine rows 2J,
// 2J+1) with the operations of prolong_flux_val; the extra column I = n_x
// and row J = n_y of threads take the fine faces on the last coarse lines.
template <typename T>
__device__ __forceinline__ void prolong_flux2d_body(const Blk& B, const Lvl& Lf, const Lvl& Lc, const T* GKB_RESTRICT xc, T* GKB_RESTRICT xf) {
  const int I = B.x * BX + threadIdx.x;
  const int J = B.y * BY + threadIdx.y;
  if (I > Lc.n[0] || J > Lc.n[1]) return;
  const bool inx = I < Lc.n[0], iny = J < Lc.n[1];
  auto add = [&](int C, int i, int j, T v) {
    if (C == 0 ? (in_store<0>(Lf, i, j, 0) && face_active<0>(Lf, i, j, 0))
               : (in_store<1>(Lf, i, j, 0) && face_active<1>(Lf, i, j, 0)))
      xf[Lf.off[C] + cix(Lf, i, j, 0)] += v;
  };
  // u slopes (along y) on the cell's left and right faces, v slopes (along x)
  // on its bottom and top faces
  const T du0 = iny ? coarse_slope<T, 0>(Lc, xc, I, J) : (T)0;
  const T du1 = (iny && inx) ? coarse_slope<T, 0>(Lc, xc, I + 1, J) : (T)0;
  const T dv0 = inx ? coarse_slope<T, 1>(Lc, xc, I, J) : (T)0;
  const T dv1 = (inx && iny) ? coarse_slope<T, 1>(Lc, xc, I, J + 1) : (T)0;
  if (iny) {
    const T u0 = coarse_face<T, 0>(Lc, xc, I, J, 0);
    const T lo0 = u0 + (T)-1 * du0, hi0 = u0 + (T)1 * du0;  // coarse line I at fine rows 2J, 2J+1
    add(0, 2 * I, 2 * J, lo0);
    add(0, 2 * I, 2 * J + 1, hi0);
    if (inx) {
      const T u1 = coarse_face<T, 0>(Lc, xc, I + 1, J, 0);
      const T lo1 = u1 + (T)-1 * du1, hi1 = u1 + (T)1 * du1;
      const T fix = (T)0.5 * (dv1 - dv0);
      add(0, 2 * I + 1, 2 * J, (T)0.5 * (lo0 + lo1) + fix);
      add(0, 2 * I + 1, 2 * J + 1, (T)0.5 * (hi0 + hi1) + fix);
    }
  }
  if (inx) {
    const T v0 = coarse_face<T, 1>(Lc, xc, I, J, 0);
    const T lo0 = v0 + (T)-1 * dv0, hi0 = v0 + (T)1 * dv0;  // coarse line J at fine columns 2I, 2I+1
    add(1, 2 * I, 2 * J, lo0);
    add(1, 2 * I + 1, 2 * J, hi0);
    if (iny) {
      const T v1 = coarse_face<T, 1>(Lc, xc, I, J + 1, 0);
      const T lo1 = v1 + (T)-1 * dv1, hi1 = v1 + (T)1 * dv1;
      const T fix = (T)0.5 * (du1 - du0);
      add(1, 2 * I, 2 * J + 1, (T)0.5 * (lo0 + lo1) + fix);
      add(1, 2 * I + 1, 2 * J + 1, (T)0.5 * (hi0 + hi1) + fix);
    }
  }
}

// launch grid of the 2D prolongation: the coarse cells plus one column and row
inline dim3 prolong2d_grid(const Lvl& Lc) {
  return dim3((Lc.n[0] + 1 + BX - 1) / BX, (Lc.n[1] + 1 + BY - 1) / BY, 1);
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_prolong_flux2d(Lvl Lf, Lvl Lc, const T* GKB_RESTRICT xc, T* GKB_RESTRICT xf) {
  prolong_flux2d_body<T>(native_blk(), Lf, Lc, xc, xf);
}

template <typename T, int C>
__device__ __forceinline__ T fine_at(const Lvl& Lf, const T* rf, int pc, int pt) {
  constexpr int t = 1 - C;
  int P[3] = {0, 0, 0};
  P[C] = pc;
  P[t] = pt;
  return fine_face<T, C>(Lf, rf, P[0], P[1], 0);
}

template <typename T, int C>
__device__ __forceinline__ void restrict_flux_gather(const Lvl& Lf, const T* rf, int Ic, int q, T& rU, T& rD) {
  constexpr int Co = 1 - C;
  T su = 0, sd = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int nn = (k == 0) ? 2 * Ic : (k == 1) ? 2 * Ic + 1 : 2 * Ic - 1;
    const T w = (k == 0) ? (T)1 : (T)0.5;
    const T lo = fine_at<T, C>(Lf, rf, nn, 2 * q);
    const T hi = fine_at<T, C>(Lf, rf, nn, 2 * q + 1);
    su += w * (lo + hi);
    sd += w * (hi - lo);
  }
  // the other component's fine faces inside the coarse cells on either side
  // (their divergence correction uses this face's slope)
  sd += (T)-0.5 * (fine_at<T, Co>(Lf, rf, 2 * q + 1, 2 * Ic) + fine_at<T, Co>(Lf, rf, 2 * q + 1, 2 * Ic + 1));
  sd += (T)0.5 * (fine_at<T, Co>(Lf, rf, 2 * q + 1, 2 * Ic - 2) + fine_at<T, Co>(Lf, rf, 2 * q + 1, 2 * Ic - 1));
  rU = su;
  rD = sd;
}

// pass a: bc = rU, tmp = rD  (launched over the coarse face grid)
template <typename T>
__device__ __forceinline__ void restrict_flux2d_a_body(const Blk& B, const Lvl& Lf, const Lvl& Lc, const T* GKB_RESTRICT rf,
                                                               T* GKB_RESTRICT bc, T* GKB_RESTRICT tmp) {
  const int I = B.x * BX + threadIdx.x;
  const int J = B.y * BY + threadIdx.y;
  if (in_store<0>(Lc, I, J, 0)) {
    const long long id = Lc.off[0] + cix(Lc, I, J, 0);
    T rU = 0, rD = 0;
    if (face_active<0>(Lc, I, J, 0)) restrict_flux_gather<T, 0>(Lf, rf, I, J, rU, rD);
    bc[id] = rU;
    tmp[id] = rD;
  }
  if (in_store<1>(Lc, I, J, 0)) {
    const long long id = Lc.off[1] + cix(Lc, I, J, 0);
    T rU = 0, rD = 0;
    if (face_active<1>(Lc, I, J, 0)) restrict_flux_gather<T, 1>(Lf, rf, J, I, rU, rD);
    bc[id] = rU;
    tmp[id] = rD;
  }
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_restrict_flux2d_a(Lvl Lf, Lvl Lc, const T* GKB_RESTRICT rf,
                                                               T* GKB_RESTRICT bc, T* GKB_RESTRICT tmp) {
  restrict_flux2d_a_body<T>(native_blk(), Lf, Lc, rf, bc, tmp);
}

// pass b: bc += G^T tmp (transpose of the tangential slope, mirror walls)
template <typename T, int C>
__device__ __forceinline__ T slope_transpose(const Lvl& Lc, const T* d, int I, int J) {
  constexpr int t = 1 - C;
  int P[3] = {I, J, 0};
  const int q = P[t], Nt = Lc.n[t];
  T acc = 0;
  int Q[3] = {P[0], P[1], 0};
  if (q - 1 >= 0) { Q[t] = q - 1; acc += GKB_LDG(d + Lc.off[C] + cix(Lc, Q[0], Q[1], 0)); }
  if (q + 1 < Nt) { Q[t] = q + 1; acc -= GKB_LDG(d + Lc.off[C] + cix(Lc, Q[0], Q[1], 0)); }
  const T own = GKB_LDG(d + Lc.off[C] + cix(Lc, I, J, 0));
  if (q == 0) acc += own;
  if (q == Nt - 1) acc -= own;
  return acc * (T)0.125;
}

template <typename T>
__device__ __forceinline__ void restrict_flux2d_b_body(const Blk& B, const Lvl& Lc, const T* GKB_RESTRICT tmp, T* GKB_RESTRICT bc) {
  const int I = B.x * BX + threadIdx.x;
  const int J = B.y * BY + threadIdx.y;
  if (in_store<0>(Lc, I, J, 0) && face_active<0>(Lc, I, J, 0))
    bc[Lc.off[0] + cix(Lc, I, J, 0)] += slope_transpose<T, 0>(Lc, tmp, I, J);
  if (in_store<1>(Lc, I, J, 0) && face_active<1>(Lc, I, J, 0))
    bc[Lc.off[1] + cix(Lc, I, J, 0)] += slope_transpose<T, 1>(Lc, tmp, I, J);
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_restrict_flux2d_b(Lvl Lc, const T* GKB_RESTRICT tmp, T* GKB_RESTRICT bc) {
  restrict_flux2d_b_body<T>(native_blk(), Lc, tmp, bc);
}

// ---- 3D flux-conserving, divergence-preserving transfers -----------------
// Same construction as in 2D with two tangential slopes per face: fine faces
// on a coarse face get U + s1 D_t1 + s2 D_t2; interior fine faces get the
// mean of the two line values plus, for each other component c', one half
// of (slope of c' along the face's normal axis on the coarse cell's high
// c'-face - the same on its low c'-face). Restriction is the exact transpose:
// a gather into (rU, rD_t1, rD_t2), then rU + G_t1^T rD_t1 + G_t2^T rD_t2.

template <int C, int K> struct Oth;   // K-th axis other than C (ascending)
template <> struct Oth<0, 0> { static constexpr int v = 1; };
template <> struct Oth<0, 1> { static constexpr int v = 2; };
template <> struct Oth<1, 0> { static constexpr int v = 0; };
template <> struct Oth<1, 1> { static constexpr int v = 2; };
template <> struct Oth<2, 0> { static constexpr int v = 0; };
template <> struct Oth<2, 1> { static constexpr int v = 1; };

// slope / 8 of component C along axis A at coarse face P (mirror walls)
template <typename T, int C, int A>
__device__ __forceinline__ T slope3(const Lvl& Lc, const T* xc, const int P[3]) {
  if (!face_active<C>(Lc, P[0], P[1], P[2])) return (T)0;
  const T* u = xc + Lc.off[C] + cix(Lc, P[0], P[1], P[2]);
  const T u0 = GKB_LDG(u);
  int Pp[3] = {P[0], P[1], P[2]}, Pm[3] = {P[0], P[1], P[2]};
  Pp[A] += 1;
  Pm[A] -= 1;
  const T up = (Pp[A] < Lc.n[A]) ? coarse_face<T, C>(Lc, xc, Pp[0], Pp[1], Pp[2]) : -u0;
  const T um = (Pm[A] >= 0) ? coarse_face<T, C>(Lc, xc, Pm[0], Pm[1], Pm[2]) : -u0;
  return (up - um) * (T)0.125;
}

// The coarse slopes of every coarse face, computed once per prolongation:
// sl[kk * nvel + index of face P of component C] = slope3<C, Oth<C, kk>>(P)
// (0 on inactive faces, which are never written and stay 0).
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_slopes3d(Lvl Lc, const T* GKB_RESTRICT xc, T* GKB_RESTRICT sl) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int P[3] = {i, j, k};
  const long long c = cix(Lc, i, j, k);
#define GKB_SLOPES(C)                                                            \
  if (in_store<C>(Lc, i, j, k) && face_active<C>(Lc, i, j, k)) {                 \
    sl[Lc.off[C] + c] = slope3<T, C, Oth<C, 0>::v>(Lc, xc, P);                   \
    sl[Lc.nvel + Lc.off[C] + c] = slope3<T, C, Oth<C, 1>::v>(Lc, xc, P);         \
  }
  GKB_SLOPES(0)
  GKB_SLOPES(1)
  GKB_SLOPES(2)
#undef GKB_SLOPES
}

// slope / 8 of component C along axis A at coarse face P, from the table
template <typename T, int C, int A>
__device__ __forceinline__ T slope3_at(const Lvl& Lc, const T* GKB_RESTRICT sl, const int P[3]) {
  constexpr int kk = (Oth<C, 0>::v == A) ? 0 : 1;
  return GKB_LDG(sl + kk * Lc.nvel + Lc.off[C] + cix(Lc, P[0], P[1], P[2]));
}

// value of the prolongation at fine face p of component C: on a coarse face,
// the coarse value plus its two tangential slopes; inside a coarse cell, the
// mean of the two line values plus half the differences of the other
// components' slopes along C (slopes read from the table of k_slopes3d)
template <typename T, int C>
__device__ __forceinline__ T prolong3_val_tab(const Lvl& Lc, const T* xc, const T* sl, const int p[3]) {
  constexpr int t1 = Oth<C, 0>::v, t2 = Oth<C, 1>::v;
  const int q[3] = {p[0] >> 1, p[1] >> 1, p[2] >> 1};
  const T s1 = (p[t1] & 1) ? (T)1 : (T)-1;
  const T s2 = (p[t2] & 1) ? (T)1 : (T)-1;
  auto line_val = [&](int I) -> T {
    int P[3] = {q[0], q[1], q[2]};
    P[C] = I;
    return coarse_face<T, C>(Lc, xc, P[0], P[1], P[2]) + s1 * slope3_at<T, C, t1>(Lc, sl, P) +
           s2 * slope3_at<T, C, t2>(Lc, sl, P);
  };
  if ((p[C] & 1) == 0) return line_val(p[C] >> 1);
  const int I = p[C] >> 1;
  T val = (T)0.5 * (line_val(I) + line_val(I + 1));
  int lo[3] = {q[0], q[1], q[2]};
  lo[C] = I;
  int hi1[3] = {lo[0], lo[1], lo[2]}, hi2[3] = {lo[0], lo[1], lo[2]};
  hi1[t1] += 1;
  hi2[t2] += 1;
  val += (T)0.5 * (slope3_at<T, t1, C>(Lc, sl, hi1) - slope3_at<T, t1, C>(Lc, sl, lo));
  val += (T)0.5 * (slope3_at<T, t2, C>(Lc, sl, hi2) - slope3_at<T, t2, C>(Lc, sl, lo));
  return val;
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_prolong_flux3d(Lvl Lf, Lvl Lc, const T* GKB_RESTRICT xc,
                                                           const T* GKB_RESTRICT sl, T* GKB_RESTRICT xf) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int p[3] = {i, j, k};
  if (in_store<0>(Lf, i, j, k) && face_active<0>(Lf, i, j, k))
    xf[Lf.off[0] + cix(Lf, i, j, k)] += prolong3_val_tab<T, 0>(Lc, xc, sl, p);
  if (in_store<1>(Lf, i, j, k) && face_active<1>(Lf, i, j, k))
    xf[Lf.off[1] + cix(Lf, i, j, k)] += prolong3_val_tab<T, 1>(Lc, xc, sl, p);
  if (in_store<2>(Lf, i, j, k) && face_active<2>(Lf, i, j, k))
    xf[Lf.off[2] + cix(Lf, i, j, k)] += prolong3_val_tab<T, 2>(Lc, xc, sl, p);
}

template <typename T, int C>
__device__ __forceinline__ T fine3(const Lvl& Lf, const T* rf, const int P[3]) {
  return fine_face<T, C>(Lf, rf, P[0], P[1], P[2]);
}

// pass a for component C at coarse face Q: rU, and rD along its two tangential axes
template <typename T, int C>
__device__ __forceinline__ void restrict3_gather(const Lvl& Lf, const T* rf, const int Q[3], T& rU, T& rD1, T& rD2) {
  constexpr int t1 = Oth<C, 0>::v, t2 = Oth<C, 1>::v;
  const int Ic = Q[C];
  T su = 0, s1 = 0, s2 = 0;
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    const int nn = (kk == 0) ? 2 * Ic : (kk == 1) ? 2 * Ic + 1 : 2 * Ic - 1;
    const T w = (kk == 0) ? (T)1 : (T)0.5;
#pragma unroll
    for (int b1 = 0; b1 < 2; ++b1)
#pragma unroll
      for (int b2 = 0; b2 < 2; ++b2) {
        int P[3];
        P[C] = nn;
        P[t1] = 2 * Q[t1] + b1;
        P[t2] = 2 * Q[t2] + b2;
        const T v = w * fine3<T, C>(Lf, rf, P);
        su += v;
        s1 += b1 ? v : -v;
        s2 += b2 ? v : -v;
      }
  }
  // slope of C along t1 enters the correction of component t1's interior
  // faces in the coarse cells above (-1/2) and below (+1/2) this face
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int cc = (kk == 0) ? 2 * Ic : (kk == 1) ? 2 * Ic + 1 : (kk == 2) ? 2 * Ic - 2 : 2 * Ic - 1;
    const T w = (kk < 2) ? (T)-0.5 : (T)0.5;
#pragma unroll
    for (int sb = 0; sb < 2; ++sb) {
      int P[3];
      P[t1] = 2 * Q[t1] + 1;
      P[C] = cc;
      P[t2] = 2 * Q[t2] + sb;
      s1 += w * fine3<T, t1>(Lf, rf, P);
      int R[3];
      R[t2] = 2 * Q[t2] + 1;
      R[C] = cc;
      R[t1] = 2 * Q[t1] + sb;
      s2 += w * fine3<T, t2>(Lf, rf, R);
    }
  }
  rU = su;
  rD1 = s1;
  rD2 = s2;
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_restrict_flux3d_a(Lvl Lf, Lvl Lc, const T* GKB_RESTRICT rf, T* GKB_RESTRICT bc,
                                                               T* GKB_RESTRICT d1, T* GKB_RESTRICT d2) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  const int K = blockIdx.z;
  const int Q[3] = {I, J, K};
#define GKB_R3A(C)                                                               \
  if (in_store<C>(Lc, I, J, K)) {                                                \
    const long long id = Lc.off[C] + cix(Lc, I, J, K);                           \
    T rU = 0, r1 = 0, r2 = 0;                                                    \
    if (face_active<C>(Lc, I, J, K)) restrict3_gather<T, C>(Lf, rf, Q, rU, r1, r2); \
    bc[id] = rU;                                                                 \
    d1[id] = r1;                                                                 \
    d2[id] = r2;                                                                 \
  }
  GKB_R3A(0)
  GKB_R3A(1)
  GKB_R3A(2)
#undef GKB_R3A
}

template <typename T, int C, int A>
__device__ __forceinline__ T slope3_transpose(const Lvl& Lc, const T* d, const int Q[3]) {
  const int q = Q[A], Nt = Lc.n[A];
  T acc = 0;
  int R[3] = {Q[0], Q[1], Q[2]};
  if (q - 1 >= 0) { R[A] = q - 1; acc += GKB_LDG(d + Lc.off[C] + cix(Lc, R[0], R[1], R[2])); }
  if (q + 1 < Nt) { R[A] = q + 1; acc -= GKB_LDG(d + Lc.off[C] + cix(Lc, R[0], R[1], R[2])); }
  const T own = GKB_LDG(d + Lc.off[C] + cix(Lc, Q[0], Q[1], Q[2]));
  if (q == 0) acc += own;
  if (q == Nt - 1) acc -= own;
  return acc * (T)0.125;
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_restrict_flux3d_b(Lvl Lc, const T* GKB_RESTRICT d1, const T* GKB_RESTRICT d2,
                                                               T* GKB_RESTRICT bc) {
  const int I = blockIdx.x * BX + threadIdx.x;
  const int J = blockIdx.y * BY + threadIdx.y;
  const int K = blockIdx.z;
  const int Q[3] = {I, J, K};
#define GKB_R3B(C)                                                               \
  if (in_store<C>(Lc, I, J, K) && face_active<C>(Lc, I, J, K))                   \
    bc[Lc.off[C] + cix(Lc, I, J, K)] += slope3_transpose<T, C, Oth<C, 0>::v>(Lc, d1, Q) + \
                                        slope3_transpose<T, C, Oth<C, 1>::v>(Lc, d2, Q);
  GKB_R3B(0)
  GKB_R3B(1)
  GKB_R3B(2)
#undef GKB_R3B
}

// coarsest level: x[idx[r]] = sum_c Minv[r][c] b[idx[c]]; one warp per row
template <typename T>
__device__ __forceinline__ void coarse_solve_body(const Blk& B, int m, const T* GKB_RESTRICT Minv, const int* GKB_RESTRICT idx,
                               const T* GKB_RESTRICT b, T* GKB_RESTRICT x) {
  const int warp = (B.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  double acc = 0.0;
  const T* row = Minv + (size_t)warp * m;
  for (int c = lane; c < m; c += 32) acc += (double)row[c] * (double)GKB_LDG(b + idx[c]);
  acc = warp_sum(acc);
  if (lane == 0) x[idx[warp]] = (T)acc;
}

template <typename T>
__global__ void k_coarse_solve(int m, const T* GKB_RESTRICT Minv, const int* GKB_RESTRICT idx,
                               const T* GKB_RESTRICT b, T* GKB_RESTRICT x) {
  coarse_solve_body<T>(native_blk(), m, Minv, idx, b, x);
}

// ---------------------------------------------------------------------------
// BLAS-1 on flat padded arrays (len multiple of 4), fused reductions
// ---------------------------------------------------------------------------

constexpr int RB = 256;

// sum a.b (and b.b when NV == 2)
template <typename T>
__device__ __forceinline__ void dot_body(const Blk& B, long long len, const T* GKB_RESTRICT a, const T* GKB_RESTRICT b,
                                             RedBuf red, int fin, void* st, const int* pred) {
  if (pred && !*pred) return;  // every block skips, so the ticket stays untouched
  T acc = 0;
  const long long stride = (long long)B.nx * RB;
  for (long long t = (long long)B.x * RB + threadIdx.x; t < len; t += stride)
    acc += a[t] * b[t];
  double v[1] = {(double)acc};
  grid_reduce<1>(v, red, fin, st, B);
}

template <typename T>
__global__ void __launch_bounds__(RB) k_dot(long long len, const T* GKB_RESTRICT a, const T* GKB_RESTRICT b,
                                             RedBuf red, int fin, void* st, const int* pred) {
  dot_body<T>(native_blk(), len, a, b, red, fin, st, pred);
}

// sums a.b and b.c in one pass
template <typename T>
__global__ void __launch_bounds__(RB) k_dot2(long long len, const T* GKB_RESTRICT a, const T* GKB_RESTRICT b,
                                              const T* GKB_RESTRICT c, RedBuf red, int fin, void* st) {
  T ab = 0, bc = 0;
  const long long stride = (long long)gridDim.x * RB;
  for (long long t = (long long)blockIdx.x * RB + threadIdx.x; t < len; t += stride) {
    const T bt = b[t];
    ab += a[t] * bt;
    bc += bt * c[t];
  }
  double v[2] = {(double)ab, (double)bc};
  grid_reduce<2>(v, red, fin, st);
}

// x += alpha p ; r -= alpha q ; sum r.r      (alpha from CgState)
template <typename T>
__device__ __forceinline__ void cg_update_body(const Blk& B, long long len, T* GKB_RESTRICT x, const T* GKB_RESTRICT p,
                                                   T* GKB_RESTRICT r, const T* GKB_RESTRICT q,
                                                   const CgState* cg, RedBuf red, void* st, int fin) {
  const T alpha = (T)cg->alpha;
  T acc = 0;
  const long long stride = (long long)B.nx * RB;
  for (long long t = (long long)B.x * RB + threadIdx.x; t < len; t += stride) {
    x[t] += alpha * p[t];
    const T rn = r[t] - alpha * q[t];
    r[t] = rn;
    acc += rn * rn;
  }
  double v[1] = {(double)acc};
  grid_reduce<1>(v, red, fin, st, B);
}

template <typename T>
__global__ void __launch_bounds__(RB) k_cg_update(long long len, T* GKB_RESTRICT x, const T* GKB_RESTRICT p,
                                                   T* GKB_RESTRICT r, const T* GKB_RESTRICT q,
                                                   const CgState* cg, RedBuf red, void* st, int fin) {
  cg_update_body<T>(native_blk(), len, x, p, r, q, cg, red, st, fin);
}

// p = z + beta p   (beta from CgState; first: p = z)
template <typename T>
__device__ __forceinline__ void cg_dir_body(const Blk& B, long long len, T* GKB_RESTRICT p, const T* GKB_RESTRICT z,
                                                const CgState* cg, int first) {
  const T beta = first ? (T)0 : (T)cg->beta;
  const long long stride = (long long)B.nx * RB;
  // the first direction never reads p: a non-finite p left by an earlier
  // failed solve must not survive as 0 * NaN
  for (long long t = (long long)B.x * RB + threadIdx.x; t < len; t += stride)
    p[t] = first ? z[t] : z[t] + beta * p[t];
}

template <typename T>
__global__ void __launch_bounds__(RB) k_cg_dir(long long len, T* GKB_RESTRICT p, const T* GKB_RESTRICT z,
                                                const CgState* cg, int first) {
  cg_dir_body<T>(native_blk(), len, p, z, cg, first);
}

// y = a x + b y (host scalars)
template <typename T>
__device__ __forceinline__ void axpby_body(const Blk& B, long long len, T a, const T* GKB_RESTRICT x, T b, T* GKB_RESTRICT y) {
  const long long stride = (long long)B.nx * RB;
  // b = 0 overwrites y without reading it (y may hold stale non-finite values)
  for (long long t = (long long)B.x * RB + threadIdx.x; t < len; t += stride)
    y[t] = (b == (T)0) ? a * x[t] : a * x[t] + b * y[t];
}

template <typename T>
__global__ void __launch_bounds__(RB) k_axpby(long long len, T a, const T* GKB_RESTRICT x, T b, T* GKB_RESTRICT y) {
  axpby_body<T>(native_blk(), len, a, x, b, y);
}

}  // namespace gkb
