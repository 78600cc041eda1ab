// solver.cu - multigrid hierarchy, conjugate gradients and the GKB driver
// (Algorithm 1 with the augmented-Lagrangian transform of Eq. (3) and the
// lower-bound stopping rule of Eq. (5)), all running on the device; the host
// only sequences launches.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <map>
#include <mutex>
#include <chrono>
#include <cstdio>
#include <cstdlib>

#include <cooperative_groups.h>

#include "solver.cuh"
#include "gkb_device.cuh"
#include "lockstep.cuh"
#include "prof.h"
#include "unet.cuh"

namespace gkb {

thread_local Profiler* g_prof = nullptr;

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw Error{e == cudaErrorMemoryAllocation ? GKB_ERR_OOM : GKB_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

static long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

Lvl make_level(int dim, const int n[3], double h, const int nat[6], double gc) {
  Lvl L{};
  L.dim = dim;
  L.n[0] = n[0];
  L.n[1] = n[1];
  L.n[2] = (dim == 3) ? n[2] : 1;
  for (int s = 0; s < 6; ++s) L.nat[s] = (s < 2 * dim) ? nat[s] : 0;
  L.P = (int)round_up(n[0] + 1, 32);
  L.S = (long long)(n[1] + 1) * L.P;
  if (dim == 2) {
    L.off[0] = 0;
    L.off[1] = L.S;
    L.off[2] = 2 * L.S;
    L.nvel = 2 * L.S;
  } else {
    L.off[0] = 0;
    L.off[1] = (long long)L.n[2] * L.S;
    L.off[2] = 2LL * L.n[2] * L.S;
    L.nvel = (3LL * L.n[2] + 1) * L.S;
  }
  L.ncell = (long long)L.n[2] * L.S;
  L.h = h;
  L.wscale = pow(h, dim - 2);
  L.ascale = pow(h, dim - 1);
  L.gc = gc;
  L.mu0 = 1.0;
  L.mu64 = nullptr;
  L.mu32 = nullptr;
  L.nw64 = nullptr;
  L.nw32 = nullptr;
  L.sym = 0;
  L.fast = 1;
  finish_level(L);
  return L;
}

template <typename T> static void set_mu(Lvl& L, const T* mu);
template <> void set_mu<double>(Lvl& L, const double* mu) { L.mu64 = mu; L.mu32 = nullptr; }
template <> void set_mu<float>(Lvl& L, const float* mu) { L.mu32 = mu; L.mu64 = nullptr; }
template <typename T> static void set_em(Lvl& L, const T* e);
template <> void set_em<double>(Lvl& L, const double* e) { L.em64 = e; L.em32 = nullptr; }
template <> void set_em<float>(Lvl& L, const float* e) { L.em32 = e; L.em64 = nullptr; }
template <typename T> static void set_nw(Lvl& L, const T* w);
template <> void set_nw<double>(Lvl& L, const double* w) { L.nw64 = w; L.nw32 = nullptr; }
template <> void set_nw<float>(Lvl& L, const float* w) { L.nw32 = w; L.nw64 = nullptr; }

// ---------------------------------------------------------------------------
// layout kernels (compact ordering <-> padded layout)
// ---------------------------------------------------------------------------

struct Compact {
  int dim;
  int lo[3][3];    // low corner of the active box of component c
  int ext[3][3];   // extents of that box
  long long base[3];
  long long m;
};

static Compact make_compact(const Lvl& L) {
  Compact c{};
  c.dim = L.dim;
  long long off = 0;
  for (int comp = 0; comp < L.dim; ++comp) {
    for (int a = 0; a < 3; ++a) {
      if (a >= L.dim) { c.lo[comp][a] = 0; c.ext[comp][a] = 1; continue; }
      if (a == comp) {
        const int lo = L.nat[2 * a] ? 0 : 1;
        const int hi = L.nat[2 * a + 1] ? L.n[a] : L.n[a] - 1;
        c.lo[comp][a] = lo;
        c.ext[comp][a] = hi - lo + 1;
      } else {
        c.lo[comp][a] = 0;
        c.ext[comp][a] = L.n[a];
      }
    }
    c.base[comp] = off;
    off += (long long)c.ext[comp][0] * c.ext[comp][1] * c.ext[comp][2];
  }
  c.m = off;
  return c;
}

__device__ __forceinline__ long long compact_to_padded(const Lvl& L, const Compact& c, long long t) {
  int comp = 0;
  if (c.dim == 3 && t >= c.base[2]) comp = 2;
  else if (t >= c.base[1]) comp = 1;
  const long long l = t - c.base[comp];
  const int ex = c.ext[comp][0], ey = c.ext[comp][1];
  const long long row = l / ex;
  const int i = (int)(l - row * ex) + c.lo[comp][0];
  const long long pl = row / ey;
  const int j = (int)(row - pl * ey) + c.lo[comp][1];
  const int k = (int)pl + c.lo[comp][2];
  return L.off[comp] + cix(L, i, j, k);
}

template <typename TO>
__global__ void k_pack_vel(Lvl L, Compact c, const double* __restrict__ src, TO* __restrict__ dst) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < c.m; t += (long long)gridDim.x * blockDim.x)
    dst[compact_to_padded(L, c, t)] = (TO)src[t];
}
__global__ void k_unpack_vel(Lvl L, Compact c, const double* __restrict__ src, double* __restrict__ dst) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < c.m; t += (long long)gridDim.x * blockDim.x)
    dst[t] = src[compact_to_padded(L, c, t)];
}
template <typename TO>
__global__ void k_pack_cell(Lvl L, const double* __restrict__ src, TO* __restrict__ dst) {
  const long long n = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / L.n[0];
    const int i = (int)(t - row * L.n[0]);
    const int k = (int)(row / L.n[1]);
    const int j = (int)(row - (long long)k * L.n[1]);
    dst[cix(L, i, j, k)] = (TO)src[t];
  }
}
__global__ void k_unpack_cell(Lvl L, const double* __restrict__ src, double* __restrict__ dst, double shift) {
  const long long n = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / L.n[0];
    const int i = (int)(t - row * L.n[0]);
    const int k = (int)(row / L.n[1]);
    const int j = (int)(row - (long long)k * L.n[1]);
    dst[t] = src[cix(L, i, j, k)] - shift;
  }
}

// coarse viscosity: mean of the 2^d fine cells
template <typename T>
__global__ void k_mu_coarsen(Lvl Lf, Lvl Lc, const T* __restrict__ muf, T* __restrict__ muc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= Lc.n[0] || J >= Lc.n[1]) return;
  const int nz = (Lf.dim == 3) ? 2 : 1;
  T s = 0;
  for (int dz = 0; dz < nz; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) s += muf[cix(Lf, 2 * I + dx, 2 * J + dy, Lf.dim == 3 ? 2 * K + dz : 0)];
  muc[cix(Lc, I, J, K)] = s / (T)(4 * nz);
}

// deterministic pseudo-random start vector for the power iteration
template <typename T>
__global__ void k_fill_hash(Lvl L, T* x) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z;
  for (int c = 0; c < L.dim; ++c) {
    bool act = (c == 0) ? face_active<0>(L, i, j, k) : (c == 1) ? face_active<1>(L, i, j, k) : face_active<2>(L, i, j, k);
    if (!act) continue;
    unsigned long long hsh = (unsigned long long)(L.off[c] + cix(L, i, j, k)) * 0x9E3779B97F4A7C15ull + 12345u;
    hsh ^= hsh >> 31; hsh *= 0xBF58476D1CE4E5B9ull; hsh ^= hsh >> 29;
    x[L.off[c] + cix(L, i, j, k)] = (T)((double)(hsh >> 11) * (1.0 / 9007199254740992.0) - 0.5);
  }
}

static dim3 fgrid(const Lvl& L) {
  const int nz = (L.dim == 3) ? L.n[2] + 1 : 1;
  return dim3((L.n[0] + 1 + 31) / 32, (L.n[1] + 1 + 7) / 8, nz);
}

static void read_scalars(double* dev, double* host, int n, cudaStream_t s) {
  GKB_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// loop graphs: "prefix; while (cond) body; suffix" captured once, launched
// once per inner solve; the loop condition is set on the device
// ---------------------------------------------------------------------------

__global__ void k_cg_cond_init(cudaGraphConditionalHandle h, CgState* c) {
  c->graph_iters = 0;
  cudaGraphSetConditional(h, c->done ? 0u : 1u);
}

// continue while the CG has not stopped; hard_max bounds the loop even if
// the iteration counter were never advanced
__global__ void k_cg_cond(cudaGraphConditionalHandle h, CgState* c, int hard_max, int fb = 0) {
  int& runs = fb ? c->fb_iters : c->graph_iters;
  runs += 1;
  unsigned cont = c->done ? 0u : 1u;
  if (runs >= hard_max) {
    cont = 0u;
    if (!c->done) {
      if (c->status == ST_OK) c->status = ST_INNER_NOT_CONVERGED;
      c->done = 1;
    }
  }
  cudaGraphSetConditional(h, cont);
}

// Capture "pre; while (cond) body; post" into the graph that stream s is
// capturing (possibly the body graph of an enclosing loop). The condition
// handle is created on that graph; `pre` must end with the kernel that sets
// it, `body` with the kernel that updates it. The body is captured on sb.
template <class Pre, class Body, class Post>
static void capture_loop(cudaStream_t s, cudaStream_t sb, int body_phase, Pre pre, Body body, Post post) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  GKB_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive) throw Error{GKB_ERR_CUDA, "stream is not capturing"};
  cudaGraphConditionalHandle h;
  GKB_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault));
  pre(s, h);
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  GKB_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wn;
  GKB_CUDA(cudaGraphAddNode(&wn, cg, deps, nullptr, nd, &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  Profiler* P = g_prof;
  const int saved = P ? P->phase : -1;
  GKB_CUDA(cudaStreamBeginCaptureToGraph(sb, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  if (P) P->phase = body_phase;
  body(sb, h);
  if (P) P->phase = saved;
  GKB_CUDA(cudaStreamEndCapture(sb, &bodyg));
  GKB_CUDA(cudaStreamUpdateCaptureDependencies(s, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
  post(s);
}

void capture_while(cudaStream_t s, cudaStream_t sb, int body_phase,
                   const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& pre,
                   const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& body,
                   const std::function<void(cudaStream_t)>& post) {
  capture_loop(s, sb, body_phase, pre, body, post);
}

// end any capture still open on these streams (error paths)
static void abandon_captures(std::initializer_list<cudaStream_t> ss) {
  for (cudaStream_t st : ss) {
    if (!st) continue;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t dummy = nullptr;
      cudaStreamEndCapture(st, &dummy);
      if (dummy) cudaGraphDestroy(dummy);
    }
  }
  (void)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// multigrid hierarchy
// ---------------------------------------------------------------------------

// In-place Gauss-Jordan inversion of an SPD matrix, pivot k: save the
// scaled pivot row (entry k = 1/p) and the pivot column, then update every
// entry (a_ij - a_ik a_kj / p; the pivot column becomes -a_ik / p)
__global__ void k_gj_save(const double* __restrict__ A, int m, int k, double* __restrict__ rowk,
                          double* __restrict__ colk, int* bad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const double p = A[(size_t)k * m + k];
  if (t == 0 && !(p > 0.0)) *bad = 1;
  colk[t] = A[(size_t)t * m + k];
  rowk[t] = (t == k) ? 1.0 / p : A[(size_t)k * m + t] / p;
}

__global__ void k_gj_update(double* __restrict__ A, int m, int k, const double* __restrict__ rowk,
                            const double* __restrict__ colk) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= m || j >= m) return;
  double& a = A[(size_t)i * m + j];
  if (i == k) a = rowk[j];
  else a = ((j == k) ? 0.0 : a) - colk[i] * rowk[j];
}

template <typename T>
__global__ void k_gj_store(const double* __restrict__ A, int m, T* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
  if (r >= m || c >= m) return;
  out[(size_t)r * m + c] = (T)(0.5 * (A[(size_t)r * m + c] + A[(size_t)c * m + r]));
}

template <typename T>
void Gmg<T>::build(const Lvl& fine, const T* fine_mu, int coarse_max, int deg, const RedBuf& red,
                   double* scratch, cudaStream_t s) {
  degree = deg;
  this->red = red;
  detach_net();
  lev.clear();
  lev.reserve(32);
  lev.emplace_back();
  lev[0].L = fine;
  set_mu<T>(lev[0].L, fine_mu);
  // coarsen while every side is even, halves to >= 2 cells and the longest
  // side exceeds coarse_max (halved in 3D to keep the dense coarse solve small)
  const int cmax = (fine.dim == 3) ? std::max(4, coarse_max / 2) : coarse_max;
  for (;;) {
    const Lvl& Lf = lev.back().L;
    bool can = true;
    int nmax = 0;
    for (int a = 0; a < Lf.dim; ++a) {
      if (Lf.n[a] % 2 != 0 || Lf.n[a] / 2 < 2) can = false;
      nmax = std::max(nmax, Lf.n[a]);
    }
    if (!can || nmax <= cmax) break;
    int nc[3] = {Lf.n[0] / 2, Lf.n[1] / 2, Lf.dim == 3 ? Lf.n[2] / 2 : 1};
    const double gc = Lf.gc / (Lf.dim == 3 ? 8.0 : 4.0);
    Lvl Lc = make_level(Lf.dim, nc, 2.0 * Lf.h, Lf.nat, gc);
    Lc.mu0 = Lf.mu0;
    Lc.fast = Lf.fast;
    Lc.sym = Lf.sym;
    finish_level(Lc);
    lev.emplace_back();
    Level& C = lev.back();
    C.L = Lc;
    const T* fmu = (sizeof(T) == 8) ? (const T*)lev[lev.size() - 2].L.mu64 : (const T*)lev[lev.size() - 2].L.mu32;
    if (fmu) {
      C.mu.alloc(Lc.ncell);
      dim3 g((nc[0] + 31) / 32, (nc[1] + 7) / 8, Lc.n[2]);
      { ProfScope ps_(GKB_KC_LAYOUT, s); k_mu_coarsen<T><<<g, dim3(32, 8), 0, s>>>(lev[lev.size() - 2].L, Lc, fmu, C.mu.p); }
      GKB_CUDA(cudaGetLastError());
      set_mu<T>(C.L, C.mu.p);
      // FP64 levels read node / edge viscosities from a table (saves six
      // FP64-pipe operations per link); FP32 levels are faster forming the
      // means from the cells than streaming one more array
      if (sizeof(T) == 8) {
        C.em.alloc(Ops<T>::edge_table_len(Lc));
        Ops<T>::edge_table(C.L, C.em.p, s);
        GKB_CUDA(cudaGetLastError());
        set_em<T>(C.L, C.em.p);
      }
    }
    // diagonal N: the coarse weight is the mean of the 2^d children's, which
    // with gc / 2^d and the divergence-preserving transfers makes the coarse
    // grad-div term the Galerkin product of the fine one
    const T* fnw = (sizeof(T) == 8) ? (const T*)lev[lev.size() - 2].L.nw64 : (const T*)lev[lev.size() - 2].L.nw32;
    set_nw<T>(C.L, (const T*)nullptr);
    if (fnw && fmu) {
      C.nw.alloc(Lc.ncell);
      dim3 g((nc[0] + 31) / 32, (nc[1] + 7) / 8, Lc.n[2]);
      { ProfScope ps_(GKB_KC_LAYOUT, s); k_mu_coarsen<T><<<g, dim3(32, 8), 0, s>>>(lev[lev.size() - 2].L, Lc, fnw, C.nw.p); }
      GKB_CUDA(cudaGetLastError());
      set_nw<T>(C.L, C.nw.p);
    }
  }
  const int nl = (int)lev.size();
  for (int l = 0; l < nl; ++l) {
    Level& V = lev[l];
    if (l > 0) {
      V.x.alloc(V.L.nvel);
      V.b.alloc(V.L.nvel);
      if (V.L.dim == 3) {
        V.t2.alloc(V.L.nvel);
        V.sl.alloc(2 * (size_t)V.L.nvel);
      }
    }
    if (l < nl - 1) {
      V.r.alloc(V.L.nvel);
      V.d.alloc(V.L.nvel);
      // constant viscosity: inverses of the 75 patch classes; variable
      // viscosity: the inverse of every patch
      V.table.alloc(Ops<T>::patch_table_len(V.L));
      Ops<T>::patch_table(V.L, V.table.p, s);
      GKB_CUDA(cudaGetLastError());
      const long long fo = Ops<T>::fold_interior_offset(V.L);
      V.fold_in.clear();
      if (fo >= 0) {
        std::vector<T> h(48);
        GKB_CUDA(cudaMemcpyAsync(h.data(), V.table.p + fo, 48 * sizeof(T), cudaMemcpyDeviceToHost, s));
        GKB_CUDA(cudaStreamSynchronize(s));
        V.fold_in.assign(h.begin(), h.end());
      }
    }
  }
  // power iteration for lambda_max(C M) on every smoothing level
  for (int l = 0; l < nl - 1; ++l) {
    Level& V = lev[l];
    DevBuf<T> xv, zv, zero;
    xv.alloc(V.L.nvel);
    zv.alloc(V.L.nvel);
    zero.alloc(V.L.nvel);
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_fill_hash<T><<<fgrid(V.L), dim3(32, 8), 0, s>>>(V.L, xv.p); }
    GKB_CUDA(cudaGetLastError());
    double hs[4];
    double lam = 0;
    for (int it = 0; it < 16; ++it) {
      Ops<T>::residual(V.L, xv.p, zero.p, V.r.p, s);       // r = -M x
      Ops<T>::patch(V.L, V.r.p, zv.p, V.table.p, s);       // z = -C M x
      Ops<T>::dot(V.L.nvel, zv.p, zv.p, red, FIN_STORE, scratch, s);
      read_scalars(scratch, hs, 1, s);
      const double zn = sqrt(hs[0]);
      Ops<T>::dot(V.L.nvel, xv.p, xv.p, red, FIN_STORE, scratch, s);
      read_scalars(scratch, hs + 1, 1, s);
      const double xn = sqrt(hs[1]);
      if (!(zn > 0) || !(xn > 0)) break;
      lam = zn / xn;
      Ops<T>::axpby(V.L.nvel, (T)(-1.0 / zn), zv.p, (T)0, xv.p, s);
    }
    GKB_CUDA(cudaGetLastError());
    V.lam_max = lam;
    const double hi = cheb_hi * lam, lo = cheb_lo * lam;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    V.ca.assign(deg, 0.0);
    V.cb.assign(deg, 0.0);
    double rho = 1.0 / sigma;
    V.ca[0] = 1.0 / theta;
    V.cb[0] = 0.0;
    for (int k = 1; k < deg; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      V.ca[k] = 2.0 * rn / delta;
      V.cb[k] = rn * rho;
      rho = rn;
    }
  }
  // coarsest level: dense M, inverted once
  Level& Cl = lev.back();
  const Lvl& L = Cl.L;
  Compact cmp = make_compact(L);
  const int m = (int)cmp.m;
  if (m > 4096) throw Error{GKB_ERR_INVALID_ARG, "coarsest multigrid level too large (" + std::to_string(m) + " unknowns)"};
  coarse_m = m;
  std::vector<long long> pidx(m);
  std::vector<int> ucomp(m), upos(3 * (size_t)m);  // component and (i, j, k) of every unknown
  {
    int t = 0;
    for (int comp = 0; comp < L.dim; ++comp)
      for (int k = 0; k < cmp.ext[comp][2]; ++k)
        for (int j = 0; j < cmp.ext[comp][1]; ++j)
          for (int i = 0; i < cmp.ext[comp][0]; ++i) {
            const int pi = i + cmp.lo[comp][0], pj = j + cmp.lo[comp][1], pk = k + cmp.lo[comp][2];
            pidx[t] = L.off[comp] + cix(L, pi, pj, pk);
            ucomp[t] = comp;
            upos[3 * t] = pi;
            upos[3 * t + 1] = pj;
            upos[3 * t + 2] = pk;
            ++t;
          }
  }
  // M by colored probing: faces interact only within one cell in every axis
  // (W links and the grad-div coupling of the faces of a cell), so the
  // columns of one component whose positions agree modulo 3 in every axis
  // have disjoint row supports and one product recovers all of them
  std::vector<int> row_of(L.nvel, -1);
  for (int r = 0; r < m; ++r) row_of[pidx[r]] = r;
  std::vector<double> A((size_t)m * m, 0.0);
  {
    DevBuf<T> e, y;
    e.alloc(L.nvel);
    y.alloc(L.nvel);
    std::vector<T> he(L.nvel), hy(L.nvel);
    const int ncol = (L.dim == 3) ? 27 : 9;
    for (int comp = 0; comp < L.dim; ++comp)
      for (int color = 0; color < ncol; ++color) {
        const int cc[3] = {color % 3, (color / 3) % 3, color / 9};
        std::fill(he.begin(), he.end(), (T)0);
        std::vector<int> cols;
        for (int c = 0; c < m; ++c) {
          if (ucomp[c] != comp || upos[3 * c] % 3 != cc[0] || upos[3 * c + 1] % 3 != cc[1] ||
              upos[3 * c + 2] % 3 != cc[2])
            continue;
          he[pidx[c]] = (T)1;
          cols.push_back(c);
        }
        if (cols.empty()) continue;
        GKB_CUDA(cudaMemcpyAsync(e.p, he.data(), L.nvel * sizeof(T), cudaMemcpyHostToDevice, s));
        Ops<T>::apply(L, 1, e.p, y.p, s);
        GKB_CUDA(cudaMemcpyAsync(hy.data(), y.p, L.nvel * sizeof(T), cudaMemcpyDeviceToHost, s));
        GKB_CUDA(cudaStreamSynchronize(s));
        for (int c : cols) {
          const int i = upos[3 * c], j = upos[3 * c + 1], k = upos[3 * c + 2];
          for (int rc = 0; rc < L.dim; ++rc)
            for (int dk = (L.dim == 3 ? -1 : 0); dk <= (L.dim == 3 ? 1 : 0); ++dk)
              for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                  const int ii = i + di, jj = j + dj, kk = k + dk;
                  // the faces of component rc: position n along axis rc, n - 1 along the others
                  if (ii < 0 || jj < 0 || kk < 0 || ii > L.n[0] - (rc != 0) || jj > L.n[1] - (rc != 1) ||
                      kk > L.n[2] - (rc != 2 || L.dim == 2 ? 1 : 0))
                    continue;
                  const long long pr = L.off[rc] + cix(L, ii, jj, kk);
                  const int r = row_of[pr];
                  if (r >= 0) A[(size_t)r * m + c] = (double)hy[pr];
                }
        }
      }
  }
  // symmetrise; in-place Gauss-Jordan inversion on the device (SPD: no pivoting)
  for (int r = 0; r < m; ++r)
    for (int c = r + 1; c < m; ++c) {
      const double a = 0.5 * (A[(size_t)r * m + c] + A[(size_t)c * m + r]);
      A[(size_t)r * m + c] = A[(size_t)c * m + r] = a;
    }
  {
    DevBuf<double> Ad, rowk, colk;
    DevBuf<int> bad;
    Ad.alloc((size_t)m * m);
    rowk.alloc(m);
    colk.alloc(m);
    bad.alloc(1);
    GKB_CUDA(cudaMemcpyAsync(Ad.p, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    const dim3 b2(32, 8), g2((m + 31) / 32, (m + 7) / 8);
    for (int k = 0; k < m; ++k) {
      { ProfScope ps_(GKB_KC_COARSE, s); k_gj_save<<<(m + 255) / 256, 256, 0, s>>>(Ad.p, m, k, rowk.p, colk.p, bad.p); }
      { ProfScope ps_(GKB_KC_COARSE, s); k_gj_update<<<g2, b2, 0, s>>>(Ad.p, m, k, rowk.p, colk.p); }
    }
    coarse_inv.alloc((size_t)m * m);
    { ProfScope ps_(GKB_KC_COARSE, s); k_gj_store<T><<<g2, b2, 0, s>>>(Ad.p, m, coarse_inv.p); }
    GKB_CUDA(cudaGetLastError());
    int hbad = 0;
    GKB_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
    if (hbad) throw Error{GKB_ERR_NOT_SPD, "coarse-level matrix is not positive definite"};
  }
  std::vector<int> idx32(m);
  for (int i = 0; i < m; ++i) idx32[i] = (int)pidx[i];
  coarse_idx.alloc(m);
  GKB_CUDA(cudaMemcpyAsync(coarse_idx.p, idx32.data(), m * sizeof(int), cudaMemcpyHostToDevice, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  gmg_tail_setup<T>(*this, tail_side, s);
}

template <typename T>
void Gmg<T>::smooth(int l, const T* b, T* x, bool x_zero, cudaStream_t s) {
  Level& V = lev[l];
  for (int k = 0; k < degree; ++k) {
    const T* r;
    if (k == 0 && x_zero) r = b;
    else {
      Ops<T>::residual(V.L, x, b, V.r.p, s);
      r = V.r.p;
    }
    Ops<T>::cheb(V.L, r, x, V.d.p, (T)V.ca[k], (T)V.cb[k], (k == 0 && x_zero) ? 1 : 0, V.table.p, s,
                 V.fold_in.empty() ? nullptr : V.fold_in.data());
  }
}

template <typename T>
void Gmg<T>::attach_net(Unet* u, int level, bool composite, cudaStream_t s) {
  if (level < 0 || level >= (int)lev.size()) throw Error{GKB_ERR_INVALID_ARG, "no multigrid level for the network"};
  const Lvl& L = lev[level].L;
  if (L.dim != 2 || L.n[0] % 4 || L.n[1] % 4)
    throw Error{GKB_ERR_INVALID_ARG, "the network level must be 2D with sides divisible by 4"};
  if (!net_act) net_act = new UnetAct();
  u->ensure(*net_act, 1, L.n[1], L.n[0]);
  net_img.alloc((size_t)L.n[0] * L.n[1] * 3);
  net_nrm.alloc(8);
  net_q.alloc(L.nvel);
  if (u->bf16_stale) u->refresh_bf16(s);
  net = u;
  net_level = level;
  net_composite = composite;
}

template <typename T>
void Gmg<T>::detach_net() {
  net = nullptr;
  net_level = -1;
}

template <typename T>
Gmg<T>::~Gmg() {
  delete net_act;
}

template <typename T>
void Gmg<T>::vcycle(const T* r0, T* z0, cudaStream_t s, bool use_net) {
  const int nl = (int)lev.size();
  const bool with_net = use_net && net && net_level >= 0;
  // replace form: the network is the correction of its level and everything
  // below it; composite form: the network's correction is the starting
  // guess of the ordinary cycle from its level down
  const bool replace = with_net && !net_composite;
  const int lc = replace ? net_level : nl - 1;  // the level of the coarsest correction
  auto lvl_b = [&](int l) { return (l == 0) ? r0 : (const T*)lev[l].b.p; };
  auto lvl_x = [&](int l) { return (l == 0) ? z0 : lev[l].x.p; };
  auto net_at = [&](int l) {
    unet_correct<T>(*net, *net_act, lev[l].L, lvl_b(l), lvl_x(l), net_q.p, net_img.p, net_nrm.p, red, s);
  };
  // the fused coarse end: levels from tail_level on run in one cluster kernel
  const bool tail = !with_net && tail_level > 0 && tail_buf.p;
  const int ld = tail ? tail_level : lc;  // levels handled by separate launches
  for (int l = 0; l < ld; ++l) {
    bool x_zero = true;
    if (with_net && l == net_level) {  // composite form
      net_at(l);
      x_zero = false;
    }
    smooth(l, lvl_b(l), lvl_x(l), x_zero, s);
    Ops<T>::residual(lev[l].L, lvl_x(l), lvl_b(l), lev[l].r.p, s);
    Ops<T>::restrict_(lev[l].L, lev[l + 1].L, lev[l].r.p, lev[l + 1].b.p, lev[l + 1].x.p, lev[l + 1].t2.p, s);
  }
  if (tail) gmg_tail_launch<T>(*this, s);
  else if (replace) net_at(lc);
  else Ops<T>::coarse(coarse_m, coarse_inv.p, coarse_idx.p, lvl_b(lc), lvl_x(lc), s);
  for (int l = ld - 1; l >= 0; --l) {
    Ops<T>::prolong(lev[l].L, lev[l + 1].L, lev[l + 1].x.p, lvl_x(l), lev[l + 1].sl.p, s);
    smooth(l, lvl_b(l), lvl_x(l), false, s);
  }
}

template struct Gmg<double>;
template struct Gmg<float>;

// ---------------------------------------------------------------------------
// conjugate gradients (host-sequenced, device scalars)
// ---------------------------------------------------------------------------

// host-sequenced forms: after a flexible solve stopped (state synchronised
// in `host`), prepare the fallback loop the way k_fb_init does; true when it
// has to run
static bool fallback_restart(CgState* dev, CgState* host, cudaStream_t s) {
  if (!host->fallback || host->status != ST_OK) return false;
  if (host->it >= host->maxit) host->status = ST_INNER_NOT_CONVERGED;
  else {
    host->done = 0;
    host->rz_old = 0.0;
  }
  GKB_CUDA(cudaMemcpyAsync(dev, host, sizeof(CgState), cudaMemcpyHostToDevice, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  return host->status == ST_OK;
}

template <typename T>
void Cg<T>::init(const Lvl& L_, Gmg<T>* pre_, const RedBuf& red_, CgState* st_dev, CgState* st_host) {
  L = L_;
  pre = pre_;
  red = red_;
  st = st_dev;
  host = st_host;
  r.alloc(L.nvel);
  p.alloc(L.nvel);
  q.alloc(L.nvel);
  z.alloc(L.nvel);  // also the second work vector of the single-kernel CG
}

template <typename T>
int Cg<T>::solve(const T* f, T* x, double tol, int maxit, cudaStream_t s, int* iters) {
  const long long len = L.nvel;
  CgState h{};
  h.tol2 = tol * tol;
  h.maxit = maxit;
  h.rho2 = flex ? rho2 : 0.0;
  GKB_CUDA(cudaMemcpyAsync(st, &h, sizeof(CgState), cudaMemcpyHostToDevice, s));
  GKB_CUDA(cudaMemsetAsync(x, 0, len * sizeof(T), s));
  GKB_CUDA(cudaMemcpyAsync(r.p, f, len * sizeof(T), cudaMemcpyDeviceToDevice, s));
  Ops<T>::dot(len, f, f, red, FIN_CG_INIT, st, s);
  T* zp = pre ? z.p : r.p;
  if (pre) pre->vcycle(r.p, zp, s);
  Ops<T>::dot(len, r.p, zp, red, FIN_CG_RZ0, st, s);
  Ops<T>::cg_dir(len, p.p, zp, st, 1, s);
  GKB_CUDA(cudaMemcpyAsync(host, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  while (!host->done) {
    Ops<T>::apply_dot(L, 1, p.p, q.p, red, FIN_CG_PAP, st, s);
    Ops<T>::cg_update(len, x, p.p, r.p, q.p, st, red, st, s);
    GKB_CUDA(cudaMemcpyAsync(host, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
    if (host->done) break;
    if (pre) pre->vcycle(r.p, zp, s);
    if (flex) Ops<T>::dot2(len, r.p, zp, q.p, red, FIN_FCG_RZ, st, s);
    else Ops<T>::dot(len, r.p, zp, red, FIN_CG_RZ, st, s);
    Ops<T>::cg_dir(len, p.p, zp, st, 0, s);
  }
  if (flex && fallback_restart(st, host, s)) {
    // plain GMG-PCG from the current iterate (beta of the first step is 0)
    while (!host->done) {
      pre->vcycle(r.p, zp, s, false);
      Ops<T>::dot(len, r.p, zp, red, FIN_CG_RZ, st, s);
      Ops<T>::cg_dir(len, p.p, zp, st, 0, s);
      Ops<T>::apply_dot(L, 1, p.p, q.p, red, FIN_CG_PAP, st, s);
      Ops<T>::cg_update(len, x, p.p, r.p, q.p, st, red, st, s);
      GKB_CUDA(cudaMemcpyAsync(host, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      GKB_CUDA(cudaStreamSynchronize(s));
    }
  }
  if (iters) *iters = host->it;
  return host->status;
}

template struct Cg<double>;
template struct Cg<float>;

// ---------------------------------------------------------------------------
// GKB kernels (FP64): launch wrappers of the bodies in gkb_device.cuh
// ---------------------------------------------------------------------------

static dim3 cgrid(const Lvl& L) { return dim3((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]); }

__global__ void __launch_bounds__(256) k_gkb_b(Lvl L, const double* __restrict__ rc, const double* __restrict__ y0,
                                               double* __restrict__ b, const GkbState* st, RedBuf red, double* out) {
  gkb_b_body(native_blk(), L, rc, y0, b, st, red, out);
}

__global__ void __launch_bounds__(256) k_gk1(Lvl L, const double* __restrict__ v, const double* __restrict__ q,
                                             double* __restrict__ gq, const GkbState* st, RedBuf red, double* out) {
  gk1_body(native_blk(), L, v, q, gq, st, red, out);
}

// out = w * a on the in-domain cells (N^-1 r of the right-hand-side transform)
__global__ void __launch_bounds__(256) k_cells_mul(Lvl L, const double* __restrict__ a, const double* __restrict__ w,
                                                   double* __restrict__ out) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= L.n[0] || j >= L.n[1]) return;
  const long long id = cix(L, i, j, k);
  out[id] = a[id] * w[id];
}

__global__ void __launch_bounds__(256) k_gk2(Lvl L, const double* __restrict__ gq, double* __restrict__ f,
                                             const GkbState* st) {
  gk2_body(native_blk(), L, gq, f, st);
}

__global__ void __launch_bounds__(CB) k_gk3(long long len, const double* __restrict__ x, const double* __restrict__ v,
                                            double* __restrict__ w, const GkbState* st) {
  gk3_body(native_blk(), len, x, v, w, st);
}

__global__ void __launch_bounds__(CB) k_gk4v(long long len, const double* __restrict__ w, double* __restrict__ v,
                                             double* __restrict__ u, const GkbState* st, int first) {
  gk4v_body(native_blk(), len, w, v, u, st, first);
}

__global__ void __launch_bounds__(256) k_gk4c(Lvl L, const double* __restrict__ gq, double* __restrict__ q,
                                              double* __restrict__ d, double* __restrict__ p, const GkbState* st,
                                              int first) {
  gk4c_body(native_blk(), L, gq, q, d, p, st, first);
}

__global__ void __launch_bounds__(256) k_gkb_q1(Lvl L, const double* __restrict__ b, double* __restrict__ q,
                                                const GkbState* st) {
  gkb_q1_body(native_blk(), L, b, q, st);
}

// scalar part of Algorithm 1 and the stopping rule (single thread)
__global__ void k_gkb_scalar(int op, GkbState* st, const double* red) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  gkb_scalar_op(op, st, red);
}

// pressure sum for the mean-zero projection
__global__ void __launch_bounds__(256) k_cell_sum(Lvl L, const double* __restrict__ p, RedBuf red, double* out) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  double v[1] = {0.0};
  if (i < L.n[0] && j < L.n[1]) v[0] = p[cix(L, i, j, k)];
  grid_reduce<1>(v, red, FIN_STORE, out);
}

__global__ void __launch_bounds__(CB) k_cvt_f32(long long len, const double* __restrict__ r, float* __restrict__ o,
                                                const int* pred) {
  cvt_f32_body(native_blk(), len, r, o, pred);
}


__global__ void __launch_bounds__(CB) k_mixed_accum(long long len, float* __restrict__ x32, double* __restrict__ x64,
                                                    const int* pred) {
  mixed_accum_body(native_blk(), len, x32, x64, pred);
}

// ---- device-side control of the graph form --------------------------------

// header of an inner CG solve (written on the device so that graphs can
// start a solve without a host copy)
__global__ void k_cg_setup(CgState* c, double tol2, int maxit, double delta2, double rho2) {
  c->tol2 = tol2;
  c->maxit = maxit;
  c->delta2 = delta2;
  c->rho2 = rho2;
  c->done = 0;
  c->status = ST_OK;
  c->it = 0;
  c->update = 0;
  c->graph_iters = 0;
  c->fallback = 0;
  c->fb_iters = 0;
}

// start of the fallback loop: run it when the flexible solve handed over
// (restarting the directions: beta of the first step is 0)
__global__ void k_fb_init(cudaGraphConditionalHandle h, CgState* c) {
  bool go = c->fallback && c->status == ST_OK;
  if (go && c->it >= c->maxit) {
    c->status = ST_INNER_NOT_CONVERGED;
    go = false;
  }
  if (go) {
    c->done = 0;
    c->rz_old = 0.0;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// small problems: a whole unpreconditioned CG solve in one thread-block
// cluster (FP64 work spread over the cluster's SMs, hardware cluster
// barriers instead of kernel launches between the steps)
// ---------------------------------------------------------------------------
constexpr int SB = 256;   // threads per block of the cluster solve

// sums over the cluster of NV values, returned to every thread: block sums
// in a fixed order, then the blocks' sums in rank order through distributed
// shared memory (deterministic). part[2][NV] alternates between calls, so
// one cluster barrier per call suffices: a block rewrites a slot only after
// the next call's barrier, which every block passes after it has read it.
template <int NV>
__device__ void cluster_sums(double (&v)[NV], double (*sh)[32], double (*part)[4], int& phase) {
  namespace cgx = cooperative_groups;
  cgx::cluster_group cl = cgx::this_cluster();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double w = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double w = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
      w = warp_sum(w);
      if (lane == 0) part[phase][k] = w;
    }
  }
  cl.sync();
  if (warp == 0) {
    const unsigned nb = cl.num_blocks();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double w = (unsigned)lane < nb ? cl.map_shared_rank(&part[phase][0], (unsigned)lane)[k] : 0.0;
      w = warp_sum(w);
      if (lane == 0) sh[k][0] = w;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sh[k][0];
  __syncthreads();  // sh is rewritten by the next call
  phase ^= 1;
}

// q = M p on this block's share of the face positions; returns (p, q) over it
template <bool VarMu>
__device__ __forceinline__ double apply_share(const Lvl& L, const double* p, double* q, int p0, int p1, int nx, int ny) {
  double pq = 0.0;
  for (int t = p0 + (int)threadIdx.x; t < p1; t += (int)blockDim.x) {
    const int i = t % nx, u = t / nx;
    const int j = u % ny, k = u / ny;
    const int pos[3] = {i, j, k};
    const long long cb = cix(L, i, j, k);
    if (face_active<0>(L, i, j, k)) {
      const double v = m_row<double, VarMu, 0, false>(L, p, pos);
      q[L.off[0] + cb] = v;
      pq += p[L.off[0] + cb] * v;
    }
    if (face_active<1>(L, i, j, k)) {
      const double v = m_row<double, VarMu, 1, false>(L, p, pos);
      q[L.off[1] + cb] = v;
      pq += p[L.off[1] + cb] * v;
    }
    if (L.dim == 3 && face_active<2>(L, i, j, k)) {
      const double v = m_row<double, VarMu, 2, false>(L, p, pos);
      q[L.off[2] + cb] = v;
      pq += p[L.off[2] + cb] * v;
    }
  }
  return pq;
}

// M x = f from x = 0 by CG in the one-reduction form of Chronopoulos and
// Gear (the CG iterates, with the two inner products of an iteration fused:
// gamma = (r, r), delta = (M r, r); beta = gamma / gamma_prev, the step
// alpha = gamma / (delta - beta gamma / alpha_prev) = gamma / (p, M p);
// p = r + beta p, s = M r + beta s, x += alpha p, r -= alpha s). The stopping
// rule is that of the multi-kernel form: ||r||^2 <= tol2 ||f||^2 on the
// recursive residual. Block `rank` of the cluster owns one contiguous share of
// the face positions and one of the padded arrays (balanced over the
// cluster's SMs); arrays the kernel rewrites are read with plain coherent
// loads. Two cluster barriers per iteration; the final state goes to c.
template <bool VarMu>
__global__ void __launch_bounds__(SB) k_cg_cluster(Lvl L, const double* __restrict__ f, double* __restrict__ x,
                                                    double* __restrict__ r, double* __restrict__ p,
                                                    double* __restrict__ w, double* __restrict__ sv, CgState* c,
                                                    double tol2, int maxit) {
  namespace cgx = cooperative_groups;
  cgx::cluster_group cl = cgx::this_cluster();
  __shared__ double sh[2][32];
  __shared__ double part[2][4];
  int phase = 0;
  const int rank = (int)cl.block_rank(), nb = (int)cl.num_blocks(), tid = threadIdx.x;
  const int len = (int)L.nvel;
  const int nx = L.n[0] + 1, ny = L.n[1] + 1, nz = (L.dim == 3) ? L.n[2] + 1 : 1;
  const int npos = nx * ny * nz;
  const int vch = (len + nb - 1) / nb, pch = (npos + nb - 1) / nb;
  const int v0 = rank * vch, v1 = min(len, v0 + vch);
  const int p0 = rank * pch, p1 = min(npos, p0 + pch);
  double ff = 0.0;
  for (int t = v0 + tid; t < v1; t += SB) {
    const double ft = f[t];
    x[t] = 0.0;
    r[t] = ft;
    p[t] = 0.0;
    sv[t] = 0.0;
    ff += ft * ft;
  }
  cl.sync();  // r complete
  double g[2] = {ff, apply_share<VarMu>(L, r, w, p0, p1, nx, ny)};  // (r, r), (M r, r)
  cluster_sums<2>(g, sh, part, phase);
  ff = g[0];
  double gamma = g[0], delta = g[1], gamma_prev = 0.0, alpha = 0.0;
  int it = 0, status = ST_OK;
  if (!isfinite(ff) || !isfinite(delta)) status = ST_NAN;
  bool done = (ff == 0.0) || status != ST_OK;
  while (!done) {
    double beta = 0.0, den = delta;
    if (it > 0) {
      beta = gamma / gamma_prev;
      den = delta - beta * gamma / alpha;
    }
    if (!(den > 0.0)) { status = isfinite(den) ? ST_NOT_SPD : ST_NAN; break; }
    alpha = gamma / den;
    double rr = 0.0;
    for (int t = v0 + tid; t < v1; t += SB) {
      const double pt = r[t] + beta * p[t];
      const double st = w[t] + beta * sv[t];
      p[t] = pt;
      sv[t] = st;
      x[t] += alpha * pt;
      const double rt = r[t] - alpha * st;
      r[t] = rt;
      rr += rt * rt;
    }
    ++it;
    cl.sync();  // r complete before the product reads neighbours
    double h[2] = {rr, apply_share<VarMu>(L, r, w, p0, p1, nx, ny)};
    cluster_sums<2>(h, sh, part, phase);
    gamma_prev = gamma;
    gamma = h[0];
    delta = h[1];
    if (!isfinite(gamma) || !isfinite(delta)) { status = ST_NAN; break; }
    if (gamma <= tol2 * ff) break;
    if (it >= maxit) { status = ST_INNER_NOT_CONVERGED; break; }
  }
  if (rank == 0 && tid == 0) {
    c->ff = ff;
    c->rr = gamma;
    c->it = it;
    c->total_it += it;
    c->solves += 1;
    c->status = status;
    c->done = 1;
    c->graph_iters = 0;
    c->fb_iters = 0;
    c->fallback = 0;
  }
}

// record an inner solve in the GKB state: status, iterations, history
__global__ void k_note_inner(GkbState* S, const CgState* c) {
  const int idx = S->inner_solves;
  if (S->h_inner && idx < S->icap) S->h_inner[idx] = c->it;
  S->inner_solves = idx + 1;
  S->inner_its += c->it;
  S->inner_runs += c->graph_iters;
  S->inner_fb_runs += c->fb_iters;
  S->inner_fallbacks += c->fallback;
  if (c->status != ST_OK && S->inner_status == ST_OK) S->inner_status = c->status;
}

__global__ void k_gkb_cond_init(cudaGraphConditionalHandle h, GkbState* S) {
  S->outer_runs = 0;
  cudaGraphSetConditional(h, (S->stop || S->status != ST_OK) ? 0u : 1u);
}

// continue the outer loop while Algorithm 1 has not stopped; hard_max bounds
// it even if the iteration counter were never advanced
__global__ void k_gkb_cond(cudaGraphConditionalHandle h, GkbState* S, int hard_max) {
  S->outer_runs += 1;
  unsigned cont = (S->stop || S->status != ST_OK) ? 0u : 1u;
  if (S->outer_runs >= hard_max) {
    cont = 0u;
    S->stop = 1;
  }
  cudaGraphSetConditional(h, cont);
}

// compact pressure with the mean (sum / n, sum on the device) removed
__global__ void k_unpack_cell_dev(Lvl L, const double* __restrict__ src, double* __restrict__ dst, const double* sum,
                                  double inv_n) {
  const long long n = (long long)L.n[0] * L.n[1] * L.n[2];
  const double shift = sum ? *sum * inv_n : 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / L.n[0];
    const int i = (int)(t - row * L.n[0]);
    const int k = (int)(row / L.n[1]);
    const int j = (int)(row - (long long)k * L.n[1]);
    dst[t] = src[cix(L, i, j, k)] - shift;
  }
}

// x64 += s e32 with s = sqrt(*nrm2) (precision conversion of a preconditioned vector)
__global__ void __launch_bounds__(CB) k_add_f32(long long len, const float* __restrict__ e, double* __restrict__ x,
                                                const double* nrm2) {
  const double s = sqrt(*nrm2);
  for (long long t = blockIdx.x * (long long)CB + threadIdx.x; t < len; t += (long long)gridDim.x * CB)
    x[t] += s * (double)e[t];
}

// ---------------------------------------------------------------------------
// Solver
// ---------------------------------------------------------------------------

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) { (void)cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static unsigned lin_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 1216) b = 1216;
  return (unsigned)(b < 1 ? 1 : b);
}

// compact ordering of include/gkb.h <-> padded layout of level L (the
// layout kernels above, for callers outside this file)
void pack_velocity(const Lvl& L, const double* compact, double* padded, cudaStream_t s) {
  const Compact c = make_compact(L);
  k_pack_vel<double><<<lin_blocks(c.m), 256, 0, s>>>(L, c, compact, padded);
}
void unpack_velocity(const Lvl& L, const double* padded, double* compact, cudaStream_t s) {
  const Compact c = make_compact(L);
  k_unpack_vel<<<lin_blocks(c.m), 256, 0, s>>>(L, c, padded, compact);
}
void pack_cells(const Lvl& L, const double* compact, double* padded, cudaStream_t s) {
  k_pack_cell<double><<<lin_blocks((long long)L.n[0] * L.n[1] * L.n[2]), 256, 0, s>>>(L, compact, padded);
}
void unpack_cells(const Lvl& L, const double* padded, double* compact, cudaStream_t s) {
  k_unpack_cell<<<lin_blocks((long long)L.n[0] * L.n[1] * L.n[2]), 256, 0, s>>>(L, padded, compact, 0.0);
}

Solver::~Solver() {
  sgraph.destroy();
  if (cg_host) cudaFreeHost(cg_host);
  if (gkb_host) cudaFreeHost(gkb_host);
  if (cap1) cudaStreamDestroy(cap1);
  if (cap2) cudaStreamDestroy(cap2);
  if (cap3) cudaStreamDestroy(cap3);
  if (cap4) cudaStreamDestroy(cap4);
}

void Solver::set_problem(const gkb_grid* g, const double* viscosity, double mu0_, double gamma_, double n_scale_,
                         const double* n_diag) {
  auto t0 = std::chrono::steady_clock::now();
  if (!g) throw Error{GKB_ERR_INVALID_ARG, "grid is NULL"};
  sgraph.destroy();
  forget_batches(this);
  if (g->dim != 2 && g->dim != 3) throw Error{GKB_ERR_INVALID_ARG, "dim must be 2 or 3"};
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] < 2) throw Error{GKB_ERR_INVALID_ARG, "every side needs at least 2 cells"};
  if (!(g->h > 0)) throw Error{GKB_ERR_INVALID_ARG, "h must be positive"};
  for (int s = 0; s < 2 * g->dim; ++s)
    if (g->bc[s] != GKB_BC_DIRICHLET && g->bc[s] != GKB_BC_NATURAL) throw Error{GKB_ERR_INVALID_ARG, "bad boundary type"};
  if (!(gamma_ >= 0)) throw Error{GKB_ERR_INVALID_ARG, "gamma must be >= 0"};
  if (!viscosity && !(mu0_ > 0)) throw Error{GKB_ERR_INVALID_ARG, "mu0 must be positive"};
  have_problem = false;
  grid = *g;
  gamma = gamma_;
  mu0 = mu0_;
  // with a diagonal N, n_scale is the reference h^d: the levels hold
  // gamma / h^d and every cell the weight h^d / N_cell
  n_scale = (n_scale_ > 0 && !n_diag) ? n_scale_ : pow(g->h, g->dim);
  int nat[6] = {0, 0, 0, 0, 0, 0};
  enclosed = true;
  for (int s = 0; s < 2 * g->dim; ++s) { nat[s] = g->bc[s] == GKB_BC_NATURAL; if (nat[s]) enclosed = false; }
  const bool use_gmg = opt.inner == GKB_INNER_GMG_PCG || opt.inner == GKB_INNER_FGMRES || learned_inner();
  if (opt.inner == GKB_INNER_FGMRES && opt.precision != GKB_PREC_FP64)
    throw Error{GKB_ERR_INVALID_ARG, "the FGMRES inner solver runs in FP64"};
  if (use_gmg && !enclosed)
    throw Error{GKB_ERR_INVALID_ARG, "the multigrid preconditioner needs Dirichlet velocity on every side"};
  const bool symgrad = opt.viscous_form == GKB_VISC_SYMGRAD;
  if (symgrad && !enclosed)
    throw Error{GKB_ERR_INVALID_ARG, "the symmetric-gradient form needs Dirichlet velocity on every side"};
  if (learned_inner() && g->dim != 2)
    throw Error{GKB_ERR_INVALID_ARG, "the learned inner solver is 2D only"};
  int n3[3] = {g->n[0], g->n[1], g->dim == 3 ? g->n[2] : 1};
  L64 = make_level(g->dim, n3, g->h, nat, gamma / n_scale);
  ncell = (int64_t)n3[0] * n3[1] * n3[2];
  // a non-uniform N and the symmetric-gradient form run on the
  // variable-viscosity kernels, which carry the per-cell weights and the
  // cross couplings: a constant viscosity becomes an array of mu0
  std::vector<double> mu_fill;
  if ((n_diag || symgrad) && !viscosity) {
    mu_fill.assign((size_t)ncell, mu0);
    viscosity = mu_fill.data();
  }
  L64.mu0 = viscosity ? 1.0 : mu0;
  L64.sym = symgrad ? 1 : 0;
  // fast paths: measured faster in FP32, slower in FP64 (FP64-pipe bound)
  L64.fast = (opt.kernel_variant == 2) ? 1 : 0;
  finish_level(L64);
  Compact cmp = make_compact(L64);
  m = cmp.m;
  // viscosity
  mu64.release();
  mu32.release();
  const bool mixed = opt.precision == GKB_PREC_MIXED;
  if (viscosity) {
    DevBuf<double> tmp;
    tmp.alloc(ncell);
    GKB_CUDA(cudaMemcpyAsync(tmp.p, viscosity, ncell * sizeof(double), cudaMemcpyDefault, stream));
    mu64.alloc(L64.ncell);
    { ProfScope ps_(GKB_KC_LAYOUT, stream); k_pack_cell<double><<<lin_blocks(ncell), 256, 0, stream>>>(L64, tmp.p, mu64.p); }
    if (mixed) {
      mu32.alloc(L64.ncell);
      { ProfScope ps_(GKB_KC_LAYOUT, stream); k_pack_cell<float><<<lin_blocks(ncell), 256, 0, stream>>>(L64, tmp.p, mu32.p); }
    }
    GKB_CUDA(cudaStreamSynchronize(stream));
    std::vector<double> hv(ncell);
    GKB_CUDA(cudaMemcpy(hv.data(), tmp.p, ncell * sizeof(double), cudaMemcpyDeviceToHost));
    for (double vv : hv)
      if (!(vv > 0) || !std::isfinite(vv)) throw Error{GKB_ERR_INVALID_ARG, "viscosity must be positive and finite"};
  }
  L64.mu64 = mu64.p;
  // diagonal N
  nd64.release();
  nw64.release();
  nw32.release();
  diag_n = n_diag != nullptr;
  nsum = ninvsum = 0;
  if (diag_n) {
    DevBuf<double> tmp;
    tmp.alloc(ncell);
    GKB_CUDA(cudaMemcpyAsync(tmp.p, n_diag, ncell * sizeof(double), cudaMemcpyDefault, stream));
    std::vector<double> hn(ncell);
    GKB_CUDA(cudaMemcpyAsync(hn.data(), tmp.p, ncell * sizeof(double), cudaMemcpyDeviceToHost, stream));
    GKB_CUDA(cudaStreamSynchronize(stream));
    std::vector<double> hw(ncell);
    for (int64_t c = 0; c < ncell; ++c) {
      if (!(hn[c] > 0) || !std::isfinite(hn[c])) throw Error{GKB_ERR_INVALID_ARG, "N must be positive and finite"};
      nsum += hn[c];
      ninvsum += 1.0 / hn[c];
      hw[c] = n_scale / hn[c];
    }
    nd64.alloc(L64.ncell);
    nw64.alloc(L64.ncell);
    { ProfScope ps_(GKB_KC_LAYOUT, stream); k_pack_cell<double><<<lin_blocks(ncell), 256, 0, stream>>>(L64, tmp.p, nd64.p); }
    GKB_CUDA(cudaMemcpyAsync(tmp.p, hw.data(), ncell * sizeof(double), cudaMemcpyHostToDevice, stream));
    { ProfScope ps_(GKB_KC_LAYOUT, stream); k_pack_cell<double><<<lin_blocks(ncell), 256, 0, stream>>>(L64, tmp.p, nw64.p); }
    if (mixed) {
      nw32.alloc(L64.ncell);
      { ProfScope ps_(GKB_KC_LAYOUT, stream); k_pack_cell<float><<<lin_blocks(ncell), 256, 0, stream>>>(L64, tmp.p, nw32.p); }
    }
    GKB_CUDA(cudaStreamSynchronize(stream));
  }
  L64.nw64 = nw64.p;
  L64.nw32 = nullptr;
  L32 = L64;
  L32.mu64 = nullptr;
  L32.mu32 = mu32.p;
  L32.nw64 = nullptr;
  L32.nw32 = nw32.p;
  // node / edge viscosity table (variable viscosity, FP64 levels only: see
  // Gmg<T>::build)
  em64.release();
  L64.em64 = nullptr;
  L64.em32 = nullptr;
  L32.em64 = nullptr;
  L32.em32 = nullptr;
  L64.sym = L32.sym = symgrad ? 1 : 0;
  if (mu64.p) {
    em64.alloc(Ops<double>::edge_table_len(L64));
    Ops<double>::edge_table(L64, em64.p, stream);
    L64.em64 = em64.p;
  }
  GKB_CUDA(cudaGetLastError());
  L32.fast = (opt.kernel_variant == 1) ? 0 : 1;
  // reduction scratch: enough partials for every launch shape used
  long long blocks = std::max<long long>(Ops<double>::face_blocks(L64), blas_blocks(L64.nvel));
  blocks = std::max<long long>(blocks, (long long)cgrid(L64).x * cgrid(L64).y * cgrid(L64).z);
  red_partial.alloc((size_t)blocks * 4 + 64);
  red_ticket.alloc(1);
  red = RedBuf{red_partial.p, red_ticket.p};
  scal.alloc(16);
  if (!cg_host) {
    GKB_CUDA(cudaMallocHost(&cg_host, sizeof(CgState)));
    GKB_CUDA(cudaMallocHost(&gkb_host, sizeof(GkbState)));
  }
  state_mem.alloc(sizeof(CgState) + sizeof(GkbState) + 256);
  cg_dev = (CgState*)state_mem.p;
  gkb_dev = (GkbState*)(state_mem.p + ((sizeof(CgState) + 127) / 128) * 128);
  // GKB vectors
  stats = gkb_stats_t{};
  if (mixed) {
    r64.alloc(L64.nvel);
    f32.alloc(L64.nvel);
    x32.alloc(L64.nvel);
  }
  for (DevBuf<double>* b : {&u, &v, &x, &w, &t, &f, &y0, &wtmp}) b->alloc(L64.nvel);
  for (DevBuf<double>* b : {&q, &d, &pp, &gq, &bc, &ctmp}) b->alloc(L64.ncell);
  stage_m.alloc(m);
  stage_n.alloc(ncell);
  hist.alloc(4 * (size_t)(opt.maxit + 2));
  hist_inner.alloc((size_t)opt.maxit + 4);
  // multigrid + CG (tuned first when asked; the FGMRES work space first, as
  // the tuner times whole inner solves)
  tuned_ms = 0;
  if (opt.inner == GKB_INNER_FGMRES) fgm.init(L64.nvel, opt.fgmres_restart);
  if (opt.autotune && use_gmg) autotune_inner(viscosity != nullptr, diag_n ? 1 : 0);
  else build_inner();
  stats.tuned_inner_ms = tuned_ms;
  attach_net_levels();
  GKB_CUDA(cudaStreamSynchronize(stream));
  generation += 1;
  have_problem = true;
  build_solve_graph();
  stats.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Multigrid hierarchy and CG of the handle's precision from the current
// options (smoother degree, coarse size, kernel variant).
void Solver::build_inner() {
  const bool mixed = opt.precision == GKB_PREC_MIXED;
  const bool use_gmg = opt.inner == GKB_INNER_GMG_PCG || opt.inner == GKB_INNER_FGMRES || learned_inner();
  // deep-interior fast paths: variant 0 enables them in FP32 only (faster
  // there, slower on the FP64 pipe), 1 nowhere, 2 everywhere
  L64.fast = (opt.kernel_variant == 2) ? 1 : 0;
  L32.fast = (opt.kernel_variant == 1) ? 0 : 1;
  gmg32.cheb_lo = gmg64.cheb_lo = opt.cheb_lo;
  gmg32.cheb_hi = gmg64.cheb_hi = opt.cheb_hi;
  gmg32.tail_side = gmg64.tail_side = opt.tail_side;
  if (mixed) {
    if (use_gmg) gmg32.build(L32, mu32.p, opt.coarse_max, opt.smoother_degree, red, scal.p, stream);
    cg32.init(L32, use_gmg ? &gmg32 : nullptr, red, cg_dev, cg_host);
    cg32.flex = learned_inner();
    cg32.rho2 = opt.fcg_rho * opt.fcg_rho;
    stats.levels = use_gmg ? (int)gmg32.lev.size() : 0;
  } else {
    if (use_gmg) gmg64.build(L64, mu64.p, opt.coarse_max, opt.smoother_degree, red, scal.p, stream);
    cg64.init(L64, use_gmg ? &gmg64 : nullptr, red, cg_dev, cg_host);
    cg64.flex = learned_inner();
    cg64.rho2 = opt.fcg_rho * opt.fcg_rho;
    stats.levels = use_gmg ? (int)gmg64.lev.size() : 0;
  }
}

// Device time (ms) of one inner solve M x = f, run as a captured graph like
// the solver's own; +inf when it fails. f = A A^T h for a fixed pseudo-random
// h lies in the range of A like the right-hand sides A q of the GKB loop.
double Solver::time_inner_solve(int* its) {
  ensure_capture_streams();
  { ProfScope ps_(GKB_KC_LAYOUT, stream); k_fill_hash<double><<<fgrid(L64), dim3(32, 8), 0, stream>>>(L64, wtmp.p); }
  Ops<double>::negdiv(L64, wtmp.p, ctmp.p, 1.0, stream);
  Ops<double>::grad(L64, ctmp.p, f.p, 1.0, stream);
  GKB_CUDA(cudaStreamSynchronize(stream));
  Profiler* P = g_prof;
  const int saved = P ? P->phase : -1;
  if (P) P->phase = 0;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  try {
    GKB_CUDA(cudaGraphCreate(&g, 0));
    GKB_CUDA(cudaStreamBeginCaptureToGraph(cap1, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capture_inner(cap1, cap2);
    GKB_CUDA(cudaStreamEndCapture(cap1, &g));
    GKB_CUDA(cudaGraphInstantiate(&ge, g, 0));
  } catch (...) {
    if (P) P->phase = saved;
    abandon_captures({cap4, cap3, cap2, cap1});
    if (g) cudaGraphDestroy(g);
    throw;
  }
  if (P) P->phase = saved;
  cudaGraphDestroy(g);
  double best = 1e300;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GKB_CUDA(cudaEventCreate(&e0));
  GKB_CUDA(cudaEventCreate(&e1));
  bool ok = true;
  for (int rep = 0; rep < 4 && ok; ++rep) {
    GKB_CUDA(cudaEventRecord(e0, stream));
    GKB_CUDA(cudaGraphLaunch(ge, stream));
    GKB_CUDA(cudaEventRecord(e1, stream));
    GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, stream));
    GKB_CUDA(cudaStreamSynchronize(stream));
    float ms = 0.f;
    GKB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ok = cg_host->status == ST_OK;
    if (rep > 0) best = std::min(best, (double)ms);  // the first launch warms up
    if (its) *its = cg_host->it;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  return ok ? best : 1e300;
}

namespace {
struct Tuned {
  int degree, variant, coarse_max;
  double lo, ms;
  int its = 0;   // iterations of the timed solve (tie-break; not stored in the file)
  int tail = 0;  // tail_side
};
std::mutex g_tune_mutex;
std::map<std::string, Tuned> g_tune_cache;
bool g_tune_file_read = false;

const char* tune_file() {
  const char* p = getenv("GKB_TUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

void tune_read_file() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = tune_file();
  if (!path) return;
  FILE* fp = fopen(path, "r");
  if (!fp) return;
  // one entry per line: key degree variant coarse_max cheb_lo ms [tail_side]
  char line[1024], key[512];
  while (fgets(line, sizeof line, fp)) {
    Tuned t{};
    const int n = sscanf(line, "%511s %d %d %d %lf %lf %d", key, &t.degree, &t.variant, &t.coarse_max, &t.lo, &t.ms,
                         &t.tail);
    if (n < 6) break;
    if (n == 6) t.tail = 0;
    g_tune_cache[key] = t;
  }
  fclose(fp);
}
}  // namespace

// Autotuner: search the inner solver's smoother degree (1..3), kernel variant
// (0..2), coarse size (8, 16, 32) and the lower end of the Chebyshev interval
// (0.05 .. 0.3 of lambda_max) one after another, each by the device
// time of a whole inner solve to tol_inner, and keep the fastest; results are
// cached per device, grid, viscosity kind, precision, inner solver and gamma
// decade, in the process and (GKB_TUNE_CACHE) in a text file.
void Solver::autotune_inner(bool var_mu, int weighted) {
  int dev = 0;
  GKB_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  GKB_CUDA(cudaGetDeviceProperties(&prop, dev));
  std::string name(prop.name);
  for (char& c : name)
    if (c == ' ') c = '_';
  char key[512];
  snprintf(key, sizeof key, "%s|d%d|%dx%dx%d|%s|p%d|i%d|g%+.0f", name.c_str(), grid.dim, L64.n[0], L64.n[1], L64.n[2],
           var_mu ? (weighted ? (L64.sym ? "symgrad-ndiag" : "varmu-ndiag") : (L64.sym ? "symgrad" : "varmu")) : "mu",
           opt.precision, opt.inner, gamma > 0 ? std::floor(std::log10(gamma)) : -99.0);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_read_file();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      opt.smoother_degree = it->second.degree;
      opt.kernel_variant = it->second.variant;
      opt.coarse_max = it->second.coarse_max;
      opt.cheb_lo = it->second.lo;
      opt.tail_side = it->second.tail;
      tuned_ms = it->second.ms;
      build_inner();
      return;
    }
  }
  Tuned best{opt.smoother_degree, opt.kernel_variant, opt.coarse_max, opt.cheb_lo, 1e300, 0, opt.tail_side};
  // a candidate replaces the best when it is faster by more than the timing
  // noise (2 %), or when the two are within it and the candidate needs fewer
  // iterations (a stronger preconditioner: more work per launch, which also
  // holds up better when several solves share the GPU)
  auto trial = [&](int deg, int var, int cmax, double lo, int tail) {
    opt.smoother_degree = deg;
    opt.kernel_variant = var;
    opt.coarse_max = cmax;
    opt.cheb_lo = lo;
    opt.tail_side = tail;
    double ms = 1e300;
    int its = 0;
    try {
      build_inner();
      ms = time_inner_solve(&its);
    } catch (const Error& e) {
      if (e.code != GKB_ERR_INVALID_ARG) throw;  // an infeasible candidate (coarse level too large)
    }
    if (!(ms < 1e300)) return;
    const bool faster = ms < 0.98 * best.ms;
    const bool tie = !faster && ms <= 1.02 * best.ms && its < best.its;
    if (faster || tie) best = Tuned{deg, var, cmax, lo, ms, its, tail};
  };
  const double lo0 = best.lo;
  const int t0 = best.tail;
  trial(best.degree, best.variant, best.coarse_max, lo0, t0);
  for (int v = 0; v <= 2; ++v)
    if (v != best.variant) trial(best.degree, v, best.coarse_max, lo0, t0);
  const int v0 = best.variant;
  for (int deg = 1; deg <= 3; ++deg)
    if (deg != best.degree) trial(deg, v0, best.coarse_max, lo0, t0);
  const int d0 = best.degree;
  for (int cmax : {8, 16, 32})
    if (cmax != best.coarse_max) trial(d0, v0, cmax, lo0, t0);
  const int c0 = best.coarse_max;
  for (double lo : {0.05, 0.1, 0.2, 0.3})
    if (lo != best.lo && lo < opt.cheb_hi) trial(d0, v0, c0, lo, t0);
  // the fused coarse end (2D, constant viscosity); with it the coarse size
  // is tried again (deeper hierarchies cost less when their end is fused)
  if (grid.dim == 2 && !var_mu) {
    const double l0 = best.lo;
    const int tb = best.tail == 64 ? 0 : 64;
    trial(d0, v0, c0, l0, tb);
    if (best.tail == 64)
      for (int cmax : {8, 16, 32})
        if (cmax != best.coarse_max) trial(d0, v0, cmax, l0, 64);
  }
  if (!(best.ms < 1e300)) throw Error{GKB_ERR_INNER_NOT_CONVERGED, "no autotuning candidate converged"};
  opt.smoother_degree = best.degree;
  opt.kernel_variant = best.variant;
  opt.coarse_max = best.coarse_max;
  opt.cheb_lo = best.lo;
  opt.tail_side = best.tail;
  tuned_ms = best.ms;
  build_inner();
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = best;
  if (const char* path = tune_file()) {
    if (FILE* fp = fopen(path, "a")) {
      fprintf(fp, "%s %d %d %d %.4f %.6f %d\n", key, best.degree, best.variant, best.coarse_max, best.lo, best.ms,
              best.tail);
      fclose(fp);
    }
  }
}

// The network gives the coarse correction of the level whose longer side is
// opt.unet_side cells (0: the finest level, i.e. the network alone).
void Solver::attach_net_levels() {
  gmg64.detach_net();
  gmg32.detach_net();
  if (!net || !learned_inner()) return;
  const bool composite = opt.inner == GKB_INNER_FCG_UNET_MG;
  const bool mixed = opt.precision == GKB_PREC_MIXED;
  const int nl = mixed ? (int)gmg32.lev.size() : (int)gmg64.lev.size();
  int level = -1;
  for (int l = 0; l < nl; ++l) {
    const Lvl& L = mixed ? gmg32.lev[l].L : gmg64.lev[l].L;
    const int side = std::max(L.n[0], L.n[1]);
    if ((opt.unet_side == 0 && l == 0) || side == opt.unet_side) { level = l; break; }
  }
  if (level < 0) throw Error{GKB_ERR_INVALID_ARG, "no multigrid level has unet_side cells per side"};
  if (mixed) gmg32.attach_net(net, level, composite, stream);
  else gmg64.attach_net(net, level, composite, stream);
}

void Solver::set_net(Unet* u) {
  net = u;
  if (!have_problem) return;
  sgraph.destroy();
  forget_batches(this);
  attach_net_levels();
  GKB_CUDA(cudaStreamSynchronize(stream));
  generation += 1;
  build_solve_graph();
}

// weights trained since the last solve: refresh their BF16 copy (the
// captured graphs read it at a fixed address)
void Solver::refresh_net() {
  if (net && net->bf16_stale && learned_inner()) net->refresh_bf16(stream);
}

void Solver::cell_sum(const double* p, double* out) {
  ProfScope ps_(GKB_KC_GKB, stream);
  k_cell_sum<<<cgrid(L64), dim3(32, 8), 0, stream>>>(L64, p, red, out);
  GKB_CUDA(cudaGetLastError());
}

// small unpreconditioned FP64 problems run each inner solve as one kernel
bool Solver::small_cg() const {
  return opt.inner == GKB_INNER_CG && opt.precision == GKB_PREC_FP64 && L64.nvel <= (1LL << 15);
}

// cluster size for k_cg_cluster: 16 blocks where the device allows it, else
// 8 (decided once per device and kernel)
static int cg_cluster_size(bool var_mu) {
  static std::mutex mtx;
  static std::map<int, int> cached;
  int dev = 0;
  GKB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mtx);
  int& cs = cached[2 * dev + (var_mu ? 1 : 0)];
  if (cs) return cs;
  const void* fn = var_mu ? (const void*)k_cg_cluster<true> : (const void*)k_cg_cluster<false>;
  cs = 8;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(SB);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) cs = 16;
  }
  (void)cudaGetLastError();
  return cs;
}

void Solver::launch_cg_block(const double* fpad, double* xpad, cudaStream_t s) {
  Cg<double>& c = cg64;
  ProfScope ps_(GKB_KC_APPLY, s, 0);  // unknowns counted per iteration in finish()
  const double tol2 = opt.tol_inner * opt.tol_inner;
  const bool var = L64.mu64 != nullptr;
  const int cs = cg_cluster_size(var);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(SB);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (var)
    GKB_CUDA(cudaLaunchKernelEx(&cfg, k_cg_cluster<true>, L64, fpad, xpad, c.r.p, c.p.p, c.q.p, c.z.p, cg_dev,
                                tol2, opt.maxit_inner));
  else
    GKB_CUDA(cudaLaunchKernelEx(&cfg, k_cg_cluster<false>, L64, fpad, xpad, c.r.p, c.p.p, c.q.p, c.z.p, cg_dev,
                                tol2, opt.maxit_inner));
}

int Solver::inner_solve(const double* fpad, double* xpad) {
  int its = 0, st = 0;
  if (opt.precision == GKB_PREC_MIXED) st = mixed_solve(fpad, xpad, &its);
  else if (opt.inner == GKB_INNER_FGMRES) {
    st = fgmres_solve(*this, fpad, xpad, &its);
    // the inner-solve record reads the CG state: its count and status
    CgState h{};
    h.it = its;
    h.status = st;
    h.done = 1;
    GKB_CUDA(cudaMemcpyAsync(cg_dev, &h, sizeof(CgState), cudaMemcpyHostToDevice, stream));
  } else if (small_cg()) {
    launch_cg_block(fpad, xpad, stream);
    GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, stream));
    GKB_CUDA(cudaStreamSynchronize(stream));
    st = cg_host->status;
  } else st = cg64.solve(fpad, xpad, opt.tol_inner, opt.maxit_inner, stream, &its);
  { ProfScope ps_(GKB_KC_GKB, stream); k_note_inner<<<1, 1, 0, stream>>>(gkb_dev, cg_dev); }
  return st;
}

// Mixed precision inner solve: conjugate gradients with FP32 vectors, FP32
// operator and FP32 V-cycle, whose solution is accumulated in FP64 and whose
// residual is recomputed in FP64 ("reliable update") each time the FP32
// residual has dropped by mixed_rtol since the last recomputation, and when
// it claims convergence. Convergence is judged on the FP64 residual only.
int Solver::mixed_solve(const double* f, double* x64, int* iters) {
  cudaStream_t s = stream;
  const long long len = L64.nvel;
  Cg<float>& c = cg32;
  CgState h{};
  h.tol2 = opt.tol_inner * opt.tol_inner;
  h.maxit = opt.maxit_inner;
  h.delta2 = opt.mixed_rtol > 0 ? opt.mixed_rtol * opt.mixed_rtol : -1.0;
  h.rho2 = c.flex ? c.rho2 : 0.0;
  GKB_CUDA(cudaMemcpyAsync(cg_dev, &h, sizeof(CgState), cudaMemcpyHostToDevice, s));
  GKB_CUDA(cudaMemsetAsync(x64, 0, len * sizeof(double), s));
  GKB_CUDA(cudaMemsetAsync(x32.p, 0, len * sizeof(float), s));
  Ops<double>::dot(len, f, f, red, FIN_CG_INIT, cg_dev, s);
  { ProfScope ps_(GKB_KC_LAYOUT, s, len); k_cvt_f32<<<lin_blocks(len), CB, 0, s>>>(len, f, c.r.p, nullptr); }
  float* zp = c.pre ? c.z.p : c.r.p;
  if (c.pre) c.pre->vcycle(c.r.p, zp, s);
  Ops<float>::dot(len, c.r.p, zp, red, FIN_CG_RZ0, cg_dev, s);
  Ops<float>::cg_dir(len, c.p.p, zp, cg_dev, 1, s);
  GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  while (!cg_host->done) {
    Ops<float>::apply_dot(L32, 1, c.p.p, c.q.p, red, FIN_CG_PAP, cg_dev, s);
    Ops<float>::cg_update(len, x32.p, c.p.p, c.r.p, c.q.p, cg_dev, red, cg_dev, s, FIN_MX_RR);
    GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
    if (cg_host->done) break;
    if (cg_host->update) {
      // x64 += x32, x32 = 0, r64 = f - M x64 (FP64), r32 = r64
      { ProfScope ps_(GKB_KC_LAYOUT, s, len); k_mixed_accum<<<lin_blocks(len), CB, 0, s>>>(len, x32.p, x64, nullptr); }
      Ops<double>::residual(L64, x64, f, r64.p, s);
      { ProfScope ps_(GKB_KC_LAYOUT, s, len); k_cvt_f32<<<lin_blocks(len), CB, 0, s>>>(len, r64.p, c.r.p, nullptr); }
      Ops<double>::dot(len, r64.p, r64.p, red, FIN_MX_RR64, cg_dev, s);
      GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      GKB_CUDA(cudaStreamSynchronize(s));
      if (cg_host->done) break;
    }
    if (c.pre) c.pre->vcycle(c.r.p, zp, s);
    if (c.flex) Ops<float>::dot2(len, c.r.p, zp, c.q.p, red, FIN_FCG_RZ, cg_dev, s);
    else Ops<float>::dot(len, c.r.p, zp, red, FIN_CG_RZ, cg_dev, s);
    Ops<float>::cg_dir(len, c.p.p, zp, cg_dev, 0, s);
  }
  auto reliable_update = [&]() {
    // x64 += x32, x32 = 0, r64 = f - M x64 (FP64), r32 = r64
    { ProfScope ps_(GKB_KC_LAYOUT, s, len); k_mixed_accum<<<lin_blocks(len), CB, 0, s>>>(len, x32.p, x64, nullptr); }
    Ops<double>::residual(L64, x64, f, r64.p, s);
    { ProfScope ps_(GKB_KC_LAYOUT, s, len); k_cvt_f32<<<lin_blocks(len), CB, 0, s>>>(len, r64.p, c.r.p, nullptr); }
    Ops<double>::dot(len, r64.p, r64.p, red, FIN_MX_RR64, cg_dev, s);
    GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
  };
  if (c.flex && fallback_restart(cg_dev, cg_host, s)) {
    // plain GMG-PCG from the current iterate (beta of the first step is 0)
    while (!cg_host->done) {
      c.pre->vcycle(c.r.p, zp, s, false);
      Ops<float>::dot(len, c.r.p, zp, red, FIN_CG_RZ, cg_dev, s);
      Ops<float>::cg_dir(len, c.p.p, zp, cg_dev, 0, s);
      Ops<float>::apply_dot(L32, 1, c.p.p, c.q.p, red, FIN_CG_PAP, cg_dev, s);
      Ops<float>::cg_update(len, x32.p, c.p.p, c.r.p, c.q.p, cg_dev, red, cg_dev, s, FIN_MX_RR);
      GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
      GKB_CUDA(cudaStreamSynchronize(s));
      if (cg_host->done) break;
      if (cg_host->update) reliable_update();
    }
  }
  // a solve that stopped on the FP32 side (NaN, not SPD) still returns the
  // FP64 accumulation of its progress
  { ProfScope ps_(GKB_KC_LAYOUT, s, len); k_mixed_accum<<<lin_blocks(len), CB, 0, s>>>(len, x32.p, x64, nullptr); }
  if (iters) *iters = cg_host->it;
  return cg_host->status;
}

void Solver::ensure_capture_streams() {
  if (!cap1) GKB_CUDA(cudaStreamCreateWithFlags(&cap1, cudaStreamNonBlocking));
  if (!cap2) GKB_CUDA(cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking));
  if (!cap3) GKB_CUDA(cudaStreamCreateWithFlags(&cap3, cudaStreamNonBlocking));
  if (!cap4) GKB_CUDA(cudaStreamCreateWithFlags(&cap4, cudaStreamNonBlocking));
}

// One inner solve x = M^-1 f in graph form (prefix; while; suffix), then its
// record in the GKB state. Straight-line parts count once per inner solve
// (profiler phase 2), the loop body once per iteration (phase 3).
void Solver::capture_inner(cudaStream_t s, cudaStream_t sb) {
  Profiler* P = g_prof;
  const int saved = P ? P->phase : -1;
  if (P) P->phase = 2;
  const long long len = L64.nvel;
  const double tol2 = opt.tol_inner * opt.tol_inner;
  const int maxit = opt.maxit_inner;
  if (opt.inner == GKB_INNER_FGMRES) {
    capture_fgmres(*this, s, sb, sb == cap3 ? cap4 : cap3);
  } else if (opt.precision == GKB_PREC_MIXED) {
    Cg<float>& c = cg32;
    float* zp = c.pre ? c.z.p : c.r.p;
    const int* upd = &cg_dev->update;
    const double delta2 = opt.mixed_rtol > 0 ? opt.mixed_rtol * opt.mixed_rtol : -1.0;
    capture_loop(
        s, sb, 3,
        [&](cudaStream_t st, cudaGraphConditionalHandle h) {
          k_cg_setup<<<1, 1, 0, st>>>(cg_dev, tol2, maxit, delta2, c.rho2);
          GKB_CUDA(cudaMemsetAsync(x.p, 0, len * sizeof(double), st));
          GKB_CUDA(cudaMemsetAsync(x32.p, 0, len * sizeof(float), st));
          Ops<double>::dot(len, f.p, f.p, red, FIN_CG_INIT, cg_dev, st);
          { ProfScope ps_(GKB_KC_LAYOUT, st, len); k_cvt_f32<<<lin_blocks(len), CB, 0, st>>>(len, f.p, c.r.p, nullptr); }
          if (c.pre) c.pre->vcycle(c.r.p, zp, st);
          Ops<float>::dot(len, c.r.p, zp, red, FIN_CG_RZ0, cg_dev, st);
          Ops<float>::cg_dir(len, c.p.p, zp, cg_dev, 1, st);
          k_cg_cond_init<<<1, 1, 0, st>>>(h, cg_dev);
        },
        [&](cudaStream_t st, cudaGraphConditionalHandle h) {
          Ops<float>::apply_dot(L32, 1, c.p.p, c.q.p, red, FIN_CG_PAP, cg_dev, st);
          Ops<float>::cg_update(len, x32.p, c.p.p, c.r.p, c.q.p, cg_dev, red, cg_dev, st, FIN_MX_RR);
          // reliable update, predicated on the flag the finaliser just set
          { ProfScope ps_(GKB_KC_LAYOUT, st, len); k_mixed_accum<<<lin_blocks(len), CB, 0, st>>>(len, x32.p, x.p, upd); }
          Ops<double>::residual(L64, x.p, f.p, r64.p, st, upd);
          { ProfScope ps_(GKB_KC_LAYOUT, st, len); k_cvt_f32<<<lin_blocks(len), CB, 0, st>>>(len, r64.p, c.r.p, upd); }
          Ops<double>::dot(len, r64.p, r64.p, red, FIN_MX_RR64, cg_dev, st, upd);
          if (c.pre) c.pre->vcycle(c.r.p, zp, st);
          if (c.flex) Ops<float>::dot2(len, c.r.p, zp, c.q.p, red, FIN_FCG_RZ, cg_dev, st);
          else Ops<float>::dot(len, c.r.p, zp, red, FIN_CG_RZ, cg_dev, st);
          Ops<float>::cg_dir(len, c.p.p, zp, cg_dev, 0, st);
          k_cg_cond<<<1, 1, 0, st>>>(h, cg_dev, maxit + 2);
        },
        [&](cudaStream_t st) {
          { ProfScope ps_(GKB_KC_LAYOUT, st, len); k_mixed_accum<<<lin_blocks(len), CB, 0, st>>>(len, x32.p, x.p, nullptr); }
        });
    if (c.flex && c.pre && c.pre->net) {
      // fallback: plain GMG-PCG from the current iterate when the flexible
      // solve handed over (zero trips otherwise); the step order is rotated
      // so that the restart needs no prefix of its own
      capture_loop(
          s, sb, 4, [&](cudaStream_t st, cudaGraphConditionalHandle h) { k_fb_init<<<1, 1, 0, st>>>(h, cg_dev); },
          [&](cudaStream_t st, cudaGraphConditionalHandle h) {
            c.pre->vcycle(c.r.p, zp, st, false);
            Ops<float>::dot(len, c.r.p, zp, red, FIN_CG_RZ, cg_dev, st);
            Ops<float>::cg_dir(len, c.p.p, zp, cg_dev, 0, st);
            Ops<float>::apply_dot(L32, 1, c.p.p, c.q.p, red, FIN_CG_PAP, cg_dev, st);
            Ops<float>::cg_update(len, x32.p, c.p.p, c.r.p, c.q.p, cg_dev, red, cg_dev, st, FIN_MX_RR);
            { ProfScope ps_(GKB_KC_LAYOUT, st, len); k_mixed_accum<<<lin_blocks(len), CB, 0, st>>>(len, x32.p, x.p, upd); }
            Ops<double>::residual(L64, x.p, f.p, r64.p, st, upd);
            { ProfScope ps_(GKB_KC_LAYOUT, st, len); k_cvt_f32<<<lin_blocks(len), CB, 0, st>>>(len, r64.p, c.r.p, upd); }
            Ops<double>::dot(len, r64.p, r64.p, red, FIN_MX_RR64, cg_dev, st, upd);
            k_cg_cond<<<1, 1, 0, st>>>(h, cg_dev, maxit + 4, 1);
          },
          [&](cudaStream_t st) {
            { ProfScope ps_(GKB_KC_LAYOUT, st, len); k_mixed_accum<<<lin_blocks(len), CB, 0, st>>>(len, x32.p, x.p, nullptr); }
          });
    }
  } else if (small_cg()) {
    launch_cg_block(f.p, x.p, s);
  } else {
    Cg<double>& c = cg64;
    double* zp = c.pre ? c.z.p : c.r.p;
    capture_loop(
        s, sb, 3,
        [&](cudaStream_t st, cudaGraphConditionalHandle h) {
          k_cg_setup<<<1, 1, 0, st>>>(cg_dev, tol2, maxit, 0.0, c.rho2);
          GKB_CUDA(cudaMemsetAsync(x.p, 0, len * sizeof(double), st));
          GKB_CUDA(cudaMemcpyAsync(c.r.p, f.p, len * sizeof(double), cudaMemcpyDeviceToDevice, st));
          Ops<double>::dot(len, f.p, f.p, red, FIN_CG_INIT, cg_dev, st);
          if (c.pre) c.pre->vcycle(c.r.p, zp, st);
          Ops<double>::dot(len, c.r.p, zp, red, FIN_CG_RZ0, cg_dev, st);
          Ops<double>::cg_dir(len, c.p.p, zp, cg_dev, 1, st);
          k_cg_cond_init<<<1, 1, 0, st>>>(h, cg_dev);
        },
        [&](cudaStream_t st, cudaGraphConditionalHandle h) {
          Ops<double>::apply_dot(L64, 1, c.p.p, c.q.p, red, FIN_CG_PAP, cg_dev, st);
          Ops<double>::cg_update(len, x.p, c.p.p, c.r.p, c.q.p, cg_dev, red, cg_dev, st);
          if (c.pre) c.pre->vcycle(c.r.p, zp, st);
          if (c.flex) Ops<double>::dot2(len, c.r.p, zp, c.q.p, red, FIN_FCG_RZ, cg_dev, st);
          else Ops<double>::dot(len, c.r.p, zp, red, FIN_CG_RZ, cg_dev, st);
          Ops<double>::cg_dir(len, c.p.p, zp, cg_dev, 0, st);
          k_cg_cond<<<1, 1, 0, st>>>(h, cg_dev, maxit + 2);
        },
        [&](cudaStream_t) {});
    if (c.flex && c.pre && c.pre->net) {
      capture_loop(
          s, sb, 4, [&](cudaStream_t st, cudaGraphConditionalHandle h) { k_fb_init<<<1, 1, 0, st>>>(h, cg_dev); },
          [&](cudaStream_t st, cudaGraphConditionalHandle h) {
            c.pre->vcycle(c.r.p, zp, st, false);
            Ops<double>::dot(len, c.r.p, zp, red, FIN_CG_RZ, cg_dev, st);
            Ops<double>::cg_dir(len, c.p.p, zp, cg_dev, 0, st);
            Ops<double>::apply_dot(L64, 1, c.p.p, c.q.p, red, FIN_CG_PAP, cg_dev, st);
            Ops<double>::cg_update(len, x.p, c.p.p, c.r.p, c.q.p, cg_dev, red, cg_dev, st);
            k_cg_cond<<<1, 1, 0, st>>>(h, cg_dev, maxit + 4, 1);
          },
          [&](cudaStream_t) {});
    }
  }
  { ProfScope ps_(GKB_KC_GKB, s); k_note_inner<<<1, 1, 0, s>>>(gkb_dev, cg_dev); }
  if (P) P->phase = saved;
}

// f = gamma A N^-1 r (the first term of Eq. (3)'s right-hand side) from the
// staged r in ctmp; the diagonal-N form scales r into gq first
void Solver::al_rhs(cudaStream_t s) {
  const Lvl& L = L64;
  if (diag_n) {
    { ProfScope ps_(GKB_KC_GKB, s); k_cells_mul<<<cgrid(L), dim3(32, 8), 0, s>>>(L, ctmp.p, nw64.p, gq.p); }
    Ops<double>::grad(L, gq.p, f.p, gamma / n_scale, s);
  } else {
    Ops<double>::grad(L, ctmp.p, f.p, gamma / n_scale, s);
  }
}

// AL transform, GKB initialisation and the while loop of Algorithm 1,
// captured into the graph that s is capturing. Inputs: wtmp (g), ctmp (r);
// outputs: u (velocity without y0), pp (pressure), y0.
void Solver::capture_core(cudaStream_t s, cudaStream_t sb1, cudaStream_t sb2) {
  const Lvl& L = L64;
  const long long len = L.nvel;
  GkbState* S = gkb_dev;
  double* red_out = (double*)((char*)gkb_dev + offsetof(GkbState, red));
  // AL transform (Eq. (3)): f = g + gamma A N^-1 r ; y0 = M^-1 f ; b = r - A^T y0
  al_rhs(s);
  Ops<double>::axpby(len, 1.0, wtmp.p, 1.0, f.p, s);
  capture_inner(s, sb1);
  GKB_CUDA(cudaMemcpyAsync(y0.p, x.p, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // init: beta_1, q_1, w = M^-1 A q_1, alpha_1, v_1, zeta_1, d_1, p, u
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_b<<<cgrid(L), dim3(32, 8), 0, s>>>(L, ctmp.p, y0.p, bc.p, S, red, red_out); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_scalar<<<1, 32, 0, s>>>(S_BETA1, S, red_out); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_q1<<<cgrid(L), dim3(32, 8), 0, s>>>(L, bc.p, q.p, S); }
  Ops<double>::grad(L, q.p, f.p, 1.0, s);
  GKB_CUDA(cudaMemsetAsync(u.p, 0, len * sizeof(double), s));
  GKB_CUDA(cudaMemsetAsync(pp.p, 0, L.ncell * sizeof(double), s));
  capture_inner(s, sb1);
  Ops<double>::apply_dot(L, 1, x.p, t.p, red, FIN_STORE, red_out, s);
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_scalar<<<1, 32, 0, s>>>(S_ALPHA1, S, red_out); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gk4v<<<lin_blocks(len), CB, 0, s>>>(len, x.p, v.p, u.p, S, 1); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gk4c<<<cgrid(L), dim3(32, 8), 0, s>>>(L, gq.p, q.p, d.p, pp.p, S, 1); }
  // the while loop of Algorithm 1 as a device-side loop
  const int hard_max = opt.maxit + 2;
  capture_loop(
      s, sb1, 1,
      [&](cudaStream_t st, cudaGraphConditionalHandle h) {
        { ProfScope ps_(GKB_KC_GKB, st); k_gkb_cond_init<<<1, 1, 0, st>>>(h, S); }
      },
      [&](cudaStream_t st, cudaGraphConditionalHandle h) {
        { ProfScope ps_(GKB_KC_GKB, st); k_gk1<<<cgrid(L), dim3(32, 8), 0, st>>>(L, v.p, q.p, gq.p, S, red, red_out); }
        { ProfScope ps_(GKB_KC_GKB, st); k_gkb_scalar<<<1, 32, 0, st>>>(S_BETA, S, red_out); }
        { ProfScope ps_(GKB_KC_GKB, st); k_gk2<<<fgrid(L), dim3(32, 8), 0, st>>>(L, gq.p, f.p, S); }
        capture_inner(st, sb2);
        { ProfScope ps_(GKB_KC_GKB, st); k_gk3<<<lin_blocks(len), CB, 0, st>>>(len, x.p, v.p, w.p, S); }
        Ops<double>::apply_dot(L, 1, w.p, t.p, red, FIN_STORE, red_out, st);
        { ProfScope ps_(GKB_KC_GKB, st); k_gkb_scalar<<<1, 32, 0, st>>>(S_ALPHA, S, red_out); }
        { ProfScope ps_(GKB_KC_GKB, st); k_gk4v<<<lin_blocks(len), CB, 0, st>>>(len, w.p, v.p, u.p, S, 0); }
        { ProfScope ps_(GKB_KC_GKB, st); k_gk4c<<<cgrid(L), dim3(32, 8), 0, st>>>(L, gq.p, q.p, d.p, pp.p, S, 0); }
        { ProfScope ps_(GKB_KC_GKB, st); k_gkb_cond<<<1, 1, 0, st>>>(h, S, hard_max); }
      },
      [&](cudaStream_t) {});
}

void Solver::build_solve_graph() {
  sgraph.destroy();
  if (!opt.use_graph || opt.profile) return;
  ensure_capture_streams();
  Profiler* P = g_prof;
  if (P) {
    for (int ph = 0; ph < 5; ++ph)
      for (int k = 0; k < GKB_KC_COUNT; ++k) { P->cap_l[ph][k] = 0; P->cap_u[ph][k] = 0; }
    P->phase = 0;
  }
  cudaGraph_t g = nullptr;
  try {
    GKB_CUDA(cudaGraphCreate(&g, 0));
    GKB_CUDA(cudaStreamBeginCaptureToGraph(cap1, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capture_core(cap1, cap2, cap3);
    GKB_CUDA(cudaStreamEndCapture(cap1, &g));
    GKB_CUDA(cudaGraphInstantiate(&sgraph.exec, g, 0));
  } catch (...) {
    if (P) P->phase = -1;
    abandon_captures({cap4, cap3, cap2, cap1});
    if (g) cudaGraphDestroy(g);
    sgraph.exec = nullptr;
    throw;
  }
  cudaGraphDestroy(g);
  if (P) {
    P->phase = -1;
    for (int ph = 0; ph < 5; ++ph)
      for (int k = 0; k < GKB_KC_COUNT; ++k) { sgraph.cl[ph][k] = P->cap_l[ph][k]; sgraph.cu[ph][k] = P->cap_u[ph][k]; }
  }
}

// right-hand side into the padded layout: wtmp = g, ctmp = r, with the
// defect correction of an initial guess (g - W w0 - A p0, r - A^T w0)
void Solver::stage_in(const double* g, const double* r, const double* w0, const double* p0) {
  cudaStream_t s = stream;
  const Lvl& L = L64;
  Compact cmp = make_compact(L);
  const long long len = L.nvel;
  auto load_m = [&](const double* src, double* dst) {
    const double* dsrc = src;
    if (!is_device_ptr(src)) {
      GKB_CUDA(cudaMemcpyAsync(stage_m.p, src, m * sizeof(double), cudaMemcpyHostToDevice, s));
      dsrc = stage_m.p;
    }
    GKB_CUDA(cudaMemsetAsync(dst, 0, len * sizeof(double), s));
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_vel<double><<<lin_blocks(m), 256, 0, s>>>(L, cmp, dsrc, dst); }
  };
  auto load_n = [&](const double* src, double* dst) {
    const double* dsrc = src;
    if (!is_device_ptr(src)) {
      GKB_CUDA(cudaMemcpyAsync(stage_n.p, src, ncell * sizeof(double), cudaMemcpyHostToDevice, s));
      dsrc = stage_n.p;
    }
    GKB_CUDA(cudaMemsetAsync(dst, 0, L.ncell * sizeof(double), s));
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_cell<double><<<lin_blocks(ncell), 256, 0, s>>>(L, dsrc, dst); }
  };
  load_m(g, wtmp.p);
  load_n(r, ctmp.p);
  if (w0) {
    load_m(w0, u.p);
    Ops<double>::apply(L, 0, u.p, t.p, s);
    Ops<double>::axpby(len, -1.0, t.p, 1.0, wtmp.p, s);
    if (p0) {
      load_n(p0, pp.p);
      Ops<double>::grad(L, pp.p, t.p, 1.0, s);
      Ops<double>::axpby(len, -1.0, t.p, 1.0, wtmp.p, s);
    }
    Ops<double>::negdiv(L, u.p, q.p, 1.0, s);
    Ops<double>::axpby(L.ncell, -1.0, q.p, 1.0, ctmp.p, s);
  }
}

void Solver::init_state(double tol, int delay) {
  cudaStream_t s = stream;
  GkbState hs{};
  hs.tol = tol;
  hs.n_scale = n_scale;
  hs.ncells = (double)ncell;
  hs.nd = diag_n ? nd64.p : nullptr;
  hs.nsum = diag_n ? nsum : n_scale * (double)ncell;
  hs.ninvsum = diag_n ? ninvsum : (double)ncell / n_scale;
  hs.delay = delay;
  hs.maxit = opt.maxit;
  hs.enclosed = enclosed ? 1 : 0;
  const int cap = opt.maxit + 2;
  hs.h_alpha = hist.p;
  hs.h_beta = hist.p + cap;
  hs.h_zeta = hist.p + 2 * cap;
  hs.h_est = hist.p + 3 * cap;
  hs.hcap = cap;
  hs.h_inner = hist_inner.p;
  hs.icap = opt.maxit + 4;
  GKB_CUDA(cudaMemsetAsync(hist.p, 0, 4 * cap * sizeof(double), s));
  GKB_CUDA(cudaMemsetAsync(hist_inner.p, 0, hs.icap * sizeof(int), s));
  GKB_CUDA(cudaMemcpyAsync(gkb_dev, &hs, sizeof(GkbState), cudaMemcpyHostToDevice, s));
}

// the same sequence as capture_core, sequenced by the host (profiling,
// use_graph = 0): one flag read per outer iteration
void Solver::run_core_host() {
  cudaStream_t s = stream;
  const Lvl& L = L64;
  const long long len = L.nvel;
  GkbState* S = gkb_dev;
  double* red_out = (double*)((char*)gkb_dev + offsetof(GkbState, red));
  al_rhs(s);
  Ops<double>::axpby(len, 1.0, wtmp.p, 1.0, f.p, s);
  inner_solve(f.p, y0.p);
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_b<<<cgrid(L), dim3(32, 8), 0, s>>>(L, ctmp.p, y0.p, bc.p, S, red, red_out); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_scalar<<<1, 32, 0, s>>>(S_BETA1, S, red_out); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_q1<<<cgrid(L), dim3(32, 8), 0, s>>>(L, bc.p, q.p, S); }
  Ops<double>::grad(L, q.p, f.p, 1.0, s);
  GKB_CUDA(cudaMemsetAsync(u.p, 0, len * sizeof(double), s));
  GKB_CUDA(cudaMemsetAsync(pp.p, 0, L.ncell * sizeof(double), s));
  inner_solve(f.p, x.p);
  Ops<double>::apply_dot(L, 1, x.p, t.p, red, FIN_STORE, red_out, s);
  { ProfScope ps_(GKB_KC_GKB, s); k_gkb_scalar<<<1, 32, 0, s>>>(S_ALPHA1, S, red_out); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gk4v<<<lin_blocks(len), CB, 0, s>>>(len, x.p, v.p, u.p, S, 1); }
  { ProfScope ps_(GKB_KC_GKB, s); k_gk4c<<<cgrid(L), dim3(32, 8), 0, s>>>(L, gq.p, q.p, d.p, pp.p, S, 1); }
  GKB_CUDA(cudaMemcpyAsync(gkb_host, S, sizeof(GkbState), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  while (!gkb_host->stop && gkb_host->status == ST_OK) {
    { ProfScope ps_(GKB_KC_GKB, s); k_gk1<<<cgrid(L), dim3(32, 8), 0, s>>>(L, v.p, q.p, gq.p, S, red, red_out); }
    { ProfScope ps_(GKB_KC_GKB, s); k_gkb_scalar<<<1, 32, 0, s>>>(S_BETA, S, red_out); }
    { ProfScope ps_(GKB_KC_GKB, s); k_gk2<<<fgrid(L), dim3(32, 8), 0, s>>>(L, gq.p, f.p, S); }
    inner_solve(f.p, x.p);
    { ProfScope ps_(GKB_KC_GKB, s); k_gk3<<<lin_blocks(len), CB, 0, s>>>(len, x.p, v.p, w.p, S); }
    Ops<double>::apply_dot(L, 1, w.p, t.p, red, FIN_STORE, red_out, s);
    { ProfScope ps_(GKB_KC_GKB, s); k_gkb_scalar<<<1, 32, 0, s>>>(S_ALPHA, S, red_out); }
    { ProfScope ps_(GKB_KC_GKB, s); k_gk4v<<<lin_blocks(len), CB, 0, s>>>(len, w.p, v.p, u.p, S, 0); }
    { ProfScope ps_(GKB_KC_GKB, s); k_gk4c<<<cgrid(L), dim3(32, 8), 0, s>>>(L, gq.p, q.p, d.p, pp.p, S, 0); }
    GKB_CUDA(cudaMemcpyAsync(gkb_host, S, sizeof(GkbState), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
  }
}

// back-transform w = u + y0 (+ w0), p (+ p0), mean-free pressure for
// enclosed flow, outputs in compact order; statistics
int Solver::finish(double* w_out, double* p_out, const double* w0, const double* p0, bool graph_run) {
  cudaStream_t s = stream;
  const Lvl& L = L64;
  Compact cmp = make_compact(L);
  const long long len = L.nvel;
  Ops<double>::axpby(len, 1.0, y0.p, 1.0, u.p, s);
  if (w0) {
    const double* src = w0;
    if (!is_device_ptr(w0)) {
      GKB_CUDA(cudaMemcpyAsync(stage_m.p, w0, m * sizeof(double), cudaMemcpyHostToDevice, s));
      src = stage_m.p;
    }
    GKB_CUDA(cudaMemsetAsync(t.p, 0, len * sizeof(double), s));
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_vel<double><<<lin_blocks(m), 256, 0, s>>>(L, cmp, src, t.p); }
    Ops<double>::axpby(len, 1.0, t.p, 1.0, u.p, s);
    if (p0) {
      const double* srcp = p0;
      if (!is_device_ptr(p0)) {
        GKB_CUDA(cudaMemcpyAsync(stage_n.p, p0, ncell * sizeof(double), cudaMemcpyHostToDevice, s));
        srcp = stage_n.p;
      }
      GKB_CUDA(cudaMemsetAsync(ctmp.p, 0, L.ncell * sizeof(double), s));
      { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_cell<double><<<lin_blocks(ncell), 256, 0, s>>>(L, srcp, ctmp.p); }
      Ops<double>::axpby(L.ncell, 1.0, ctmp.p, 1.0, pp.p, s);
    }
  }
  if (enclosed) { ProfScope ps_(GKB_KC_GKB, s); k_cell_sum<<<cgrid(L), dim3(32, 8), 0, s>>>(L, pp.p, red, scal.p); }
  const bool wdev = is_device_ptr(w_out), pdev = is_device_ptr(p_out);
  { ProfScope ps_(GKB_KC_LAYOUT, s); k_unpack_vel<<<lin_blocks(m), 256, 0, s>>>(L, cmp, u.p, wdev ? w_out : stage_m.p); }
  { ProfScope ps_(GKB_KC_LAYOUT, s); k_unpack_cell_dev<<<lin_blocks(ncell), 256, 0, s>>>(L, pp.p, pdev ? p_out : stage_n.p, enclosed ? scal.p : nullptr, 1.0 / (double)ncell); }
  if (!wdev) GKB_CUDA(cudaMemcpyAsync(w_out, stage_m.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!pdev) GKB_CUDA(cudaMemcpyAsync(p_out, stage_n.p, ncell * sizeof(double), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaMemcpyAsync(gkb_host, gkb_dev, sizeof(GkbState), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  GKB_CUDA(cudaGetLastError());
  const GkbState& H = *gkb_host;
  int status = H.status;
  if (status == ST_OK && !H.converged) status = ST_NOT_CONVERGED;
  if (status == ST_OK && H.inner_status != ST_OK) status = H.inner_status;
  if (graph_run) {
    // launches of the graph: captured counts times the executions of each part
    for (int k = 0; k < GKB_KC_COUNT; ++k) {
      prof.launches[k] += sgraph.cl[0][k] + H.outer_runs * sgraph.cl[1][k] + H.inner_solves * sgraph.cl[2][k] +
                          H.inner_runs * sgraph.cl[3][k] + H.inner_fb_runs * sgraph.cl[4][k];
      prof.units[k] += sgraph.cu[0][k] + H.outer_runs * sgraph.cu[1][k] + H.inner_solves * sgraph.cu[2][k] +
                       H.inner_runs * sgraph.cu[3][k] + H.inner_fb_runs * sgraph.cu[4][k];
    }
  }
  // the single-kernel CG solves: one operator product per iteration
  if (small_cg()) prof.units[GKB_KC_APPLY] += H.inner_its * L64.nvel;
  prof.collect();
  for (int kc = 0; kc < GKB_KC_COUNT; ++kc) {
    stats.kernel_launches[kc] = prof.launches[kc];
    stats.kernel_units[kc] = prof.units[kc];
    stats.kernel_ms[kc] = prof.ms[kc];
    stats.kernel_top_launches[kc] = prof.top_launches[kc];
    stats.kernel_top_units[kc] = prof.top_units[kc];
    stats.kernel_top_ms[kc] = prof.top_ms[kc];
  }
  stats.status = status;
  stats.outer_iterations = H.k;
  stats.estimate = H.est;
  stats.inner_iterations = H.inner_its;
  stats.inner_fallbacks = H.inner_fallbacks;
  stats.tuned_inner_ms = tuned_ms;
  stats.inner_solves = H.inner_solves;
  return status;
}

int Solver::solve(const double* g, const double* r, double tol, int delay, double* w_out, double* p_out,
                  const double* w0, const double* p0) {
  if (!have_problem) throw Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
  if (!g || !r || !w_out || !p_out) throw Error{GKB_ERR_INVALID_ARG, "g, r, w_out and p_out must not be NULL"};
  if (!(tol >= 0)) throw Error{GKB_ERR_INVALID_ARG, "tol must be >= 0"};
  if (delay < 0 || delay > GKB_RING - 2) throw Error{GKB_ERR_INVALID_ARG, "delay out of range"};
  auto t0 = std::chrono::steady_clock::now();
  prof.reset();
  if (opt.profile) prof.enable(32768);
  stage_in(g, r, w0, p0);
  init_state(tol, delay);
  refresh_net();
  const bool graph_run = sgraph.exec != nullptr && !opt.profile;
  if (graph_run) GKB_CUDA(cudaGraphLaunch(sgraph.exec, stream));
  else run_core_host();
  const int status = finish(w_out, p_out, w0, p0, graph_run);
  stats.solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

void Solver::apply(int op, const double* xin, double* yout) {
  if (!have_problem) throw Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
  if (!xin || !yout) throw Error{GKB_ERR_INVALID_ARG, "NULL vector"};
  cudaStream_t s = stream;
  const Lvl& L = L64;
  Compact cmp = make_compact(L);
  const long long len = L.nvel;
  const bool in_cells = (op == GKB_OP_A);
  const bool out_cells = (op == GKB_OP_AT);
  const long long nin = in_cells ? ncell : m, nout = out_cells ? ncell : m;
  const double* src = xin;
  if (!is_device_ptr(xin)) {
    double* st_in = in_cells ? stage_n.p : stage_m.p;
    GKB_CUDA(cudaMemcpyAsync(st_in, xin, nin * sizeof(double), cudaMemcpyHostToDevice, s));
    src = st_in;
  }
  if (in_cells) {
    GKB_CUDA(cudaMemsetAsync(ctmp.p, 0, L.ncell * sizeof(double), s));
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_cell<double><<<lin_blocks(ncell), 256, 0, s>>>(L, src, ctmp.p); }
  } else {
    GKB_CUDA(cudaMemsetAsync(wtmp.p, 0, len * sizeof(double), s));
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_vel<double><<<lin_blocks(m), 256, 0, s>>>(L, cmp, src, wtmp.p); }
  }
  switch (op) {
    case GKB_OP_W: Ops<double>::apply(L, 0, wtmp.p, t.p, s); break;
    case GKB_OP_M: Ops<double>::apply(L, 1, wtmp.p, t.p, s); break;
    case GKB_OP_A: Ops<double>::grad(L, ctmp.p, t.p, 1.0, s); break;
    case GKB_OP_AT: Ops<double>::negdiv(L, wtmp.p, q.p, 1.0, s); break;
    default: throw Error{GKB_ERR_INVALID_ARG, "unknown operator"};
  }
  const bool ydev = is_device_ptr(yout);
  double* dst = ydev ? yout : (out_cells ? stage_n.p : stage_m.p);
  if (out_cells) { ProfScope ps_(GKB_KC_LAYOUT, s); k_unpack_cell<<<lin_blocks(ncell), 256, 0, s>>>(L, q.p, dst, 0.0); }
  else { ProfScope ps_(GKB_KC_LAYOUT, s); k_unpack_vel<<<lin_blocks(m), 256, 0, s>>>(L, cmp, t.p, dst); }
  if (!ydev) GKB_CUDA(cudaMemcpyAsync(yout, dst, nout * sizeof(double), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  GKB_CUDA(cudaGetLastError());
}

// Dirichlet normal velocity on one side folded into compact (g, r)
__global__ void k_boundary_rhs(Lvl L, Compact cmp, int side, const double* __restrict__ ub,
                               double* __restrict__ g, double* __restrict__ r) {
  const int c = side / 2, hi = side % 2;
  int oth[2], no = 0;
  for (int a = 0; a < L.dim; ++a)
    if (a != c) oth[no++] = a;
  const int n0 = L.n[oth[0]], n1 = (no > 1) ? L.n[oth[1]] : 1;
  const long long nb = (long long)n0 * n1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nb; t += (long long)gridDim.x * blockDim.x) {
    int p[3] = {0, 0, 0};
    p[oth[0]] = (int)(t % n0);
    if (no > 1) p[oth[1]] = (int)(t / n0);
    const double u = ub[t];
    // adjacent active face and the cell between them
    int f[3] = {p[0], p[1], p[2]};
    int cell[3] = {p[0], p[1], p[2]};
    f[c] = hi ? L.n[c] - 1 : 1;
    cell[c] = hi ? L.n[c] - 1 : 0;
    const double mu = L.mu64 ? L.mu64[cix(L, cell[0], cell[1], cell[2])] : L.mu0;
    const long long fi = cmp.base[c] + ((long long)(f[2] - cmp.lo[c][2]) * cmp.ext[c][1] + (f[1] - cmp.lo[c][1])) * cmp.ext[c][0] +
                         (f[0] - cmp.lo[c][0]);
    g[fi] += L.wscale * mu * u;
    const long long ci = ((long long)cell[2] * L.n[1] + cell[1]) * L.n[0] + cell[0];
    r[ci] += (hi ? 1.0 : -1.0) * L.ascale * u;
  }
}

void Solver::boundary_rhs(int side, const double* ub, double* g, double* r) {
  if (!have_problem) throw Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
  if (L64.sym) throw Error{GKB_ERR_INVALID_ARG, "boundary data is not supported with the symmetric-gradient form"};
  if (side < 0 || side >= 2 * grid.dim) throw Error{GKB_ERR_INVALID_ARG, "side out of range"};
  if (grid.bc[side] != GKB_BC_DIRICHLET) throw Error{GKB_ERR_INVALID_ARG, "side is not Dirichlet"};
  if (!ub || !g || !r) throw Error{GKB_ERR_INVALID_ARG, "NULL vector"};
  cudaStream_t s = stream;
  const Lvl& L = L64;
  Compact cmp = make_compact(L);
  const int c = side / 2;
  long long nb = 1;
  for (int a = 0; a < grid.dim; ++a)
    if (a != c) nb *= grid.n[a];
  DevBuf<double> ubd;
  const double* ud = ub;
  if (!is_device_ptr(ub)) {
    ubd.alloc(nb);
    GKB_CUDA(cudaMemcpyAsync(ubd.p, ub, nb * sizeof(double), cudaMemcpyHostToDevice, s));
    ud = ubd.p;
  }
  const bool gdev = is_device_ptr(g), rdev = is_device_ptr(r);
  double* gd = gdev ? g : stage_m.p;
  double* rd = rdev ? r : stage_n.p;
  if (!gdev) GKB_CUDA(cudaMemcpyAsync(gd, g, m * sizeof(double), cudaMemcpyHostToDevice, s));
  if (!rdev) GKB_CUDA(cudaMemcpyAsync(rd, r, ncell * sizeof(double), cudaMemcpyHostToDevice, s));
  { ProfScope ps_(GKB_KC_LAYOUT, s); k_boundary_rhs<<<lin_blocks(nb), 256, 0, s>>>(L, cmp, side, ud, gd, rd); }
  if (!gdev) GKB_CUDA(cudaMemcpyAsync(g, gd, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!rdev) GKB_CUDA(cudaMemcpyAsync(r, rd, ncell * sizeof(double), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  GKB_CUDA(cudaGetLastError());
}

void Solver::precond(const double* rin, double* zout) {
  if (!have_problem) throw Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
  if (!rin || !zout) throw Error{GKB_ERR_INVALID_ARG, "NULL vector"};
  cudaStream_t s = stream;
  const Lvl& L = L64;
  Compact cmp = make_compact(L);
  const long long len = L.nvel;
  const double* src = rin;
  if (!is_device_ptr(rin)) {
    GKB_CUDA(cudaMemcpyAsync(stage_m.p, rin, m * sizeof(double), cudaMemcpyHostToDevice, s));
    src = stage_m.p;
  }
  GKB_CUDA(cudaMemsetAsync(wtmp.p, 0, len * sizeof(double), s));
  { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_vel<double><<<lin_blocks(m), 256, 0, s>>>(L, cmp, src, wtmp.p); }
  const bool use_gmg = opt.inner == GKB_INNER_GMG_PCG || opt.inner == GKB_INNER_FGMRES || learned_inner();
  refresh_net();
  if (opt.precision == GKB_PREC_MIXED) {
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_vel<float><<<lin_blocks(m), 256, 0, s>>>(L, cmp, src, f32.p); }
    if (use_gmg) gmg32.vcycle(f32.p, x32.p, s);
    else GKB_CUDA(cudaMemcpyAsync(x32.p, f32.p, len * sizeof(float), cudaMemcpyDeviceToDevice, s));
    GKB_CUDA(cudaMemsetAsync(scal.p + 8, 0, sizeof(double), s));
    double one = 1.0;
    GKB_CUDA(cudaMemcpyAsync(scal.p + 8, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    GKB_CUDA(cudaMemsetAsync(t.p, 0, len * sizeof(double), s));
    { ProfScope ps_(GKB_KC_LAYOUT, s); k_add_f32<<<lin_blocks(len), CB, 0, s>>>(len, x32.p, t.p, scal.p + 8); }
  } else {
    if (use_gmg) gmg64.vcycle(wtmp.p, t.p, s);
    else GKB_CUDA(cudaMemcpyAsync(t.p, wtmp.p, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  const bool zdev = is_device_ptr(zout);
  double* dst = zdev ? zout : stage_m.p;
  { ProfScope ps_(GKB_KC_LAYOUT, s); k_unpack_vel<<<lin_blocks(m), 256, 0, s>>>(L, cmp, t.p, dst); }
  if (!zdev) GKB_CUDA(cudaMemcpyAsync(zout, dst, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  GKB_CUDA(cudaGetLastError());
}


// Training pairs for the learned correction: FP64 GMG-PCG on M x = f from a
// zero start; after every iteration k that has not yet converged, the
// residual r_k and the iterate x_k are kept; once the solve has converged to
// x*, pair k is the image of r_k / ||r_k|| and of the error x* - x_k / ||r_k||
// (both times sqrt(nx ny)), so that M e^ = r^ up to the solve's tolerance.
int Solver::harvest(const double* fin, int max_pairs, float* x_img, float* t_img, int* n_pairs) {
  if (!have_problem) throw Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
  if (!fin || !x_img || !t_img || !n_pairs || max_pairs < 1) throw Error{GKB_ERR_INVALID_ARG, "bad harvest arguments"};
  if (grid.dim != 2 || grid.n[0] % 4 || grid.n[1] % 4)
    throw Error{GKB_ERR_INVALID_ARG, "pairs are harvested on 2D grids with sides divisible by 4"};
  if (opt.precision != GKB_PREC_FP64 || opt.inner != GKB_INNER_GMG_PCG)
    throw Error{GKB_ERR_INVALID_ARG, "pairs are harvested by the FP64 GMG-PCG inner solver"};
  if (!is_device_ptr(x_img) || !is_device_ptr(t_img)) throw Error{GKB_ERR_INVALID_ARG, "images must be device arrays"};
  cudaStream_t s = stream;
  const Lvl& L = L64;
  const long long len = L.nvel;
  const long long px = (long long)L.n[0] * L.n[1];
  Compact cmp = make_compact(L);
  const double* src = fin;
  if (!is_device_ptr(fin)) {
    GKB_CUDA(cudaMemcpyAsync(stage_m.p, fin, m * sizeof(double), cudaMemcpyHostToDevice, s));
    src = stage_m.p;
  }
  GKB_CUDA(cudaMemsetAsync(wtmp.p, 0, len * sizeof(double), s));
  { ProfScope ps_(GKB_KC_LAYOUT, s); k_pack_vel<double><<<lin_blocks(m), 256, 0, s>>>(L, cmp, src, wtmp.p); }
  DevBuf<double> xk, nrm;
  xk.alloc((size_t)max_pairs * len);
  nrm.alloc((size_t)max_pairs * 4);
  Cg<double>& c = cg64;
  CgState h{};
  h.tol2 = opt.tol_inner * opt.tol_inner;
  h.maxit = opt.maxit_inner;
  GKB_CUDA(cudaMemcpyAsync(cg_dev, &h, sizeof(CgState), cudaMemcpyHostToDevice, s));
  GKB_CUDA(cudaMemsetAsync(x.p, 0, len * sizeof(double), s));
  GKB_CUDA(cudaMemcpyAsync(c.r.p, wtmp.p, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
  Ops<double>::dot(len, wtmp.p, wtmp.p, red, FIN_CG_INIT, cg_dev, s);
  int np = 0;
  auto keep = [&]() {
    if (np >= max_pairs) return;
    Ops<double>::dot(len, c.r.p, c.r.p, red, FIN_STORE, nrm.p + 4 * np, s);
    mac_to_img<double>(L, c.r.p, nrm.p + 4 * np, x_img + (size_t)np * px * 3, s);
    GKB_CUDA(cudaMemcpyAsync(xk.p + (size_t)np * len, x.p, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
    ++np;
  };
  GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  if (!cg_host->done) keep();
  c.pre->vcycle(c.r.p, c.z.p, s);
  Ops<double>::dot(len, c.r.p, c.z.p, red, FIN_CG_RZ0, cg_dev, s);
  Ops<double>::cg_dir(len, c.p.p, c.z.p, cg_dev, 1, s);
  GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  while (!cg_host->done) {
    Ops<double>::apply_dot(L, 1, c.p.p, c.q.p, red, FIN_CG_PAP, cg_dev, s);
    Ops<double>::cg_update(len, x.p, c.p.p, c.r.p, c.q.p, cg_dev, red, cg_dev, s);
    GKB_CUDA(cudaMemcpyAsync(cg_host, cg_dev, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
    if (cg_host->done) break;
    keep();
    c.pre->vcycle(c.r.p, c.z.p, s);
    Ops<double>::dot(len, c.r.p, c.z.p, red, FIN_CG_RZ, cg_dev, s);
    Ops<double>::cg_dir(len, c.p.p, c.z.p, cg_dev, 0, s);
  }
  const int status = cg_host->status;
  if (status != ST_OK) np = 0;
  // x* - x_k is known only to about ||r*|| / ||r_k|| relative: keep the
  // leading pairs whose residual is at least 1e4 times the final one
  std::vector<double> hn(4 * (size_t)std::max(np, 1));
  if (np > 0) GKB_CUDA(cudaMemcpy(hn.data(), nrm.p, 4 * np * sizeof(double), cudaMemcpyDeviceToHost));
  int keep_n = 0;
  while (keep_n < np && hn[4 * keep_n] >= 1e8 * cg_host->rr) ++keep_n;
  if (keep_n < np)
    GKB_CUDA(cudaMemsetAsync(x_img + (size_t)keep_n * px * 3, 0, (size_t)(np - keep_n) * px * 3 * sizeof(float), s));
  np = keep_n;
  for (int k = 0; k < np; ++k)
    err_to_img(L, x.p, xk.p + (size_t)k * len, nrm.p + 4 * k, t_img + (size_t)k * px * 2, s);
  GKB_CUDA(cudaStreamSynchronize(s));
  *n_pairs = np;
  return status;
}

// ---------------------------------------------------------------------------
// batched solves: one graph, one branch per problem
// ---------------------------------------------------------------------------

namespace {

// one graph per batch: either every problem's whole solve as a branch, or
// the lock-step form (lockstep.cu) where each step is one launch over all
// problems
struct BatchGraph {
  std::vector<const Solver*> members;
  std::vector<int> gens;
  cudaGraphExec_t exec = nullptr;
  Lockstep* lock = nullptr;
  ~BatchGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    delete lock;
  }
};

// the first handle's batch_lockstep option asks for the lock-step form; a
// batch that does not qualify keeps one graph branch per problem
bool lockstep_wanted(Solver** S, int count) {
  return S[0]->opt.batch_lockstep == 1 && lockstep_eligible(S, count);
}

std::mutex g_batch_mutex;
std::vector<BatchGraph*> g_batches;

}  // namespace

void forget_batches(const Solver* sv) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (size_t i = 0; i < g_batches.size();) {
    BatchGraph* b = g_batches[i];
    bool hit = false;
    for (const Solver* m : b->members) hit = hit || (m == sv);
    if (hit) {
      delete b;
      g_batches.erase(g_batches.begin() + i);
    } else {
      ++i;
    }
  }
}

static BatchGraph* build_batch(Solver** S, int count, cudaStream_t origin) {
  BatchGraph* B = new BatchGraph();
  for (int i = 0; i < count; ++i) {
    B->members.push_back(S[i]);
    B->gens.push_back(S[i]->generation);
  }
  if (lockstep_wanted(S, count)) {
    Profiler* saved = g_prof;
    g_prof = nullptr;
    try {
      S[0]->ensure_capture_streams();
      B->lock = new Lockstep(S, count, origin, S[0]->cap2, S[0]->cap3);
    } catch (...) {
      g_prof = saved;
      delete B;
      throw;
    }
    g_prof = saved;
    return B;
  }
  std::vector<cudaStream_t> br(count, nullptr);
  std::vector<cudaEvent_t> ev(count + 1, nullptr);
  cudaGraph_t g = nullptr;
  Profiler* saved = g_prof;
  g_prof = nullptr;  // launches are accounted from each handle's own graph counts
  try {
    for (int i = 0; i < count; ++i) GKB_CUDA(cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking));
    for (int i = 0; i <= count; ++i) GKB_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
    GKB_CUDA(cudaGraphCreate(&g, 0));
    GKB_CUDA(cudaStreamBeginCaptureToGraph(origin, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    GKB_CUDA(cudaEventRecord(ev[count], origin));
    for (int i = 0; i < count; ++i) {
      GKB_CUDA(cudaStreamWaitEvent(br[i], ev[count], 0));
      S[i]->ensure_capture_streams();
      S[i]->capture_core(br[i], S[i]->cap2, S[i]->cap3);
      GKB_CUDA(cudaEventRecord(ev[i], br[i]));
      GKB_CUDA(cudaStreamWaitEvent(origin, ev[i], 0));
    }
    GKB_CUDA(cudaStreamEndCapture(origin, &g));
    GKB_CUDA(cudaGraphInstantiate(&B->exec, g, 0));
  } catch (...) {
    g_prof = saved;
    std::vector<cudaStream_t> all(br.begin(), br.end());
    all.push_back(origin);
    for (int i = 0; i < count; ++i) { all.push_back(S[i]->cap2); all.push_back(S[i]->cap3); }
    for (cudaStream_t st : all) abandon_captures({st});
    if (g) cudaGraphDestroy(g);
    for (cudaStream_t st : br) if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
    delete B;
    throw;
  }
  g_prof = saved;
  cudaGraphDestroy(g);
  for (cudaStream_t st : br) cudaStreamDestroy(st);
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  return B;
}

int solve_batched(Solver** S, int count, const double* const* g, const double* const* r, double tol, int delay,
                  double* const* w, double* const* p) {
  if (count < 1 || !S || !g || !r || !w || !p) throw Error{GKB_ERR_INVALID_ARG, "bad batched arguments"};
  if (!(tol >= 0)) throw Error{GKB_ERR_INVALID_ARG, "tol must be >= 0"};
  if (delay < 0 || delay > GKB_RING - 2) throw Error{GKB_ERR_INVALID_ARG, "delay out of range"};
  for (int i = 0; i < count; ++i) {
    if (!S[i] || !S[i]->have_problem) throw Error{GKB_ERR_INVALID_ARG, "every handle needs gkb_set_problem"};
    if (!S[i]->sgraph.exec) throw Error{GKB_ERR_INVALID_ARG, "batched solves need use_graph = 1 and profile = 0"};
    if (!g[i] || !r[i] || !w[i] || !p[i]) throw Error{GKB_ERR_INVALID_ARG, "NULL vector in the batch"};
    for (int j = 0; j < i; ++j)
      if (S[j] == S[i]) throw Error{GKB_ERR_INVALID_ARG, "a handle appears twice in the batch"};
  }
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = S[0]->stream;
  BatchGraph* B = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    for (BatchGraph* b : g_batches) {
      if ((int)b->members.size() != count) continue;
      bool same = true;
      for (int i = 0; i < count && same; ++i) same = b->members[i] == S[i] && b->gens[i] == S[i]->generation;
      if (same) { B = b; break; }
    }
  }
  if (!B) {
    Solver* s0 = S[0];
    s0->ensure_capture_streams();
    B = build_batch(S, count, s0->cap1);
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    g_batches.push_back(B);
  }
  // every problem stages its inputs and state on the batch stream
  std::vector<cudaStream_t> own(count);
  for (int i = 0; i < count; ++i) {
    own[i] = S[i]->stream;
    S[i]->stream = st;
  }
  int status = GKB_OK;
  try {
    for (int i = 0; i < count; ++i) {
      S[i]->prof.reset();
      S[i]->stage_in(g[i], r[i], nullptr, nullptr);
      S[i]->init_state(tol, delay);
      S[i]->refresh_net();
    }
    if (B->lock) B->lock->launch(st);
    else GKB_CUDA(cudaGraphLaunch(B->exec, st));
    for (int i = 0; i < count; ++i) {
      const int si = S[i]->finish(w[i], p[i], nullptr, nullptr, B->lock == nullptr);
      if (status == GKB_OK && si != GKB_OK) status = si;
    }
    if (B->lock) {
      // the batch's launches (each covers every problem) go to the first handle
      long long lc[GKB_KC_COUNT];
      B->lock->launch_counts(st, lc);
      for (int k = 0; k < GKB_KC_COUNT; ++k) S[0]->stats.kernel_launches[k] += lc[k];
    }
  } catch (...) {
    for (int i = 0; i < count; ++i) S[i]->stream = own[i];
    throw;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < count; ++i) {
    S[i]->stream = own[i];
    S[i]->stats.solve_seconds = secs;
  }
  return status;
}

}  // namespace gkb
