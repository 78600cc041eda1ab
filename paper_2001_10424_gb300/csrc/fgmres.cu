// fgmres.cu - restarted flexible GMRES (FGMRES(m)) in two roles: the inner
// solve M x = f with one V-cycle as the right preconditioner (the paper's
// alternative inner Krylov method to CG, Sec. 3, Sec. 4.1.3), and the outer
// solve of the saddle system [W A; A^T 0] with the GKB solver itself, run to
// a loose tolerance, as the preconditioner (Sec. 3: GKB used as a
// preconditioner rather than a solver). The inner solve runs device-resident
// inside the whole-solve graph (capture_fgmres: the Hessenberg column, the
// Givens rotations, the back substitution and the restart test are
// single-thread kernels on device state, the Arnoldi and restart loops
// conditional graph nodes); fgmres_solve is its host-sequenced form
// (profiling, use_graph = 0), and the outer saddle solve stays host-sequenced.
//
// One cycle builds an orthonormal basis V of the Krylov space of M B (B: one
// V-cycle, which may vary from step to step, hence the flexible form keeps
// the preconditioned vectors Z = B V), orthogonalises each new vector twice
// by classical Gram-Schmidt (two fused multi-dot and multi-axpy passes),
// reduces the Hessenberg matrix by Givens rotations on the host as it grows,
// and stops when the least-squares residual |g_{j+1}| meets the inner rule
// ||f - M x|| <= tol_inner ||f||; x += Z y, then the true residual decides
// whether to restart.
#include <math.h>

#include <algorithm>
#include <vector>

#include "solver.cuh"

namespace gkb {

namespace {

constexpr int FB = 256;            // threads per block
constexpr int FBLK = 304;          // blocks of the multi-dot (2 x 152 SMs)

// part[k * gridDim.x + b] = block b's share of V_k . w (k = blockIdx.y)
__global__ void __launch_bounds__(FB) k_mdot(const double* __restrict__ V, long long len, const double* __restrict__ w,
                                            double* __restrict__ part) {
  __shared__ double sh[FB / 32];
  const int k = blockIdx.y;
  const double* v = V + (long long)k * len;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)FB + threadIdx.x; t < len; t += (long long)gridDim.x * FB)
    acc += v[t] * w[t];
  acc = warp_sum(acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    double s = lane < FB / 32 ? sh[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) part[(long long)k * gridDim.x + blockIdx.x] = s;
  }
}

// out[k] (+)= sum over the blocks of part[k][.] in block order (deterministic)
__global__ void k_mcols(const double* __restrict__ part, int nblk, int nv, double* __restrict__ out, int add) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)k * nblk + b];
  out[k] = add ? out[k] + s : s;
}

// w += sign * sum_k c[k] V_k
__global__ void __launch_bounds__(FB) k_maxpy(double* __restrict__ w, const double* __restrict__ V, long long len,
                                             int nv, const double* __restrict__ c, double sign) {
  for (long long t = blockIdx.x * (long long)FB + threadIdx.x; t < len; t += (long long)gridDim.x * FB) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s += c[k] * V[(long long)k * len + t];
    w[t] += sign * s;
  }
}

__global__ void __launch_bounds__(FB) k_scale_to(double* __restrict__ dst, const double* __restrict__ src, long long len,
                                                double a) {
  for (long long t = blockIdx.x * (long long)FB + threadIdx.x; t < len; t += (long long)gridDim.x * FB) dst[t] = a * src[t];
}

// zp = pp - (sum / ncells) on the in-domain cells (sum = nullptr: copy)
__global__ void k_shift_cells(Lvl L, const double* __restrict__ pp, double* __restrict__ zp, const double* sum,
                              double inv_n) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= L.n[0] || j >= L.n[1]) return;
  const long long c = cix(L, i, j, k);
  zp[c] = pp[c] - (sum ? *sum * inv_n : 0.0);
}

unsigned fblocks(long long len) {
  long long b = (len + FB - 1) / FB;
  return (unsigned)std::max<long long>(1, std::min<long long>(b, 4 * FBLK));
}

}  // namespace

// ---- device-resident inner solve ------------------------------------------

// state of one inner solve; H, cs, sn, g, y follow it in the same buffer
struct FgState {
  double ff, tol2, beta2, hn, inv_hn;
  int m, j, k, it, maxit, status, done, cyc_done, nv, cycles;
};

__device__ __forceinline__ double* fg_H(FgState* F) { return (double*)(F + 1); }
__device__ __forceinline__ double* fg_cs(FgState* F) { return fg_H(F) + (size_t)(F->m + 1) * F->m; }
__device__ __forceinline__ double* fg_sn(FgState* F) { return fg_cs(F) + F->m; }
__device__ __forceinline__ double* fg_g(FgState* F) { return fg_sn(F) + F->m; }

// h[0..nv) of the multi-dot, nv on the device (rows beyond it do nothing)
__global__ void __launch_bounds__(FB) k_mdot_d(const double* __restrict__ V, long long len, const double* __restrict__ w,
                                              double* __restrict__ part, const FgState* F) {
  if ((int)blockIdx.y >= F->nv) return;
  __shared__ double sh[FB / 32];
  const int k = blockIdx.y;
  const double* v = V + (long long)k * len;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)FB + threadIdx.x; t < len; t += (long long)gridDim.x * FB)
    acc += v[t] * w[t];
  acc = warp_sum(acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    double s = lane < FB / 32 ? sh[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) part[(long long)k * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void k_mcols_d(const double* __restrict__ part, int nblk, double* __restrict__ out, int add,
                          const FgState* F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= F->nv) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)k * nblk + b];
  out[k] = add ? out[k] + s : s;
}
// w += sign * sum_{k < n} c[k] V_k with n = F->nv (use_k: F->k)
__global__ void __launch_bounds__(FB) k_maxpy_d(double* __restrict__ w, const double* __restrict__ V, long long len,
                                               const double* __restrict__ c, double sign, const FgState* F, int use_k) {
  const int nv = use_k ? F->k : F->nv;
  for (long long t = blockIdx.x * (long long)FB + threadIdx.x; t < len; t += (long long)gridDim.x * FB) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s += c[k] * V[(long long)k * len + t];
    w[t] += sign * s;
  }
}
// dst = column `col` of the basis (or the reverse), col = F->j (+1)
__global__ void __launch_bounds__(FB) k_fg_col(double* __restrict__ base, double* __restrict__ vec, long long len,
                                              const FgState* F, int to_vec) {
  double* col = base + (long long)F->j * len;
  for (long long t = blockIdx.x * (long long)FB + threadIdx.x; t < len; t += (long long)gridDim.x * FB) {
    if (to_vec) vec[t] = col[t];
    else col[t] = vec[t];
  }
}
// V_0 = r / beta (at a cycle's start), or V_{j+1} = w / hn
__global__ void __launch_bounds__(FB) k_fg_scale(double* __restrict__ V, const double* __restrict__ src, long long len,
                                                const FgState* F, int next) {
  double a;
  double* dst;
  if (next) {
    if (!(F->hn > 0.0) || F->cyc_done == 2) return;
    a = F->inv_hn;
    dst = V + (long long)(F->j + 1) * len;
  } else {
    a = 1.0 / sqrt(F->beta2);
    dst = V;
  }
  for (long long t = blockIdx.x * (long long)FB + threadIdx.x; t < len; t += (long long)gridDim.x * FB)
    dst[t] = a * src[t];
}

enum { FG_BEGIN = 0, FG_CYCLE, FG_GIVENS, FG_NEXT, FG_BACKSUB, FG_RESTART };

__global__ void k_fg_setup(FgState* F, int m, double tol2, int maxit) {
  F->m = m;
  F->tol2 = tol2;
  F->maxit = maxit;
  F->status = ST_OK;
}

// scalar steps of one inner solve (one thread); `red` holds the last
// FIN_STORE sums (f.f, w.w or r.r), h the Hessenberg column from the
// multi-dots, y the back substitution's output
__global__ void k_fg_scalar(int op, FgState* F, const double* red, const double* h, double* y, CgState* cg,
                            cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = F->m;
  double* H = fg_H(F);
  double* cs = fg_cs(F);
  double* sn = fg_sn(F);
  double* g = fg_g(F);
  unsigned go = 0;
  switch (op) {
    case FG_BEGIN:  // x = 0, r = f: the restart test of the first cycle
      F->ff = red[0];
      F->beta2 = red[0];
      F->it = 0;
      F->status = ST_OK;
      F->done = 0;
      F->cycles = 0;
      // fall through to the restart test
    case FG_RESTART: {
      if (op == FG_RESTART) F->beta2 = red[0];
      if (!isfinite(F->beta2)) { F->status = ST_NAN; F->done = 1; }
      else if (F->beta2 <= F->tol2 * F->ff) F->done = 1;
      else if (F->it >= F->maxit) { F->status = ST_INNER_NOT_CONVERGED; F->done = 1; }
      go = F->done ? 0u : 1u;
      if (!go && cg) {  // the solve's record in the CG state (k_note_inner reads it)
        cg->it = F->it;
        cg->status = F->status;
        cg->graph_iters = F->it;
        cg->fb_iters = F->cycles;
        cg->fallback = 0;
        cg->done = 1;
      }
    } break;
    case FG_CYCLE:  // a cycle starts: g = beta e_1
      F->cycles += 1;
      for (int i = 0; i <= m; ++i) g[i] = 0.0;
      g[0] = sqrt(F->beta2);
      F->j = 0;
      F->k = 0;
      F->nv = 1;
      F->cyc_done = 0;
      go = 1u;
      break;
    case FG_GIVENS: {  // column j of H from h and ||w||, its rotation, the test
      const int j = F->j;
      const double hn = sqrt(red[0]);
      F->it += 1;
      F->hn = hn;
      if (!isfinite(hn)) { F->status = ST_NAN; F->cyc_done = 2; break; }
      F->inv_hn = hn > 0.0 ? 1.0 / hn : 0.0;
      double hc[66];
      for (int i = 0; i <= j; ++i) hc[i] = h[i];
      hc[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * hc[i] + sn[i] * hc[i + 1];
        hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
        hc[i] = a;
      }
      const double rho = hypot(hc[j], hc[j + 1]);
      if (!(rho > 0.0)) { F->status = ST_NOT_SPD; F->cyc_done = 2; break; }
      cs[j] = hc[j] / rho;
      sn[j] = hc[j + 1] / rho;
      hc[j] = rho;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hc[i];
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      F->k = j + 1;
      if (g[j + 1] * g[j + 1] <= F->tol2 * F->ff || F->it >= F->maxit || hn == 0.0 || j + 1 >= m) F->cyc_done = 1;
    } break;
    case FG_NEXT:  // the Arnoldi loop's condition
      if (F->cyc_done == 0) {
        F->j += 1;
        F->nv = F->j + 1;
        go = 1u;
      }
      break;
    case FG_BACKSUB: {  // y = R^-1 g (nothing to add after a failed cycle)
      const int k = (F->status == ST_OK) ? F->k : 0;
      F->k = k;
      for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int c = i + 1; c < k; ++c) t -= H[(size_t)i * m + c] * y[c];
        y[i] = t / H[(size_t)i * m + i];
      }
      if (F->status != ST_OK) F->done = 1;
    } break;
  }
  if (cond) cudaGraphSetConditional(cond, go);
}

void Fgmres::init(long long len_, int m_) {
  len = len_;
  m = m_;
  V.alloc((size_t)(m + 1) * len);
  Z.alloc((size_t)m * len);
  w.alloc(len);
  r.alloc(len);
  h.alloc(m + 2);
  h2.alloc(m + 2);
  y.alloc(m + 1);
  part.alloc((size_t)FBLK * (m + 2));
  // device state: FgState, H ((m+1) x m), cs, sn (m each), g (m+1)
  state.alloc(sizeof(FgState) / sizeof(double) + 1 + (size_t)(m + 1) * m + 3 * (size_t)m + 2);
  vin.alloc(len);
  zt.alloc(len);
}

// h[0..nv) = V_{0..nv}^T w (device)
static void mdot(Fgmres& F, int nv, double* out, int add, cudaStream_t s) {
  ProfScope ps_(GKB_KC_BLAS, s, F.len * nv);
  k_mdot<<<dim3(FBLK, nv), FB, 0, s>>>(F.V.p, F.len, F.w.p, F.part.p);
  k_mcols<<<(nv + 63) / 64, 64, 0, s>>>(F.part.p, FBLK, nv, out, add);
  GKB_CUDA(cudaGetLastError());
}

static double norm2(Solver& S, const double* a, cudaStream_t s) {
  double hs[4];
  Ops<double>::dot(S.L64.nvel, a, a, S.red, FIN_STORE, S.scal.p, s);
  GKB_CUDA(cudaMemcpyAsync(hs, S.scal.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  return hs[0];
}

int fgmres_solve(Solver& S, const double* f, double* x, int* iters) {
  Fgmres& F = S.fgm;
  cudaStream_t s = S.stream;
  const Lvl& L = S.L64;
  const long long len = L.nvel;
  const int m = F.m;
  const double tol2 = S.opt.tol_inner * S.opt.tol_inner;
  const int maxit = S.opt.maxit_inner;
  GKB_CUDA(cudaMemsetAsync(x, 0, len * sizeof(double), s));
  const double ff = norm2(S, f, s);
  int it = 0, status = ST_OK;
  double beta2 = ff;
  const double* r0 = f;  // residual of x = 0
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), hcol(m + 2), yv(m);
  while (status == ST_OK) {
    if (!std::isfinite(beta2)) { status = ST_NAN; break; }
    if (beta2 <= tol2 * ff) break;
    if (it >= maxit) { status = ST_INNER_NOT_CONVERGED; break; }
    const double beta = sqrt(beta2);
    { ProfScope ps_(GKB_KC_BLAS, s, len); k_scale_to<<<fblocks(len), FB, 0, s>>>(F.V.p, r0, len, 1.0 / beta); }
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = F.V.p + (long long)j * len;
      double* zj = F.Z.p + (long long)j * len;
      S.gmg64.vcycle(vj, zj, s);
      Ops<double>::apply(L, 1, zj, F.w.p, s);
      // two passes of classical Gram-Schmidt against V_0..V_j
      mdot(F, j + 1, F.h.p, 0, s);
      { ProfScope ps_(GKB_KC_BLAS, s, len * (j + 1)); k_maxpy<<<fblocks(len), FB, 0, s>>>(F.w.p, F.V.p, len, j + 1, F.h.p, -1.0); }
      mdot(F, j + 1, F.h2.p, 0, s);
      { ProfScope ps_(GKB_KC_BLAS, s, len * (j + 1)); k_maxpy<<<fblocks(len), FB, 0, s>>>(F.w.p, F.V.p, len, j + 1, F.h2.p, -1.0); }
      { ProfScope ps_(GKB_KC_BLAS, s); k_mcols<<<1, 64, 0, s>>>(F.h2.p, 1, j + 1, F.h.p, 1); }  // h += h2
      const double hn2 = norm2(S, F.w.p, s);
      GKB_CUDA(cudaMemcpyAsync(hcol.data(), F.h.p, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
      GKB_CUDA(cudaStreamSynchronize(s));
      const double hn = sqrt(hn2);
      ++it;
      if (!std::isfinite(hn)) { status = ST_NAN; break; }
      if (hn > 0.0) {
        ProfScope ps_(GKB_KC_BLAS, s, len);
        k_scale_to<<<fblocks(len), FB, 0, s>>>(F.V.p + (long long)(j + 1) * len, F.w.p, len, 1.0 / hn);
      }
      // Givens: apply the previous rotations to column j, then zero H(j+1, j)
      hcol[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = a;
      }
      const double rho = hypot(hcol[j], hcol[j + 1]);
      if (!(rho > 0.0)) { status = ST_NOT_SPD; break; }  // no progress possible in this space
      cs[j] = hcol[j] / rho;
      sn[j] = hcol[j + 1] / rho;
      hcol[j] = rho;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      if (g[j + 1] * g[j + 1] <= tol2 * ff || it >= maxit || hn == 0.0) break;
    }
    if (status != ST_OK || k == 0) break;
    // y = R^-1 g (back substitution), x += Z y
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int c = i + 1; c < k; ++c) t -= H[(size_t)i * m + c] * yv[c];
      yv[i] = t / H[(size_t)i * m + i];
    }
    GKB_CUDA(cudaMemcpyAsync(F.y.p, yv.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    { ProfScope ps_(GKB_KC_BLAS, s, len * k); k_maxpy<<<fblocks(len), FB, 0, s>>>(x, F.Z.p, len, k, F.y.p, 1.0); }
    // the true residual decides convergence (and starts the next cycle)
    Ops<double>::residual(L, x, f, F.r.p, s);
    r0 = F.r.p;
    beta2 = norm2(S, F.r.p, s);
  }
  if (iters) *iters = it;
  return status;
}

void capture_fgmres(Solver& S, cudaStream_t s, cudaStream_t sb, cudaStream_t sc) {
  Fgmres& F = S.fgm;
  const Lvl& L = S.L64;
  const long long len = L.nvel;
  FgState* st = (FgState*)F.state.p;
  double* red = S.scal.p;
  CgState* cg = S.cg_dev;
  const double tol2 = S.opt.tol_inner * S.opt.tol_inner;
  const int maxit = S.opt.maxit_inner;
  { ProfScope ps_(GKB_KC_BLAS, s); k_fg_setup<<<1, 1, 0, s>>>(st, F.m, tol2, maxit); }
  GKB_CUDA(cudaMemsetAsync(S.x.p, 0, len * sizeof(double), s));
  GKB_CUDA(cudaMemcpyAsync(F.r.p, S.f.p, len * sizeof(double), cudaMemcpyDeviceToDevice, s));  // r = f - M 0
  Ops<double>::dot(len, S.f.p, S.f.p, S.red, FIN_STORE, red, s);
  auto scalar = [&](cudaStream_t q, int op, cudaGraphConditionalHandle h) {
    ProfScope ps_(GKB_KC_BLAS, q);
    k_fg_scalar<<<1, 32, 0, q>>>(op, st, red, F.h.p, F.y.p, cg, h);
  };
  capture_while(
      s, sb, 4, [&](cudaStream_t q, cudaGraphConditionalHandle h) { scalar(q, FG_BEGIN, h); },
      [&](cudaStream_t q, cudaGraphConditionalHandle hr) {
        // one cycle: V_0 = r / beta, Arnoldi steps to convergence or m
        capture_while(
            q, sc, 3,
            [&](cudaStream_t q2, cudaGraphConditionalHandle ha) {
              scalar(q2, FG_CYCLE, ha);
              ProfScope ps_(GKB_KC_BLAS, q2, len);
              k_fg_scale<<<fblocks(len), FB, 0, q2>>>(F.V.p, F.r.p, len, st, 0);
            },
            [&](cudaStream_t q2, cudaGraphConditionalHandle ha) {
              { ProfScope ps_(GKB_KC_LAYOUT, q2, len); k_fg_col<<<fblocks(len), FB, 0, q2>>>(F.V.p, F.vin.p, len, st, 1); }
              S.gmg64.vcycle(F.vin.p, F.zt.p, q2);
              { ProfScope ps_(GKB_KC_LAYOUT, q2, len); k_fg_col<<<fblocks(len), FB, 0, q2>>>(F.Z.p, F.zt.p, len, st, 0); }
              Ops<double>::apply(L, 1, F.zt.p, F.w.p, q2);
              // two passes of classical Gram-Schmidt against V_0..V_j
              for (int pass = 0; pass < 2; ++pass) {
                double* hh = pass ? F.h2.p : F.h.p;
                ProfScope ps_(GKB_KC_BLAS, q2, len * F.m / 2);
                k_mdot_d<<<dim3(FBLK, F.m + 1), FB, 0, q2>>>(F.V.p, len, F.w.p, F.part.p, st);
                k_mcols_d<<<(F.m + 64) / 64, 64, 0, q2>>>(F.part.p, FBLK, hh, 0, st);
                k_maxpy_d<<<fblocks(len), FB, 0, q2>>>(F.w.p, F.V.p, len, hh, -1.0, st, 0);
              }
              { ProfScope ps_(GKB_KC_BLAS, q2); k_mcols_d<<<(F.m + 64) / 64, 64, 0, q2>>>(F.h2.p, 1, F.h.p, 1, st); }
              Ops<double>::dot(len, F.w.p, F.w.p, S.red, FIN_STORE, red, q2);
              scalar(q2, FG_GIVENS, 0);
              { ProfScope ps_(GKB_KC_BLAS, q2, len); k_fg_scale<<<fblocks(len), FB, 0, q2>>>(F.V.p, F.w.p, len, st, 1); }
              scalar(q2, FG_NEXT, ha);
            },
            [&](cudaStream_t q2) {
              // x += Z y, then the true residual decides the restart
              scalar(q2, FG_BACKSUB, 0);
              { ProfScope ps_(GKB_KC_BLAS, q2, len * F.m / 2); k_maxpy_d<<<fblocks(len), FB, 0, q2>>>(S.x.p, F.Z.p, len, F.y.p, 1.0, st, 1); }
              Ops<double>::residual(L, S.x.p, S.f.p, F.r.p, q2);
              Ops<double>::dot(len, F.r.p, F.r.p, S.red, FIN_STORE, red, q2);
              scalar(q2, FG_RESTART, hr);
            });
      },
      [&](cudaStream_t) {});
}

// ---------------------------------------------------------------------------
// GKB as the preconditioner of an outer FGMRES on the saddle system
// ---------------------------------------------------------------------------

// Saddle vectors are one padded array: velocity (nvel) then cells (ncell).
struct SaddleOps {
  Solver& S;
  long long nv, nc;
  // y = K x = [W x_u + A x_p ; A^T x_u]
  void apply(const double* x, double* y) {
    cudaStream_t s = S.stream;
    Ops<double>::apply(S.L64, 0, x, y, s);
    Ops<double>::grad(S.L64, x + nv, S.t.p, 1.0, s);
    Ops<double>::axpby(nv, 1.0, S.t.p, 1.0, y, s);
    Ops<double>::negdiv(S.L64, x, y + nv, 1.0, s);
  }
  // z = GKB(v) to pc_tol: the AL transform and Algorithm 1 on the right-hand
  // side (v_u, v_p), velocity u + y0, pressure with zero mean when enclosed
  int precondition(const double* v, double* z, double pc_tol, int delay) {
    cudaStream_t s = S.stream;
    const Lvl& L = S.L64;
    GKB_CUDA(cudaMemcpyAsync(S.wtmp.p, v, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    GKB_CUDA(cudaMemcpyAsync(S.ctmp.p, v + nv, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    S.init_state(pc_tol, delay);
    if (S.sgraph.exec) GKB_CUDA(cudaGraphLaunch(S.sgraph.exec, s));
    else S.run_core_host();
    Ops<double>::axpby(nv, 1.0, S.u.p, 0.0, z, s);
    Ops<double>::axpby(nv, 1.0, S.y0.p, 1.0, z, s);
    const dim3 cg((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]);
    if (S.enclosed) S.cell_sum(S.pp.p, S.scal.p);
    GKB_CUDA(cudaMemsetAsync(z + nv, 0, nc * sizeof(double), s));
    {
      ProfScope ps_(GKB_KC_LAYOUT, s);
      k_shift_cells<<<cg, dim3(32, 8), 0, s>>>(L, S.pp.p, z + nv, S.enclosed ? S.scal.p : nullptr,
                                                1.0 / (double)S.ncell);
    }
    GKB_CUDA(cudaMemcpyAsync(S.gkb_host, S.gkb_dev, sizeof(GkbState), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
    const GkbState& H = *S.gkb_host;
    if (H.status != ST_OK) return H.status;
    return H.inner_status;
  }
};

int solve_preconditioned(Solver& S, const double* g, const double* r, double tol, int restart, int maxit,
                         double pc_tol, int delay, double* w_out, double* p_out, int* iters) {
  cudaStream_t s = S.stream;
  const long long nv = S.L64.nvel, nc = S.L64.ncell, len = nv + nc;
  Fgmres& F = S.fgo;
  if (F.len != len || F.m != restart) F.init(len, restart);
  const int m = restart;
  SaddleOps K{S, nv, nc};
  // right-hand side in the padded layout
  S.stage_in(g, r, nullptr, nullptr);
  DevBuf<double> b, x;
  b.alloc(len);
  x.alloc(len);
  GKB_CUDA(cudaMemcpyAsync(b.p, S.wtmp.p, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
  GKB_CUDA(cudaMemcpyAsync(b.p + nv, S.ctmp.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  auto nrm2 = [&](const double* a) {
    double hs[4];
    Ops<double>::dot(len, a, a, S.red, FIN_STORE, S.scal.p, s);
    GKB_CUDA(cudaMemcpyAsync(hs, S.scal.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    GKB_CUDA(cudaStreamSynchronize(s));
    return hs[0];
  };
  const double bb = nrm2(b.p);
  const double tol2 = tol * tol;
  double beta2 = bb;
  const double* r0 = b.p;
  int it = 0, status = ST_OK;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1), hcol(m + 2), yv(m);
  while (status == ST_OK) {
    if (!std::isfinite(beta2)) { status = ST_NAN; break; }
    if (beta2 <= tol2 * bb) break;
    if (it >= maxit) { status = ST_NOT_CONVERGED; break; }
    const double beta = sqrt(beta2);
    { ProfScope ps_(GKB_KC_BLAS, s, len); k_scale_to<<<fblocks(len), FB, 0, s>>>(F.V.p, r0, len, 1.0 / beta); }
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = F.V.p + (long long)j * len;
      double* zj = F.Z.p + (long long)j * len;
      const int pst = K.precondition(vj, zj, pc_tol, delay);
      if (pst != ST_OK && pst != ST_NOT_CONVERGED) { status = pst; break; }
      K.apply(zj, F.w.p);
      mdot(F, j + 1, F.h.p, 0, s);
      { ProfScope ps_(GKB_KC_BLAS, s, len * (j + 1)); k_maxpy<<<fblocks(len), FB, 0, s>>>(F.w.p, F.V.p, len, j + 1, F.h.p, -1.0); }
      mdot(F, j + 1, F.h2.p, 0, s);
      { ProfScope ps_(GKB_KC_BLAS, s, len * (j + 1)); k_maxpy<<<fblocks(len), FB, 0, s>>>(F.w.p, F.V.p, len, j + 1, F.h2.p, -1.0); }
      { ProfScope ps_(GKB_KC_BLAS, s); k_mcols<<<1, 64, 0, s>>>(F.h2.p, 1, j + 1, F.h.p, 1); }
      const double hn2 = nrm2(F.w.p);
      GKB_CUDA(cudaMemcpyAsync(hcol.data(), F.h.p, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
      GKB_CUDA(cudaStreamSynchronize(s));
      const double hn = sqrt(hn2);
      ++it;
      if (!std::isfinite(hn)) { status = ST_NAN; break; }
      if (hn > 0.0) {
        ProfScope ps_(GKB_KC_BLAS, s, len);
        k_scale_to<<<fblocks(len), FB, 0, s>>>(F.V.p + (long long)(j + 1) * len, F.w.p, len, 1.0 / hn);
      }
      hcol[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = a;
      }
      const double rho = hypot(hcol[j], hcol[j + 1]);
      if (!(rho > 0.0)) { status = ST_NOT_CONVERGED; break; }
      cs[j] = hcol[j] / rho;
      sn[j] = hcol[j + 1] / rho;
      hcol[j] = rho;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      k = j + 1;
      if (gv[j + 1] * gv[j + 1] <= tol2 * bb || it >= maxit || hn == 0.0) break;
    }
    if (status != ST_OK || k == 0) break;
    for (int i = k - 1; i >= 0; --i) {
      double tt = gv[i];
      for (int c = i + 1; c < k; ++c) tt -= H[(size_t)i * m + c] * yv[c];
      yv[i] = tt / H[(size_t)i * m + i];
    }
    GKB_CUDA(cudaMemcpyAsync(F.y.p, yv.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    { ProfScope ps_(GKB_KC_BLAS, s, len * k); k_maxpy<<<fblocks(len), FB, 0, s>>>(x.p, F.Z.p, len, k, F.y.p, 1.0); }
    // true residual b - K x
    K.apply(x.p, F.r.p);
    Ops<double>::axpby(len, 1.0, b.p, -1.0, F.r.p, s);
    r0 = F.r.p;
    beta2 = nrm2(F.r.p);
  }
  if (iters) *iters = it;
  // the solution through the solver's output path (mean-free pressure)
  GKB_CUDA(cudaMemcpyAsync(S.u.p, x.p, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
  GKB_CUDA(cudaMemsetAsync(S.y0.p, 0, nv * sizeof(double), s));
  GKB_CUDA(cudaMemcpyAsync(S.pp.p, x.p + nv, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  S.finish(w_out, p_out, nullptr, nullptr, false);
  return status;
}

}  // namespace gkb
