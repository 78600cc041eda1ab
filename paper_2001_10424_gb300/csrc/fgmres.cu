// fgmres.cu - restarted flexible GMRES (FGMRES(m)), host-sequenced, in two
// roles: the inner solve M x = f with one V-cycle as the right
// preconditioner (the paper's alternative inner Krylov method to CG, Sec. 3,
// Sec. 4.1.3), and the outer solve of the saddle system [W A; A^T 0] with the
// GKB solver itself, run to a loose tolerance, as the preconditioner (Sec. 3:
// GKB used as a preconditioner rather than a solver).
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
