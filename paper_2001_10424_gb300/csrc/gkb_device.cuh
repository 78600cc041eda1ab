// gkb_device.cuh - device code of the GKB recurrence (Algorithm 1 with the
// transform of Eq. (3) and the stopping rule of Eq. (5)) and of the mixed
// precision inner solve: kernel bodies with explicit block coordinates (Blk),
// shared by the per-problem launches of solver.cu and the lock-step batched
// launches of lockstep.cu.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"
#include "reduce.cuh"
#include "state.cuh"

namespace gkb {

constexpr int CB = 256;

// b = r - A^T y0 ; reduce sum b^2 / N, sum b, sum b / N
__device__ __forceinline__ void gkb_b_body(const Blk& B, const Lvl& L, const double* __restrict__ rc, const double* __restrict__ y0,
                                               double* __restrict__ b, const GkbState* st, RedBuf red, double* out) {
  const int i = B.x * 32 + threadIdx.x, j = B.y * 8 + threadIdx.y, k = B.z;
  double v[3] = {0.0, 0.0, 0.0};
  if (i < L.n[0] && j < L.n[1]) {
    const long long id = cix(L, i, j, k);
    const double bv = rc[id] - L.ascale * neg_div<double>(L, y0, i, j, k);
    const double ni = st->nd ? st->nd[id] : st->n_scale;
    b[id] = bv;
    v[0] = bv * bv / ni;
    v[1] = bv;
    v[2] = bv / ni;
  }
  grid_reduce<3>(v, red, FIN_STORE, out, B);
}

// g = N^-1 A^T v - alpha q ; reduce sum N g^2, sum N g
__device__ __forceinline__ void gk1_body(const Blk& B, const Lvl& L, const double* __restrict__ v, const double* __restrict__ q,
                                             double* __restrict__ gq, const GkbState* st, RedBuf red, double* out) {
  const int i = B.x * 32 + threadIdx.x, j = B.y * 8 + threadIdx.y, k = B.z;
  double acc[2] = {0.0, 0.0};
  if (i < L.n[0] && j < L.n[1]) {
    const long long id = cix(L, i, j, k);
    const double ni = st->nd ? st->nd[id] : st->n_scale;
    const double g = L.ascale * neg_div<double>(L, v, i, j, k) / ni - st->alpha * q[id];
    gq[id] = g;
    acc[0] = ni * g * g;
    acc[1] = ni * g;
  }
  grid_reduce<2>(acc, red, FIN_STORE, out, B);
}

// f = A q_{k+1} with q_{k+1} = (g - mean) / beta (mean cancels on active faces)
__device__ __forceinline__ void gk2_body(const Blk& B, const Lvl& L, const double* __restrict__ gq, double* __restrict__ f,
                                             const GkbState* st) {
  const int i = B.x * 32 + threadIdx.x, j = B.y * 8 + threadIdx.y, k = B.z;
  const double sc = (st->beta > 0.0 && !st->stop) ? L.ascale / st->beta : 0.0;
  const double mean = st->mean;
#define GKB_GK2(C, DI, DJ, DK)                                                   \
  {                                                                              \
    bool store = (L.dim == 2) ? (k == 0 && i <= L.n[0] && j <= L.n[1])           \
                              : (i <= L.n[0] && j <= L.n[1] && (C == 2 ? k <= L.n[2] : k < L.n[2])); \
    if (store) {                                                                 \
      double val = 0.0;                                                          \
      if (face_active<C>(L, i, j, k)) {                                          \
        const double pp = cell_in(L, i, j, k) ? gq[cix(L, i, j, k)] - mean : 0.0; \
        const double pm = cell_in(L, i - DI, j - DJ, k - DK) ? gq[cix(L, i - DI, j - DJ, k - DK)] - mean : 0.0; \
        val = sc * (pp - pm);                                                    \
      }                                                                          \
      f[L.off[C] + cix(L, i, j, k)] = val;                                       \
    }                                                                            \
  }
  GKB_GK2(0, 1, 0, 0)
  GKB_GK2(1, 0, 1, 0)
  if (L.dim == 3) GKB_GK2(2, 0, 0, 1)
#undef GKB_GK2
}

// w = x - beta v
__device__ __forceinline__ void gk3_body(const Blk& B, long long len, const double* __restrict__ x, const double* __restrict__ v,
                                            double* __restrict__ w, const GkbState* st) {
  const double beta = st->stop && st->beta == 0.0 ? 0.0 : st->beta;
  for (long long t = B.x * (long long)CB + threadIdx.x; t < len; t += (long long)B.nx * CB)
    w[t] = x[t] - beta * v[t];
}

// v = w / alpha ; u += zeta v     (first: u = zeta v)
__device__ __forceinline__ void gk4v_body(const Blk& B, long long len, const double* __restrict__ w, double* __restrict__ v,
                                             double* __restrict__ u, const GkbState* st, int first) {
  if (st->stop && st->converged && st->alpha == 0.0) return;
  if (st->status != 0) return;
  const double ia = 1.0 / st->alpha, z = st->zeta;
  for (long long t = B.x * (long long)CB + threadIdx.x; t < len; t += (long long)B.nx * CB) {
    const double vn = w[t] * ia;
    v[t] = vn;
    u[t] = first ? z * vn : u[t] + z * vn;
  }
}

// q = (g - mean) / beta ; d = (q - beta d) / alpha ; p -= zeta d   (first: d = q / alpha, p = -zeta d)
__device__ __forceinline__ void gk4c_body(const Blk& B, const Lvl& L, const double* __restrict__ gq, double* __restrict__ q,
                                              double* __restrict__ d, double* __restrict__ p, const GkbState* st,
                                              int first) {
  if (st->stop && st->converged && st->alpha == 0.0) return;
  if (st->status != 0) return;
  const int i = B.x * 32 + threadIdx.x, j = B.y * 8 + threadIdx.y, k = B.z;
  if (i >= L.n[0] || j >= L.n[1]) return;
  const long long id = cix(L, i, j, k);
  const double ia = 1.0 / st->alpha, z = st->zeta, beta = st->beta;
  if (first) {
    const double dn = q[id] * ia;
    d[id] = dn;
    p[id] = -z * dn;
  } else {
    const double qn = (gq[id] - st->mean) / beta;
    q[id] = qn;
    const double dn = (qn - beta * d[id]) * ia;
    d[id] = dn;
    p[id] -= z * dn;
  }
}

// q1 = N^-1 (b - mean) / beta1
__device__ __forceinline__ void gkb_q1_body(const Blk& B, const Lvl& L, const double* __restrict__ b, double* __restrict__ q,
                                                const GkbState* st) {
  const int i = B.x * 32 + threadIdx.x, j = B.y * 8 + threadIdx.y, k = B.z;
  if (i >= L.n[0] || j >= L.n[1]) return;
  const long long id = cix(L, i, j, k);
  const double ni = st->nd ? st->nd[id] : st->n_scale;
  q[id] = (st->beta > 0.0) ? (b[id] - st->mean) / (ni * st->beta) : 0.0;
}

// mixed precision: r32 = (float) r64 ; x64 += x32, x32 = 0
__device__ __forceinline__ void cvt_f32_body(const Blk& B, long long len, const double* __restrict__ r, float* __restrict__ o,
                                                const int* pred) {
  if (pred && !*pred) return;
  for (long long t = B.x * (long long)CB + threadIdx.x; t < len; t += (long long)B.nx * CB)
    o[t] = (float)r[t];
}

__device__ __forceinline__ void mixed_accum_body(const Blk& B, long long len, float* __restrict__ x32, double* __restrict__ x64,
                                                    const int* pred) {
  if (pred && !*pred) return;
  for (long long t = B.x * (long long)CB + threadIdx.x; t < len; t += (long long)B.nx * CB) {
    x64[t] += (double)x32[t];
    x32[t] = 0.0f;
  }
}

enum { S_BETA1 = 0, S_ALPHA1 = 1, S_BETA = 2, S_ALPHA = 3 };

__device__ __forceinline__ void hist_put(double* h, int cap, int i, double v) {
  if (h && i >= 0 && i < cap) h[i] = v;
}

// scalar part of Algorithm 1 and the stopping rule (one thread)
__device__ __forceinline__ void gkb_scalar_op(int op, GkbState* st, const double* red) {
  GkbState& S = *st;
  switch (op) {
    case S_BETA1: {
      // beta_1 = ||b||_{N^-1} on the mean-free b:
      // sum (b - m)^2 / N = sum b^2 / N - 2 m sum b / N + m^2 sum 1 / N
      const double mean = S.enclosed ? red[1] / S.ncells : 0.0;
      double s2 = red[0] - 2.0 * mean * red[2] + mean * mean * S.ninvsum;
      if (s2 < 0) s2 = 0;
      S.mean = mean;
      S.beta = sqrt(s2);
      hist_put(S.h_beta, S.hcap, 0, S.beta);
      if (!isfinite(S.beta)) { S.status = ST_NAN; S.stop = 1; }
      else if (S.beta == 0.0) { S.stop = 1; S.converged = 1; }
    } break;
    case S_ALPHA1: {
      const double a2 = red[0];
      if (!isfinite(a2)) { S.status = ST_NAN; S.stop = 1; break; }
      if (!(a2 > 0.0)) {
        if (a2 < 0.0) S.status = ST_NOT_SPD;
        S.alpha = 0.0; S.stop = 1; S.converged = (a2 == 0.0);
        break;
      }
      S.alpha = sqrt(a2);
      S.zeta = S.beta / S.alpha;
      S.K = 1;
      S.zsum = S.zeta * S.zeta;
      S.ring[1 % GKB_RING] = S.zeta * S.zeta;
      hist_put(S.h_alpha, S.hcap, 0, S.alpha);
      hist_put(S.h_zeta, S.hcap, 0, S.zeta);
      if (S.maxit <= 0) S.stop = 1;
    } break;
    case S_BETA: {
      // beta_{k+1} = ||g - c||_N with c = sum N g / sum N, the N-weighted
      // mean (the plain mean when N = n I): sum N g^2 - c^2 sum N
      S.k += 1;
      const double mean = S.enclosed ? red[1] / S.nsum : 0.0;
      double s2 = red[0] - S.nsum * mean * mean;
      if (s2 < 0) s2 = 0;
      S.mean = mean;
      S.beta = sqrt(s2);
      hist_put(S.h_beta, S.hcap, S.k, S.beta);
      if (!isfinite(S.beta)) { S.status = ST_NAN; S.stop = 1; }
      else if (S.beta == 0.0) { S.stop = 1; S.converged = 1; S.alpha = 0.0; }
    } break;
    case S_ALPHA: {
      if (S.stop) break;  // breakdown already handled
      const double a2 = red[0];
      if (!isfinite(a2)) { S.status = ST_NAN; S.stop = 1; break; }
      if (!(a2 > 0.0)) {
        if (a2 < 0.0) S.status = ST_NOT_SPD;
        S.alpha = 0.0; S.stop = 1; S.converged = (a2 == 0.0);
        break;
      }
      S.alpha = sqrt(a2);
      S.zeta = -S.beta / S.alpha * S.zeta;
      S.K += 1;
      const double z2 = S.zeta * S.zeta;
      S.zsum += z2;
      S.ring[S.K % GKB_RING] = z2;
      double tail = 0.0;
      const int j0 = (S.K - S.delay > 1) ? S.K - S.delay : 1;
      for (int j = j0; j <= S.K; ++j) tail += S.ring[j % GKB_RING];
      S.est = sqrt(tail / S.zsum);
      hist_put(S.h_alpha, S.hcap, S.k, S.alpha);
      hist_put(S.h_zeta, S.hcap, S.K - 1, S.zeta);
      hist_put(S.h_est, S.hcap, S.k - 1, S.est);
      if (S.est <= S.tol) { S.converged = 1; S.stop = 1; }
      else if (S.k >= S.maxit) S.stop = 1;
    } break;
  }
}

}  // namespace gkb
