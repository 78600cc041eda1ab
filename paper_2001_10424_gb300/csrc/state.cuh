// state.cuh - device-resident solver scalars and the reduction finalisers.
//
// All scalars of the inner CG and of the GKB recurrence live in device
// memory; kernels read them through pointers and the finalisers of the
// fused reductions update them, so no host round trip is needed inside a
// solve.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace gkb {

// status codes mirrored from include/gkb.h
constexpr int ST_OK = 0;
constexpr int ST_INVALID = 1;
constexpr int ST_NOT_SPD = 2;
constexpr int ST_NOT_CONVERGED = 3;
constexpr int ST_INNER_NOT_CONVERGED = 4;
constexpr int ST_NAN = 5;
constexpr int ST_TIMEOUT = 6;

enum FinOp {
  FIN_NONE = 0,
  FIN_STORE = 1,   // st is double[4]: store the sums
  FIN_CG_INIT,     // s0 = f.f
  FIN_CG_RZ0,      // s0 = r.z (first)
  FIN_CG_PAP,      // s0 = p.Mp -> alpha
  FIN_CG_RR,       // s0 = r.r  -> convergence test
  FIN_CG_RZ,       // s0 = r.z  -> beta
  FIN_MX_RR,       // s0 = r32.r32 -> iteration count, reliable-update trigger
  FIN_MX_RR64,     // s0 = r64.r64 (true FP64 residual) -> convergence test
  FIN_FCG_RZ,      // s0 = r.z, s1 = z.q -> flexible beta = -z.q / p.q
};

struct CgState {
  double ff;        // ||f||^2
  double rr;        // ||r||^2
  double rz_old;    // r.z of the previous iteration
  double pAp;
  double alpha, beta;
  double tol2;      // tol_inner^2
  int it;           // iterations of this solve
  int maxit;
  int done;         // 1 once the solve has stopped
  int status;       // ST_* of this solve
  long long total_it;
  int solves;
  int update;       // mixed form: 1 when an FP64 residual recomputation is due
  double rmax2;     // mixed form: ||r||^2 at the last FP64 recomputation
  double delta2;    // mixed form: trigger ratio squared (< 0: no replacement)
  double rr64;      // mixed form: last true FP64 ||r||^2
  int graph_iters;  // loop-body executions of the graph form (device counted)
  int fallback;     // flexible form: 1 once the solve has switched to plain GMG-PCG
  int fb_iters;     // loop-body executions of the fallback loop (graph form)
  double rho2;      // flexible form: fall back when ||r_k||^2 > rho2^k ||f||^2 (k >= 5)
};

// the flexible CG gives up on its preconditioner: it stops here and the
// solve continues as plain GMG-PCG from the current iterate
__device__ __forceinline__ void fcg_fallback(CgState* c) {
  c->fallback = 1;
  c->done = 1;
}

__device__ __forceinline__ void cg_fail(CgState* c, int code) {
  if (c->status == ST_OK) c->status = code;
  c->done = 1;
}

__device__ __forceinline__ void finalize(int op, const double* s, void* st) {
  switch (op) {
    case FIN_STORE: {
      double* o = (double*)st;
      o[0] = s[0]; o[1] = s[1]; o[2] = s[2]; o[3] = s[3];
    } break;
    case FIN_CG_INIT: {
      CgState* c = (CgState*)st;
      c->ff = s[0]; c->rr = s[0]; c->it = 0; c->status = ST_OK; c->alpha = 0.0; c->beta = 0.0;
      c->rmax2 = s[0]; c->rr64 = s[0]; c->update = 0;
      c->done = (s[0] == 0.0) ? 1 : 0;
      c->solves += 1;
      if (!isfinite(s[0])) cg_fail(c, ST_NAN);
    } break;
    case FIN_CG_RZ0: {
      CgState* c = (CgState*)st;
      c->rz_old = s[0];
      if (!isfinite(s[0])) cg_fail(c, ST_NAN);
    } break;
    case FIN_CG_PAP: {
      CgState* c = (CgState*)st;
      c->pAp = s[0];
      if (c->done) { c->alpha = 0.0; break; }
      if (!isfinite(s[0])) { c->alpha = 0.0; cg_fail(c, ST_NAN); }
      else if (!(s[0] > 0.0)) { c->alpha = 0.0; cg_fail(c, ST_NOT_SPD); }
      else c->alpha = c->rz_old / s[0];
    } break;
    case FIN_CG_RR: {
      CgState* c = (CgState*)st;
      if (c->done) break;
      c->rr = s[0];
      c->it += 1;
      c->total_it += 1;
      if (!isfinite(s[0])) cg_fail(c, ST_NAN);
      else if (s[0] <= c->tol2 * c->ff) c->done = 1;
      else if (c->it >= c->maxit) cg_fail(c, ST_INNER_NOT_CONVERGED);
    } break;
    case FIN_MX_RR: {
      CgState* c = (CgState*)st;
      if (c->done) break;
      c->rr = s[0];
      c->it += 1;
      c->total_it += 1;
      if (!isfinite(s[0])) { cg_fail(c, ST_NAN); break; }
      if (c->delta2 < 0.0) {
        // ablation without FP64 residual replacement: the FP32 recursion's
        // own convergence claim ends the solve
        c->update = 0;
        if (s[0] <= c->tol2 * c->ff) c->done = 1;
        else if (c->it >= c->maxit) cg_fail(c, ST_INNER_NOT_CONVERGED);
        break;
      }
      c->update = (s[0] <= c->delta2 * c->rmax2 || s[0] <= c->tol2 * c->ff || c->it >= c->maxit) ? 1 : 0;
    } break;
    case FIN_MX_RR64: {
      CgState* c = (CgState*)st;
      c->rr64 = s[0];
      c->rmax2 = s[0];
      c->update = 0;
      if (!isfinite(s[0])) cg_fail(c, ST_NAN);
      else if (s[0] <= c->tol2 * c->ff) c->done = 1;
      else if (c->it >= c->maxit) cg_fail(c, ST_INNER_NOT_CONVERGED);
    } break;
    case FIN_CG_RZ: {
      CgState* c = (CgState*)st;
      if (c->done) break;
      c->beta = (c->rz_old != 0.0) ? s[0] / c->rz_old : 0.0;
      c->rz_old = s[0];
    } break;
    case FIN_FCG_RZ: {
      // flexible CG (Notay's FCG(1)): the new direction is made M-orthogonal
      // to the previous one, beta = -(z, M p) / (p, M p); with a fixed SPD
      // preconditioner this equals the Polak-Ribiere form of the CG beta
      CgState* c = (CgState*)st;
      if (c->done) break;
      // a non-finite preconditioned vector, or a residual that falls behind
      // the contraction rate rho per iteration, hands over to GMG-PCG
      if (!isfinite(s[0]) || !isfinite(s[1])) { c->beta = 0.0; fcg_fallback(c); break; }
      if (c->rho2 > 0.0 && c->it >= 5 && c->rr > c->ff * pow(c->rho2, (double)c->it)) { fcg_fallback(c); break; }
      c->beta = (c->pAp > 0.0) ? -s[1] / c->pAp : 0.0;
      c->rz_old = s[0];
    } break;
    default: break;
  }
}

constexpr int GKB_RING = 64;  // delay d <= GKB_RING - 2

struct GkbState {
  double alpha, beta, zeta;  // current alpha_k, beta_k, zeta_k
  double mean;               // mean removed from the N-step vector (enclosed)
  double zsum;               // sum_{j<=K} zeta_j^2
  double est;                // latest lower-bound estimate
  double tol;
  double n_scale;            // N = n_scale * I (nd == null)
  double ncells;             // number of cells (for the mean)
  const double* nd;          // diagonal of N per padded cell, or null
  double nsum, ninvsum;      // sum of N_i and of 1 / N_i over the cells
  double red[4];             // raw results of the last FIN_STORE reduction
  double ring[GKB_RING];     // zeta^2, indexed by K mod GKB_RING
  int delay, maxit, enclosed;
  int k;                     // while-loop iterations done
  int K;                     // zetas known
  int status;                // ST_* (ST_OK while running or converged)
  int stop;                  // 1 once the loop must end
  int converged;             // 1 if the estimate met tol (or happy breakdown)
  double* h_alpha;           // history buffers (device), capacity hcap
  double* h_beta;
  double* h_zeta;
  double* h_est;
  int* h_inner;              // CG iterations of each inner solve, capacity icap
  int hcap;
  int icap;
  // inner-solve bookkeeping kept on the device (graph form)
  int inner_status;          // first non-OK inner status
  int inner_solves;
  long long inner_its;       // total CG iterations
  long long inner_runs;      // total loop-body executions of the inner graphs
  long long inner_fb_runs;   // total loop-body executions of the fallback loops
  int outer_runs;            // loop-body executions of the outer graph
  int inner_fallbacks;       // flexible inner solves that switched to GMG-PCG
};

}  // namespace gkb
