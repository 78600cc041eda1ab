// api.cu - the extern "C" boundary declared in include/gkb.h. Every entry
// point converts internal errors into status codes; nothing is thrown across
// the ABI.
#include <string.h>

#include <new>

#include "solver.cuh"
#include "unet.cuh"

struct gkb_ctx {
  gkb::Solver s;
  int device = 0;
};

namespace {

thread_local std::string g_create_error = "no error";

template <class F>
int guarded(gkb_handle h, F&& fn) {
  if (!h) return GKB_ERR_INVALID_ARG;
  struct ProfBind {
    explicit ProfBind(gkb::Profiler* p) { gkb::g_prof = p; }
    ~ProfBind() { gkb::g_prof = nullptr; }
  } bind(&h->s.prof);
  try {
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
      h->s.last_error = cudaGetErrorString(e);
      return GKB_ERR_CUDA;
    }
    int rc = fn();
    if (rc != GKB_OK) {
      if (h->s.last_error.empty() || h->s.last_error == "no error") h->s.last_error = "solver status " + std::to_string(rc);
    }
    return rc;
  } catch (const gkb::Error& err) {
    h->s.last_error = err.msg;
    return err.code;
  } catch (const std::bad_alloc&) {
    h->s.last_error = "host allocation failed";
    return GKB_ERR_OOM;
  } catch (...) {
    h->s.last_error = "unexpected internal error";
    return GKB_ERR_CUDA;
  }
}

}  // namespace

extern "C" {

int gkb_default_options(gkb_options* opt) {
  if (!opt) return GKB_ERR_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->precision = GKB_PREC_FP64;
  opt->inner = GKB_INNER_GMG_PCG;
  opt->tol_inner = 1e-10;
  opt->maxit = 1000;
  opt->maxit_inner = 2000;
  opt->smoother_degree = 2;
  opt->coarse_max = 8;
  opt->mixed_rtol = 1e-3;
  opt->use_graph = 1;
  opt->profile = 0;
  opt->kernel_variant = 0;
  opt->unet_side = 0;
  opt->fcg_rho = 0.8;
  opt->fgmres_restart = 30;
  opt->cheb_lo = 0.1;
  opt->cheb_hi = 1.1;
  opt->stream = nullptr;
  opt->viscous_form = GKB_VISC_LAPLACE;
  opt->batch_lockstep = 0;
  opt->tail_side = 0;
  return GKB_OK;
}

int gkb_create(gkb_handle* out, const gkb_options* opt) {
  if (!out || !opt) return GKB_ERR_INVALID_ARG;
  *out = nullptr;
  if (opt->precision != GKB_PREC_FP64 && opt->precision != GKB_PREC_MIXED) return GKB_ERR_INVALID_ARG;
  if (opt->inner < GKB_INNER_CG || opt->inner > GKB_INNER_FGMRES) return GKB_ERR_INVALID_ARG;
  if (opt->inner == GKB_INNER_FGMRES && (opt->fgmres_restart < 1 || opt->fgmres_restart > 64))
    return GKB_ERR_INVALID_ARG;
  if (!(opt->cheb_lo > 0 && opt->cheb_lo < opt->cheb_hi && opt->cheb_hi < 10)) return GKB_ERR_INVALID_ARG;
  if (opt->viscous_form != GKB_VISC_LAPLACE && opt->viscous_form != GKB_VISC_SYMGRAD) return GKB_ERR_INVALID_ARG;
  if (opt->batch_lockstep < 0 || opt->batch_lockstep > 1 || opt->tail_side < 0) return GKB_ERR_INVALID_ARG;
  if (opt->unet_side < 0 || !(opt->fcg_rho >= 0 && opt->fcg_rho < 1) || opt->autotune < 0 || opt->autotune > 1)
    return GKB_ERR_INVALID_ARG;
  if (!(opt->tol_inner > 0) || opt->maxit < 0 || opt->maxit > 100000000 || opt->maxit_inner < 1 ||
      opt->smoother_degree < 1 || opt->smoother_degree > 16 || opt->coarse_max < 4 ||
      !(opt->mixed_rtol >= 0 && opt->mixed_rtol < 1) || opt->kernel_variant < 0 || opt->kernel_variant > 2)
    return GKB_ERR_INVALID_ARG;
  gkb_ctx* h = new (std::nothrow) gkb_ctx();
  if (!h) return GKB_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete h;
    return GKB_ERR_CUDA;
  }
  h->s.opt = *opt;
  h->s.stream = (cudaStream_t)opt->stream;
  h->s.last_error = "no error";
  *out = h;
  return GKB_OK;
}

int gkb_set_problem(gkb_handle h, const gkb_grid* grid, const double* viscosity, double mu0, double gamma,
                    double n_scale) {
  return guarded(h, [&] {
    h->s.set_problem(grid, viscosity, mu0, gamma, n_scale);
    return GKB_OK;
  });
}

int gkb_set_problem_n(gkb_handle h, const gkb_grid* grid, const double* viscosity, double mu0, double gamma,
                      const double* n_diag) {
  return guarded(h, [&] {
    if (!n_diag) throw gkb::Error{GKB_ERR_INVALID_ARG, "n_diag is NULL"};
    h->s.set_problem(grid, viscosity, mu0, gamma, 0.0, n_diag);
    return GKB_OK;
  });
}

int gkb_set_unet(gkb_handle h, gkb_unet u) {
  return guarded(h, [&] {
    if (u && u->device != h->device) throw gkb::Error{GKB_ERR_INVALID_ARG, "the network lives on another device"};
    h->s.set_net(u ? &u->u : nullptr);
    return GKB_OK;
  });
}

int gkb_harvest_pairs(gkb_handle h, const double* f, int max_pairs, float* x_img, float* t_img, int* n_pairs) {
  return guarded(h, [&] { return h->s.harvest(f, max_pairs, x_img, t_img, n_pairs); });
}

int gkb_get_options(gkb_handle h, gkb_options* out) {
  return guarded(h, [&] {
    if (!out) return GKB_ERR_INVALID_ARG;
    *out = h->s.opt;
    return GKB_OK;
  });
}

int gkb_layout(gkb_handle h, int64_t* m, int64_t* n) {
  return guarded(h, [&] {
    if (!h->s.have_problem) throw gkb::Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
    if (m) *m = h->s.m;
    if (n) *n = h->s.ncell;
    return GKB_OK;
  });
}

int gkb_solve(gkb_handle h, const double* g, const double* r, double tol, int delay, double* w_out, double* p_out,
              const double* w0, const double* p0) {
  return guarded(h, [&] { return h->s.solve(g, r, tol, delay, w_out, p_out, w0, p0); });
}

int gkb_solve_preconditioned(gkb_handle h, const double* g, const double* r, double tol, int restart, int maxit,
                             double pc_tol, int delay, double* w_out, double* p_out, int* iterations) {
  return guarded(h, [&] {
    gkb::Solver& S = h->s;
    if (!S.have_problem) throw gkb::Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
    if (!g || !r || !w_out || !p_out) throw gkb::Error{GKB_ERR_INVALID_ARG, "g, r, w_out and p_out must not be NULL"};
    if (!(tol > 0) || !(pc_tol > 0) || restart < 1 || restart > 64 || maxit < 1 || delay < 0 || delay > gkb::GKB_RING - 2)
      throw gkb::Error{GKB_ERR_INVALID_ARG, "bad outer solver arguments"};
    int it = 0;
    const int st = gkb::solve_preconditioned(S, g, r, tol, restart, maxit, pc_tol, delay, w_out, p_out, &it);
    if (iterations) *iterations = it;
    return st;
  });
}

int gkb_solve_batched(gkb_handle* hs, int count, const double* const* g, const double* const* r, double tol,
                      int delay, double* const* w_out, double* const* p_out) {
  if (!hs || count < 1 || !hs[0]) return GKB_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!hs[i] || hs[i]->device != hs[0]->device) return GKB_ERR_INVALID_ARG;
  return guarded(hs[0], [&] {
    std::vector<gkb::Solver*> S(count);
    for (int i = 0; i < count; ++i) S[i] = &hs[i]->s;
    return gkb::solve_batched(S.data(), count, g, r, tol, delay, w_out, p_out);
  });
}

int gkb_stats(gkb_handle h, gkb_stats_t* out) {
  return guarded(h, [&] {
    if (!out) throw gkb::Error{GKB_ERR_INVALID_ARG, "NULL stats"};
    *out = h->s.stats;
    return GKB_OK;
  });
}

int gkb_history(gkb_handle h, double* alpha, double* beta, double* zeta, double* estimate, int* inner_its,
                int capacity) {
  int written = 0;
  int rc = guarded(h, [&] {
    if (!h->s.have_problem) throw gkb::Error{GKB_ERR_INVALID_ARG, "gkb_set_problem has not been called"};
    if (capacity < 0) throw gkb::Error{GKB_ERR_INVALID_ARG, "negative capacity"};
    const int cap = h->s.opt.maxit + 2;
    std::vector<double> hv(4 * (size_t)cap);
    gkb::check_cuda(cudaMemcpy(hv.data(), h->s.hist.p, hv.size() * sizeof(double), cudaMemcpyDeviceToHost), "history");
    const int k = h->s.stats.outer_iterations;
    const int nz = std::min(capacity, std::min(cap, k + 1));
    const int nb = std::min(capacity, std::min(cap, k + 1));
    for (int i = 0; i < nz; ++i) {
      if (alpha) alpha[i] = hv[i];
      if (zeta) zeta[i] = hv[2 * (size_t)cap + i];
    }
    for (int i = 0; i < nb; ++i)
      if (beta) beta[i] = hv[(size_t)cap + i];
    for (int i = 0; i < std::min(capacity, k); ++i)
      if (estimate) estimate[i] = hv[3 * (size_t)cap + i];
    if (inner_its) {
      const int ni = std::min<int>(capacity, std::min<int>(h->s.stats.inner_solves, h->s.opt.maxit + 4));
      if (ni > 0)
        gkb::check_cuda(cudaMemcpy(inner_its, h->s.hist_inner.p, ni * sizeof(int), cudaMemcpyDeviceToHost), "history");
    }
    written = nz;
    return GKB_OK;
  });
  return rc == GKB_OK ? written : -rc;
}

int gkb_apply(gkb_handle h, int op, const double* x, double* y) {
  return guarded(h, [&] {
    h->s.apply(op, x, y);
    return GKB_OK;
  });
}

int gkb_precond(gkb_handle h, const double* r, double* z) {
  return guarded(h, [&] {
    h->s.precond(r, z);
    return GKB_OK;
  });
}

int gkb_boundary_rhs(gkb_handle h, int side, const double* normal_velocity, double* g, double* r) {
  return guarded(h, [&] {
    h->s.boundary_rhs(side, normal_velocity, g, r);
    return GKB_OK;
  });
}

const char* gkb_last_error(gkb_handle h) {
  if (!h) return "invalid handle";
  return h->s.last_error.c_str();
}

int gkb_destroy(gkb_handle h) {
  if (!h) return GKB_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  gkb::forget_batches(&h->s);
  delete h;
  return GKB_OK;
}

}  // extern "C"
