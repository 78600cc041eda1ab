// lockstep.cu - lock-step batched solve of independent problems.
//
// The problems of a batch advance together: every step of the solve (a
// smoothing step of one multigrid level, a CG update, a GKB vector update, a
// reduction) is ONE kernel launch over all problems that take part in it.
// A launch's 1D grid is the concatenation of the problems' own grids; a
// block map sends block b to (problem, block of that problem's grid), and the
// kernel bodies shared with the single-problem launches run with exactly the
// block coordinates, grid extents and reduction buffers of the problem's own
// launch. Results therefore equal the problems' individual solves bit for bit.
//
// Control flow follows the individual solves through per-problem snapshot
// flags: at the top of every iteration of the outer loop of Algorithm 1 and
// of the inner CG loop, a small kernel records which problems still run that
// loop (their own stopping rule, Eq. (5), and the inner tolerance decide) and
// sets the graph's loop condition to "any problem still runs". Every launch
// in a loop body skips the blocks of problems whose flag is 0, so a problem
// executes the same sequence of steps as its own graph would, and finished
// problems cost only an early exit of their blocks.
//
// The V-cycle walks the levels by depth from the finest: problems with more
// levels than d + 1 smooth and restrict at depth d; every problem's coarsest
// level is solved in one launch (independent dense products); the up-sweep
// mirrors the down-sweep.
//
// Scope: 2D problems with constant viscosity, the Laplacian viscous form,
// N = n_scale I, GMG-PCG inner solves in FP64 or in the mixed form, the same
// smoother degree and iteration limits. Other batches use one graph branch
// per problem (solver.cu).
#include <cuda_runtime.h>

#include <cstring>
#include <functional>
#include <map>
#include <type_traits>
#include <vector>

#include "../../include/gkb.h"
#include "gkb_device.cuh"
#include "kernels_impl.cuh"
#include "lockstep.cuh"
#include "solver.cuh"

namespace gkb {

namespace {

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------

// common head of every job: where its blocks start in the batched grid, its
// own launch grid, and the flags that gate it (null: always on)
struct JobHead {
  unsigned first, gx, gy, gz;
  const int* active;  // the problem's flag for this step
  const int* pred;    // an extra per-problem condition (mixed reliable update)
};

__device__ __forceinline__ bool job_on(const JobHead& h) {
  return (!h.active || *h.active) && (!h.pred || *h.pred);
}

__device__ __forceinline__ Blk job_blk(const JobHead& h) {
  const unsigned l = blockIdx.x - h.first;
  Blk B;
  B.nx = h.gx;
  B.ny = h.gy;
  B.nz = h.gz;
  B.x = l % h.gx;
  const unsigned r = l / h.gx;
  B.y = r % h.gy;
  B.z = r / h.gy;
  return B;
}

// this block's job (map: job of every block of the launch): its gate is
// read first (gated-off blocks exit after two dependent loads), then the job
// is copied into shared memory so that the body reads the level descriptor
// and pointers from there
#define LS_RUN(JT, ...)                                                  \
  __shared__ __align__(16) unsigned js_raw[sizeof(JT) / 4];              \
  {                                                                      \
    const JT* jg_ = jobs + map[blockIdx.x];                              \
    if (!job_on(jg_->h)) return;                                         \
    const unsigned* jw_ = (const unsigned*)jg_;                          \
    const int tid_ = threadIdx.x + blockDim.x * threadIdx.y;             \
    for (int w_ = tid_; w_ < (int)(sizeof(JT) / 4); w_ += blockDim.x * blockDim.y) \
      js_raw[w_] = jw_[w_];                                              \
  }                                                                      \
  __syncthreads();                                                       \
  const JT& job = *(const JT*)js_raw;                                    \
  const Blk B = job_blk(job.h);                                          \
  __VA_ARGS__;

template <typename T>
struct JTile { JobHead h; Lvl L; int wonly; const T* x; const T* b; T* y; RedBuf red; int fin; void* st; };
template <typename T, int MODE, bool DOT>
__global__ void __launch_bounds__(BX* BY) kb_tile(const JTile<T>* jobs, const unsigned* map) {
  LS_RUN(JTile<T>, mac_tile_body<T, false, MODE, DOT>(B, job.L, job.wonly, job.x, job.b, job.y, job.red, job.fin, job.st, nullptr))
}

// use2: the level takes the class-stencil smoother (as Ops::cheb decides)
template <typename T>
struct JCheb { JobHead h; Lvl L; const T* r; T* x; T* d; T ca, cb; int x_zero, use2; const T* table; Fold2In<T> fs; };
template <typename T>
__device__ __forceinline__ void cheb_job(const Blk& B, const JCheb<T>& job) {
  if (job.use2) cheb2_body<T>(B, job.L, job.r, job.x, job.d, job.ca, job.cb, job.x_zero, job.table, job.fs);
  else cheb_body<T, false>(B, job.L, job.r, job.x, job.d, job.ca, job.cb, job.x_zero, job.table);
}
template <typename T>
__global__ void __launch_bounds__(BX* BY) kb_cheb(const JCheb<T>* jobs, const unsigned* map) {
  LS_RUN(JCheb<T>, cheb_job<T>(B, job))
}

template <typename T>
struct JRestr { JobHead h; Lvl Lf, Lc; const T* rf; T* bc; T* tmp; };
template <typename T>
__global__ void __launch_bounds__(BX* BY) kb_restr_a(const JRestr<T>* jobs, const unsigned* map) {
  LS_RUN(JRestr<T>, restrict_flux2d_a_body<T>(B, job.Lf, job.Lc, job.rf, job.bc, job.tmp))
}
template <typename T>
__global__ void __launch_bounds__(BX* BY) kb_restr_b(const JRestr<T>* jobs, const unsigned* map) {
  LS_RUN(JRestr<T>, restrict_flux2d_b_body<T>(B, job.Lc, job.tmp, job.bc))
}

template <typename T>
struct JProl { JobHead h; Lvl Lf, Lc; const T* xc; T* xf; };
template <typename T>
__global__ void __launch_bounds__(BX* BY) kb_prolong(const JProl<T>* jobs, const unsigned* map) {
  LS_RUN(JProl<T>, prolong_flux2d_body<T>(B, job.Lf, job.Lc, job.xc, job.xf))
}

template <typename T>
struct JCoarse { JobHead h; int m; const T* Minv; const int* idx; const T* b; T* x; };
template <typename T>
__global__ void kb_coarse(const JCoarse<T>* jobs, const unsigned* map) {
  LS_RUN(JCoarse<T>, coarse_solve_body<T>(B, job.m, job.Minv, job.idx, job.b, job.x))
}

template <typename T>
struct JDot { JobHead h; long long len; const T* a; const T* b; RedBuf red; int fin; void* st; };
template <typename T>
__global__ void __launch_bounds__(RB) kb_dot(const JDot<T>* jobs, const unsigned* map) {
  LS_RUN(JDot<T>, dot_body<T>(B, job.len, job.a, job.b, job.red, job.fin, job.st, nullptr))
}

template <typename T>
struct JCgUpd { JobHead h; long long len; T* x; const T* p; T* r; const T* q; const CgState* cg; RedBuf red; void* st; int fin; };
template <typename T>
__global__ void __launch_bounds__(RB) kb_cg_update(const JCgUpd<T>* jobs, const unsigned* map) {
  LS_RUN(JCgUpd<T>, cg_update_body<T>(B, job.len, job.x, job.p, job.r, job.q, job.cg, job.red, job.st, job.fin))
}

template <typename T>
struct JCgDir { JobHead h; long long len; T* p; const T* z; const CgState* cg; int first; };
template <typename T>
__global__ void __launch_bounds__(RB) kb_cg_dir(const JCgDir<T>* jobs, const unsigned* map) {
  LS_RUN(JCgDir<T>, cg_dir_body<T>(B, job.len, job.p, job.z, job.cg, job.first))
}

// y = a x + b y (op 0), y = 0 (op 1), y = x (op 2) on flat arrays
struct JVec { JobHead h; long long len; double a, b; const double* x; double* y; int op; };
__device__ __forceinline__ void vec64_body(const Blk& B, const JVec& job) {
  if (job.op == 0) {
    axpby_body<double>(B, job.len, job.a, job.x, job.b, job.y);
    return;
  }
  const long long stride = (long long)B.nx * RB;
  for (long long t = (long long)B.x * RB + threadIdx.x; t < job.len; t += stride)
    job.y[t] = job.op == 1 ? 0.0 : job.x[t];
}
__global__ void __launch_bounds__(RB) kb_vec64(const JVec* jobs, const unsigned* map) {
  LS_RUN(JVec, vec64_body(B, job))
}
struct JVec32 { JobHead h; long long len; float* y; };
__device__ __forceinline__ void zero32_body(const Blk& B, const JVec32& job) {
  const long long stride = (long long)B.nx * RB;
  for (long long t = (long long)B.x * RB + threadIdx.x; t < job.len; t += stride) job.y[t] = 0.0f;
}
__global__ void __launch_bounds__(RB) kb_zero32(const JVec32* jobs, const unsigned* map) {
  LS_RUN(JVec32, zero32_body(B, job))
}

struct JGrad { JobHead h; Lvl L; const double* pc; double* y; double s; };
__global__ void __launch_bounds__(BX* BY) kb_grad(const JGrad* jobs, const unsigned* map) {
  LS_RUN(JGrad, grad_body<double>(B, job.L, job.pc, job.y, job.s))
}

struct JCvt { JobHead h; long long len; const double* r; float* o; float* x32; double* x64; };
__global__ void __launch_bounds__(CB) kb_cvt(const JCvt* jobs, const unsigned* map) {
  LS_RUN(JCvt, cvt_f32_body(B, job.len, job.r, job.o, nullptr))
}
__global__ void __launch_bounds__(CB) kb_accum(const JCvt* jobs, const unsigned* map) {
  LS_RUN(JCvt, mixed_accum_body(B, job.len, job.x32, job.x64, nullptr))
}

// the GKB vector kernels (one job type, op selects the body)
enum { G_B = 0, G_Q1, G_GK1, G_GK2, G_GK3, G_GK4V, G_GK4C };
struct JGkb {
  JobHead h;
  Lvl L;
  long long len;
  int op, first;
  const double *a, *b;
  double *c, *d, *e;
  const GkbState* st;
  RedBuf red;
  double* out;
};
__device__ __forceinline__ void gkb_vec_body(const Blk& B, const JGkb& job) {
  switch (job.op) {
    case G_B: gkb_b_body(B, job.L, job.a, job.b, job.c, job.st, job.red, job.out); break;
    case G_Q1: gkb_q1_body(B, job.L, job.a, job.c, job.st); break;
    case G_GK1: gk1_body(B, job.L, job.a, job.b, job.c, job.st, job.red, job.out); break;
    case G_GK2: gk2_body(B, job.L, job.a, job.c, job.st); break;
    case G_GK3: gk3_body(B, job.len, job.a, job.b, job.c, job.st); break;
    case G_GK4V: gk4v_body(B, job.len, job.a, job.c, job.d, job.st, job.first); break;
    default: gk4c_body(B, job.L, job.a, job.c, job.d, job.e, job.st, job.first); break;
  }
}
__global__ void __launch_bounds__(256) kb_gkb(const JGkb* jobs, const unsigned* map) {
  LS_RUN(JGkb, gkb_vec_body(B, job))
}

// per-problem scalar steps: one thread per problem
enum { P_SCALAR = 0, P_CG_SETUP, P_NOTE_INNER };
struct JSer {
  const int* active;
  GkbState* S;
  CgState* cg;
  const double* red;
  double tol2, delta2, rho2;
  int maxit;
};
__global__ void kb_serial(const JSer* jobs, int n, int op, int arg) {
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const JSer& J = jobs[p];
    if (J.active && !*J.active) continue;
    if (op == P_SCALAR) {
      gkb_scalar_op(arg, J.S, J.red);
    } else if (op == P_CG_SETUP) {
      CgState* c = J.cg;
      c->tol2 = J.tol2;
      c->maxit = J.maxit;
      c->delta2 = J.delta2;
      c->rho2 = J.rho2;
      c->done = 0;
      c->status = ST_OK;
      c->it = 0;
      c->update = 0;
      c->graph_iters = 0;
      c->fallback = 0;
      c->fb_iters = 0;
    } else {
      GkbState* S = J.S;
      const CgState* c = J.cg;
      const int idx = S->inner_solves;
      if (S->h_inner && idx < S->icap) S->h_inner[idx] = c->it;
      S->inner_solves = idx + 1;
      S->inner_its += c->it;
      S->inner_runs += c->graph_iters;
      S->inner_fb_runs += c->fb_iters;
      S->inner_fallbacks += c->fallback;
      if (c->status != ST_OK && S->inner_status == ST_OK) S->inner_status = c->status;
    }
  }
}

// ---- control of the flattened solve ---------------------------------------
// Every problem moves through its own sequence: the inner solve of Eq. (3),
// the initialisation of Algorithm 1 with its inner solve, then outer steps
// each with one inner solve. One loop iteration of the batch runs one CG
// iteration of every problem inside an inner solve; a problem whose inner
// solve ended takes its next GKB steps in the same iteration and starts its
// next inner solve, without waiting for the others.
enum { EV_AL = 1, EV_INIT = 2, EV_OUTER = 3 };
enum { K_INIT = 0, K_PRE, K_OUTER, K_START, K_POST, K_UPD };
struct Flat {
  GkbState** S;
  CgState** cg;
  int* incg;         // inside an inner solve (its prefix has run)
  int* event;        // what follows the current inner solve (EV_*)
  int* ended;        // Algorithm 1 has ended for this problem
  // this iteration's steps
  int *body, *fin, *al, *init, *outer, *start_outer, *start_cg, *pc;
  unsigned long long* counts;  // [0] iterations, [1..7] taken conditional sections
};
struct Handles {
  cudaGraphConditionalHandle h[4];
  int nh;
};
__global__ void __launch_bounds__(1024) kb_ctl(int op, Flat f, int n, int hard_outer, int hard_inner, Handles H) {
  int any[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    if (op == K_INIT) {
      f.incg[p] = 1;
      f.event[p] = EV_AL;
      f.ended[p] = 0;
      f.body[p] = f.fin[p] = f.al[p] = f.init[p] = f.outer[p] = f.start_outer[p] = 0;
      f.start_cg[p] = 1;
      f.pc[p] = 1;
    } else if (op == K_PRE) {
      const int in = f.incg[p] && !f.ended[p];
      const int dn = in && f.cg[p]->done;
      f.body[p] = in && !dn;
      f.fin[p] = dn;
      f.al[p] = dn && f.event[p] == EV_AL;
      f.init[p] = dn && f.event[p] == EV_INIT;
      f.outer[p] = dn && f.event[p] == EV_OUTER;
      if (dn) f.incg[p] = 0;
      f.start_outer[p] = 0;
      f.start_cg[p] = 0;
      any[0] |= dn;
      any[1] |= f.al[p];
      any[2] |= f.init[p];
      any[3] |= f.outer[p];
    } else if (op == K_OUTER) {
      // the while test of Algorithm 1 after alpha_1 (loop entry) or after
      // an outer step (its iteration bound included)
      int cont = 0;
      if (f.init[p] || f.outer[p]) {
        GkbState* S = f.S[p];
        if (f.init[p]) S->outer_runs = 0;
        else S->outer_runs += 1;
        cont = (S->stop || S->status != ST_OK) ? 0 : 1;
        if (f.outer[p] && S->outer_runs >= hard_outer) {
          cont = 0;
          S->stop = 1;
        }
        if (!cont) f.ended[p] = 1;
      }
      f.start_outer[p] = cont;
      any[0] |= cont;
    } else if (op == K_UPD) {
      // a mixed-form FP64 residual replacement is due in some CG iteration
      any[0] |= f.body[p] && f.cg[p]->update;
    } else if (op == K_START) {
      const int st = f.al[p] || f.start_outer[p];
      f.start_cg[p] = st;
      if (st) {
        f.incg[p] = 1;
        f.event[p] = f.al[p] ? EV_INIT : EV_OUTER;
      }
      f.pc[p] = f.body[p] || st;
      any[0] |= st;
    } else {
      // after a CG iteration: its loop bound; then the batch's loop condition
      if (f.body[p]) {
        CgState* g = f.cg[p];
        g->graph_iters += 1;
        if (g->graph_iters >= hard_inner && !g->done) {
          if (g->status == ST_OK) g->status = ST_INNER_NOT_CONVERGED;
          g->done = 1;
        }
      }
      any[0] |= !f.ended[p];
    }
  }
  for (int i = 0; i < 4; ++i) any[i] = __syncthreads_or(any[i]);
  if (threadIdx.x == 0) {
    if (op == K_POST) f.counts[0] += 1;
    if (op == K_PRE)
      for (int i = 0; i < 4; ++i) f.counts[1 + i] += any[i];
    if (op == K_OUTER) f.counts[5] += any[0];
    if (op == K_START) f.counts[6] += any[0];
    if (op == K_UPD) f.counts[7] += any[0];
    for (int i = 0; i < H.nh; ++i) cudaGraphSetConditional(H.h[i], any[i] ? 1u : 0u);
  }
}

#undef LS_RUN

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

bool lockstep_eligible(Solver* const* S, int count) {
  if (count < 2) return false;
  const gkb_options& o0 = S[0]->opt;
  for (int i = 0; i < count; ++i) {
    const Solver& s = *S[i];
    if (s.grid.dim != 2 || s.opt.inner != GKB_INNER_GMG_PCG || s.small_cg() || s.diag_n || s.mu64.p ||
        s.mu32.p || s.opt.viscous_form != GKB_VISC_LAPLACE || s.net)
      return false;
    if (s.opt.precision != o0.precision || s.opt.maxit != o0.maxit || s.opt.maxit_inner != o0.maxit_inner)
      return false;
    const int deg = (s.opt.precision == GKB_PREC_MIXED) ? s.gmg32.degree : s.gmg64.degree;
    const int deg0 = (o0.precision == GKB_PREC_MIXED) ? S[0]->gmg32.degree : S[0]->gmg64.degree;
    if (deg != deg0) return false;
  }
  return true;
}

struct Lockstep::Impl {
  std::vector<Solver*> S;
  int n = 0;
  bool mixed = false;
  DevBuf<int> state;                 // 11 arrays of n ints (Flat)
  DevBuf<unsigned long long> counts;
  DevBuf<GkbState*> sp;
  DevBuf<CgState*> cp;
  std::vector<DevBuf<unsigned char>> store;
  std::map<std::vector<unsigned>, const unsigned*> maps;
  // launches captured, by section (0 once, 1 every iteration, 2..8 the
  // conditional sections, each counted when taken) and kernel class
  long long cl[9][GKB_KC_COUNT] = {};
  int sect = 0;
  cudaGraphExec_t exec = nullptr;
  Flat F{};

  template <class J>
  const J* put(const std::vector<J>& v) {
    store.emplace_back();
    store.back().alloc(v.size() * sizeof(J));
    GKB_CUDA(cudaMemcpy(store.back().p, v.data(), v.size() * sizeof(J), cudaMemcpyHostToDevice));
    return (const J*)store.back().p;
  }
  const unsigned* put_map(const std::vector<unsigned>& m) {
    auto it = maps.find(m);
    if (it != maps.end()) return it->second;
    store.emplace_back();
    store.back().alloc(m.size() * sizeof(unsigned));
    GKB_CUDA(cudaMemcpy(store.back().p, m.data(), m.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    const unsigned* d = (const unsigned*)store.back().p;
    maps.emplace(m, d);
    return d;
  }

  // one batched launch over the problems `ps`: make(p, job) fills problem
  // p's job (head flags included) and returns its own launch grid
  template <class J, class Make>
  void launch(cudaStream_t st, int kc, const std::vector<int>& ps, dim3 block, Make make,
              void (*kern)(const J*, const unsigned*)) {
    std::vector<J> jobs;
    std::vector<unsigned> map;
    unsigned first = 0;
    for (int p : ps) {
      J j;
      memset(&j, 0, sizeof(J));
      const dim3 g = make(p, j);
      const unsigned nb = g.x * g.y * g.z;
      if (nb == 0) continue;
      j.h.first = first;
      j.h.gx = g.x;
      j.h.gy = g.y;
      j.h.gz = g.z;
      map.insert(map.end(), nb, (unsigned)jobs.size());
      jobs.push_back(j);
      first += nb;
    }
    if (jobs.empty()) return;
    const J* dj = put(jobs);
    const unsigned* dm = put_map(map);
    kern<<<first, block, 0, st>>>(dj, dm);
    GKB_CUDA(cudaGetLastError());
    cl[sect][kc] += 1;
  }

  void serial(cudaStream_t st, int kc, const int* G, int op, int arg, double tol2 = 0, double delta2 = 0) {
    std::vector<JSer> jobs(n);
    for (int p = 0; p < n; ++p) {
      Solver& s = *S[p];
      JSer& J = jobs[p];
      J.active = G ? G + p : nullptr;
      J.S = s.gkb_dev;
      J.cg = s.cg_dev;
      J.red = (const double*)((const char*)s.gkb_dev + offsetof(GkbState, red));
      J.tol2 = tol2;
      J.delta2 = delta2;
      J.rho2 = 0.0;
      J.maxit = s.opt.maxit_inner;
    }
    kb_serial<<<1, 256, 0, st>>>(put(jobs), n, op, arg);
    GKB_CUDA(cudaGetLastError());
    cl[sect][kc] += 1;
  }

  void ctl(cudaStream_t st, int op, std::initializer_list<cudaGraphConditionalHandle> hs = {}) {
    Handles H{};
    for (cudaGraphConditionalHandle h : hs) H.h[H.nh++] = h;
    kb_ctl<<<1, 1024, 0, st>>>(op, F, n, S[0]->opt.maxit + 2, S[0]->opt.maxit_inner + 2, H);
    GKB_CUDA(cudaGetLastError());
    cl[sect][GKB_KC_GKB] += 1;
  }

  std::vector<int> all() const {
    std::vector<int> v(n);
    for (int p = 0; p < n; ++p) v[p] = p;
    return v;
  }

  // ---- V-cycle in lock-step ------------------------------------------------
  template <typename T>
  Gmg<T>& gmg(int p) const;

  template <typename T>
  void smooth(cudaStream_t st, const std::vector<int>& ps, int d, const int* F,
              const std::function<const T*(int)>& bfun, const std::function<T*(int)>& xfun, bool x_zero) {
    const int deg = gmg<T>(ps[0]).degree;
    for (int k = 0; k < deg; ++k) {
      const bool first = (k == 0 && x_zero);
      if (!first) {
        launch<JTile<T>>(st, GKB_KC_RESIDUAL, ps, dim3(BX, BY), [&](int p, JTile<T>& j) {
          auto& V = gmg<T>(p).lev[d];
          j.h.active = F + p;
          j.L = V.L;
          j.x = xfun(p);
          j.b = bfun(p);
          j.y = V.r.p;
          return face_grid(V.L);
        }, kb_tile<T, 0, false>);
      }
      launch<JCheb<T>>(st, GKB_KC_SMOOTH, ps, dim3(BX, BY), [&](int p, JCheb<T>& j) {
        auto& V = gmg<T>(p).lev[d];
        j.h.active = F + p;
        j.L = V.L;
        j.r = first ? bfun(p) : V.r.p;
        j.x = xfun(p);
        j.d = V.d.p;
        j.ca = (T)V.ca[k];
        j.cb = (T)V.cb[k];
        j.x_zero = first ? 1 : 0;
        j.table = V.table.p;
        j.use2 = (!V.fold_in.empty() && V.table.p && cheb2_level(V.L)) ? 1 : 0;
        // the same rounded ca as the single-problem launch (Ops::cheb gets T)
        if (j.use2) j.fs = fold2_scaled<T>(V.fold_in.data(), (double)(T)V.ca[k]);
        return face_grid(V.L);
      }, kb_cheb<T>);
    }
  }

  // z = B r on the finest level of every problem (r0(p), z0(p) its arrays)
  template <typename T>
  void vcycle(cudaStream_t st, const int* F, const std::function<const T*(int)>& r0,
              const std::function<T*(int)>& z0) {
    int dmax = 0;
    for (int p = 0; p < n; ++p) dmax = std::max(dmax, (int)gmg<T>(p).lev.size() - 1);
    auto lb = [&](int d) { return std::function<const T*(int)>([&, d](int p) -> const T* {
      return d == 0 ? r0(p) : (const T*)gmg<T>(p).lev[d].b.p; }); };
    auto lx = [&](int d) { return std::function<T*(int)>([&, d](int p) -> T* {
      return d == 0 ? z0(p) : gmg<T>(p).lev[d].x.p; }); };
    auto deeper = [&](int d) {
      std::vector<int> v;
      for (int p = 0; p < n; ++p)
        if ((int)gmg<T>(p).lev.size() - 1 > d) v.push_back(p);
      return v;
    };
    for (int d = 0; d < dmax; ++d) {
      const std::vector<int> ps = deeper(d);
      if (ps.empty()) break;
      const auto bf = lb(d);
      const auto xf = lx(d);
      smooth<T>(st, ps, d, F, bf, xf, true);
      launch<JTile<T>>(st, GKB_KC_RESIDUAL, ps, dim3(BX, BY), [&](int p, JTile<T>& j) {
        auto& V = gmg<T>(p).lev[d];
        j.h.active = F + p;
        j.L = V.L;
        j.x = xf(p);
        j.b = bf(p);
        j.y = V.r.p;
        return face_grid(V.L);
      }, kb_tile<T, 0, false>);
      launch<JRestr<T>>(st, GKB_KC_RESTRICT, ps, dim3(BX, BY), [&](int p, JRestr<T>& j) {
        auto& G = gmg<T>(p);
        j.h.active = F + p;
        j.Lf = G.lev[d].L;
        j.Lc = G.lev[d + 1].L;
        j.rf = G.lev[d].r.p;
        j.bc = G.lev[d + 1].b.p;
        j.tmp = G.lev[d + 1].x.p;
        return face_grid(j.Lc);
      }, kb_restr_a<T>);
      launch<JRestr<T>>(st, GKB_KC_RESTRICT, ps, dim3(BX, BY), [&](int p, JRestr<T>& j) {
        auto& G = gmg<T>(p);
        j.h.active = F + p;
        j.Lf = G.lev[d].L;
        j.Lc = G.lev[d + 1].L;
        j.bc = G.lev[d + 1].b.p;
        j.tmp = G.lev[d + 1].x.p;
        return face_grid(j.Lc);
      }, kb_restr_b<T>);
    }
    // every problem's coarsest level in one launch (8 rows per block)
    launch<JCoarse<T>>(st, GKB_KC_COARSE, all(), dim3(256), [&](int p, JCoarse<T>& j) {
      auto& G = gmg<T>(p);
      const int lc = (int)G.lev.size() - 1;
      j.h.active = F + p;
      j.m = G.coarse_m;
      j.Minv = G.coarse_inv.p;
      j.idx = G.coarse_idx.p;
      j.b = lb(lc)(p);
      j.x = lx(lc)(p);
      return dim3((G.coarse_m + 7) / 8);
    }, kb_coarse<T>);
    for (int d = dmax - 1; d >= 0; --d) {
      const std::vector<int> ps = deeper(d);
      if (ps.empty()) continue;
      const auto bf = lb(d);
      const auto xf = lx(d);
      launch<JProl<T>>(st, GKB_KC_PROLONG, ps, dim3(BX, BY), [&](int p, JProl<T>& j) {
        auto& G = gmg<T>(p);
        j.h.active = F + p;
        j.Lf = G.lev[d].L;
        j.Lc = G.lev[d + 1].L;
        j.xc = G.lev[d + 1].x.p;
        j.xf = xf(p);
        return prolong2d_grid(j.Lc);
      }, kb_prolong<T>);
      smooth<T>(st, ps, d, F, bf, xf, false);
    }
  }

  template <typename T>
  void dot(cudaStream_t st, int kc, const int* F, const int* (*pred)(Solver&), long long (*len)(Solver&),
           const std::function<const T*(int)>& a, const std::function<const T*(int)>& b, int fin) {
    launch<JDot<T>>(st, kc, all(), dim3(RB), [&](int p, JDot<T>& j) {
      Solver& s = *S[p];
      j.h.active = F + p;
      j.h.pred = pred ? pred(s) : nullptr;
      j.len = len(s);
      j.a = a(p);
      j.b = b(p);
      j.red = s.red;
      j.fin = fin;
      j.st = s.cg_dev;
      return dim3((unsigned)blas_blocks(j.len));
    }, kb_dot<T>);
  }

  // the steps of the flattened solve (lockstep.cu, below)
  void cg_prefix(cudaStream_t st);   // [D] start the inner solves flagged start_cg
  void cg_body(cudaStream_t st, cudaStream_t sc);  // [A] first half of a CG iteration (flag body)
  void replace64(cudaStream_t su);   // the mixed form's FP64 reliable update
  void cg_precond(cudaStream_t st);  // [E] preconditioner, r.z, direction (flag pc)
  void cg_suffix(cudaStream_t st);   // [B] end the inner solves flagged fin
  void capture(cudaStream_t st, cudaStream_t sb, cudaStream_t sc);
  // "if (the handle's condition) body", the body captured on sc
  void if_node(cudaStream_t st, cudaStream_t sc, cudaGraphConditionalHandle h, int section,
               const std::function<void(cudaStream_t)>& body);
};

template <>
Gmg<double>& Lockstep::Impl::gmg<double>(int p) const { return S[p]->gmg64; }
template <>
Gmg<float>& Lockstep::Impl::gmg<float>(int p) const { return S[p]->gmg32; }

static unsigned lin_blocks_ls(long long n) {
  long long b = (n + 255) / 256;
  if (b > 1216) b = 1216;
  return (unsigned)(b < 1 ? 1 : b);
}
static dim3 cgrid_ls(const Lvl& L) { return dim3((L.n[0] + 31) / 32, (L.n[1] + 7) / 8, L.n[2]); }

// "if (condition) body": a conditional node on the graph stream st is
// capturing, whose body is captured on sc
void Lockstep::Impl::if_node(cudaStream_t st, cudaStream_t sc, cudaGraphConditionalHandle h, int section,
                             const std::function<void(cudaStream_t)>& body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  GKB_CUDA(cudaStreamGetCaptureInfo(st, &cst, nullptr, &g, &deps, nullptr, &nd));
  if (cst != cudaStreamCaptureStatusActive) throw Error{GKB_ERR_CUDA, "stream is not capturing"};
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  GKB_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  GKB_CUDA(cudaStreamBeginCaptureToGraph(sc, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const int saved = sect;
  sect = section;
  body(sc);
  sect = saved;
  GKB_CUDA(cudaStreamEndCapture(sc, &bodyg));
  GKB_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
}

static cudaGraphConditionalHandle new_handle(cudaStream_t st) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  GKB_CUDA(cudaStreamGetCaptureInfo(st, &cst, nullptr, &g, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive) throw Error{GKB_ERR_CUDA, "stream is not capturing"};
  cudaGraphConditionalHandle h;
  GKB_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  return h;
}

// [D] the part of an inner solve's start that comes before its first
// preconditioner application (Solver::capture_inner's prefix, up to the
// V-cycle), for the problems flagged start_cg
void Lockstep::Impl::cg_prefix(cudaStream_t st) {
  const std::vector<int> ps = all();
  const int* G = F.start_cg;
  const double tol2 = S[0]->opt.tol_inner * S[0]->opt.tol_inner;
  auto vlen = [](Solver& s) { return (long long)s.L64.nvel; };
  auto zero64 = [&](std::function<double*(Solver&)> y, bool cells) {
    launch<JVec>(st, GKB_KC_LAYOUT, ps, dim3(RB), [&](int p, JVec& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.len = cells ? s.L64.ncell : s.L64.nvel;
      j.y = y(s);
      j.op = 1;
      return dim3((unsigned)blas_blocks(j.len));
    }, kb_vec64);
  };
  if (mixed) {
    const double delta2 = S[0]->opt.mixed_rtol > 0 ? S[0]->opt.mixed_rtol * S[0]->opt.mixed_rtol : -1.0;
    serial(st, GKB_KC_GKB, G, P_CG_SETUP, 0, tol2, delta2);
    zero64([](Solver& s) { return s.x.p; }, false);
    launch<JVec32>(st, GKB_KC_LAYOUT, ps, dim3(RB), [&](int p, JVec32& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.len = s.L64.nvel;
      j.y = s.x32.p;
      return dim3((unsigned)blas_blocks(j.len));
    }, kb_zero32);
    dot<double>(st, GKB_KC_BLAS, G, nullptr, vlen, [&](int p) { return (const double*)S[p]->f.p; },
                [&](int p) { return (const double*)S[p]->f.p; }, FIN_CG_INIT);
    launch<JCvt>(st, GKB_KC_LAYOUT, ps, dim3(CB), [&](int p, JCvt& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.len = s.L64.nvel;
      j.r = s.f.p;
      j.o = s.cg32.r.p;
      return dim3(lin_blocks_ls(j.len));
    }, kb_cvt);
  } else {
    serial(st, GKB_KC_GKB, G, P_CG_SETUP, 0, tol2, 0.0);
    zero64([](Solver& s) { return s.x.p; }, false);
    launch<JVec>(st, GKB_KC_LAYOUT, ps, dim3(RB), [&](int p, JVec& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.len = s.L64.nvel;
      j.x = s.f.p;
      j.y = s.cg64.r.p;
      j.op = 2;
      return dim3((unsigned)blas_blocks(j.len));
    }, kb_vec64);
    dot<double>(st, GKB_KC_BLAS, G, nullptr, vlen, [&](int p) { return (const double*)S[p]->f.p; },
                [&](int p) { return (const double*)S[p]->f.p; }, FIN_CG_INIT);
  }
}

// the mixed form's FP64 residual replacement (x64 += x32, r64 = f - M x64,
// r32 = r64, r64.r64), gated per problem by its finaliser's update flag
void Lockstep::Impl::replace64(cudaStream_t su) {
  const std::vector<int> ps = all();
  const int* G = F.body;
  auto vlen = [](Solver& s) { return (long long)s.L64.nvel; };
  auto upd = [](Solver& s) { return (const int*)&s.cg_dev->update; };
  launch<JCvt>(su, GKB_KC_LAYOUT, ps, dim3(CB), [&](int p, JCvt& j) {
    Solver& s = *S[p];
    j.h.active = G + p;
    j.h.pred = upd(s);
    j.len = s.L64.nvel;
    j.x32 = s.x32.p;
    j.x64 = s.x.p;
    return dim3(lin_blocks_ls(j.len));
  }, kb_accum);
  launch<JTile<double>>(su, GKB_KC_RESIDUAL, ps, dim3(BX, BY), [&](int p, JTile<double>& j) {
    Solver& s = *S[p];
    j.h.active = G + p;
    j.h.pred = upd(s);
    j.L = s.L64;
    j.x = s.x.p;
    j.b = s.f.p;
    j.y = s.r64.p;
    return face_grid(s.L64);
  }, kb_tile<double, 0, false>);
  launch<JCvt>(su, GKB_KC_LAYOUT, ps, dim3(CB), [&](int p, JCvt& j) {
    Solver& s = *S[p];
    j.h.active = G + p;
    j.h.pred = upd(s);
    j.len = s.L64.nvel;
    j.r = s.r64.p;
    j.o = s.cg32.r.p;
    return dim3(lin_blocks_ls(j.len));
  }, kb_cvt);
  dot<double>(su, GKB_KC_BLAS, G, upd, vlen, [&](int p) { return (const double*)S[p]->r64.p; },
              [&](int p) { return (const double*)S[p]->r64.p; }, FIN_MX_RR64);
}

// [A] operator product, step and residual update of a CG iteration (and the
// mixed form's FP64 reliable update where its finaliser asks for one), for
// the problems flagged body
void Lockstep::Impl::cg_body(cudaStream_t st, cudaStream_t sc) {
  const std::vector<int> ps = all();
  const int* G = F.body;
  auto vlen = [](Solver& s) { return (long long)s.L64.nvel; };
  if (mixed) {
    launch<JTile<float>>(st, GKB_KC_APPLY, ps, dim3(BX, BY), [&](int p, JTile<float>& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.L = s.L32;
      j.x = s.cg32.p.p;
      j.y = s.cg32.q.p;
      j.red = s.red;
      j.fin = FIN_CG_PAP;
      j.st = s.cg_dev;
      return face_grid(s.L32);
    }, kb_tile<float, 1, true>);
    launch<JCgUpd<float>>(st, GKB_KC_BLAS, ps, dim3(RB), [&](int p, JCgUpd<float>& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.len = s.L64.nvel;
      j.x = s.x32.p;
      j.p = s.cg32.p.p;
      j.r = s.cg32.r.p;
      j.q = s.cg32.q.p;
      j.cg = s.cg_dev;
      j.red = s.red;
      j.st = s.cg_dev;
      j.fin = FIN_MX_RR;
      return dim3((unsigned)blas_blocks(j.len));
    }, kb_cg_update<float>);
    // the FP64 residual replacement under a conditional node: most
    // iterations need it in no problem
    const cudaGraphConditionalHandle hu = new_handle(st);
    ctl(st, K_UPD, {hu});
    if_node(st, sc, hu, 8, [&](cudaStream_t su) { replace64(su); });
  } else {
    launch<JTile<double>>(st, GKB_KC_APPLY, ps, dim3(BX, BY), [&](int p, JTile<double>& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.L = s.L64;
      j.x = s.cg64.p.p;
      j.y = s.cg64.q.p;
      j.red = s.red;
      j.fin = FIN_CG_PAP;
      j.st = s.cg_dev;
      return face_grid(s.L64);
    }, kb_tile<double, 1, true>);
    launch<JCgUpd<double>>(st, GKB_KC_BLAS, ps, dim3(RB), [&](int p, JCgUpd<double>& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.len = s.L64.nvel;
      j.x = s.x.p;
      j.p = s.cg64.p.p;
      j.r = s.cg64.r.p;
      j.q = s.cg64.q.p;
      j.cg = s.cg_dev;
      j.red = s.red;
      j.st = s.cg_dev;
      j.fin = FIN_CG_RR;
      return dim3((unsigned)blas_blocks(j.len));
    }, kb_cg_update<double>);
  }
}

// [E] z = B r, r.z and the new direction, for the problems flagged pc: those
// in a CG iteration (beta from r.z) and those starting a solve (first
// direction)
void Lockstep::Impl::cg_precond(cudaStream_t st) {
  const std::vector<int> ps = all();
  auto vlen = [](Solver& s) { return (long long)s.L64.nvel; };
  auto dirs = [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    for (int first = 1; first >= 0; --first) {
      const int* G = first ? F.start_cg : F.body;
      launch<JCgDir<T>>(st, GKB_KC_BLAS, ps, dim3(RB), [&](int p, JCgDir<T>& j) {
        Solver& s = *S[p];
        j.h.active = G + p;
        j.len = s.L64.nvel;
        if constexpr (sizeof(T) == 4) {
          j.p = s.cg32.p.p;
          j.z = s.cg32.z.p;
        } else {
          j.p = s.cg64.p.p;
          j.z = s.cg64.z.p;
        }
        j.cg = s.cg_dev;
        j.first = first;
        return dim3((unsigned)blas_blocks(j.len));
      }, kb_cg_dir<T>);
    }
  };
  if (mixed) {
    auto r32 = [&](int p) { return (const float*)S[p]->cg32.r.p; };
    auto z32c = [&](int p) { return (const float*)S[p]->cg32.z.p; };
    vcycle<float>(st, F.pc, r32, [&](int p) { return S[p]->cg32.z.p; });
    dot<float>(st, GKB_KC_BLAS, F.start_cg, nullptr, vlen, r32, z32c, FIN_CG_RZ0);
    dot<float>(st, GKB_KC_BLAS, F.body, nullptr, vlen, r32, z32c, FIN_CG_RZ);
    dirs((float*)nullptr);
  } else {
    auto r64 = [&](int p) { return (const double*)S[p]->cg64.r.p; };
    auto z64c = [&](int p) { return (const double*)S[p]->cg64.z.p; };
    vcycle<double>(st, F.pc, r64, [&](int p) { return S[p]->cg64.z.p; });
    dot<double>(st, GKB_KC_BLAS, F.start_cg, nullptr, vlen, r64, z64c, FIN_CG_RZ0);
    dot<double>(st, GKB_KC_BLAS, F.body, nullptr, vlen, r64, z64c, FIN_CG_RZ);
    dirs((double*)nullptr);
  }
}

// [B] the end of the inner solves flagged fin: FP64 accumulation of the
// mixed form's last FP32 correction, bookkeeping in the GKB state
void Lockstep::Impl::cg_suffix(cudaStream_t st) {
  const std::vector<int> ps = all();
  const int* G = F.fin;
  if (mixed) {
    launch<JCvt>(st, GKB_KC_LAYOUT, ps, dim3(CB), [&](int p, JCvt& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.len = s.L64.nvel;
      j.x32 = s.x32.p;
      j.x64 = s.x.p;
      return dim3(lin_blocks_ls(j.len));
    }, kb_accum);
  }
  serial(st, GKB_KC_GKB, G, P_NOTE_INNER, 0);
}

// Eq. (3), the initialisation and the while loop of Algorithm 1 with their
// inner solves, each problem on its own schedule (Solver::capture_core is the
// same sequence for one problem)
void Lockstep::Impl::capture(cudaStream_t st, cudaStream_t sb, cudaStream_t sc) {
  for (int p = 0; p < n; ++p)
    if (S[p]->opt.tol_inner != S[0]->opt.tol_inner || S[p]->opt.mixed_rtol != S[0]->opt.mixed_rtol)
      throw Error{GKB_ERR_INVALID_ARG, "lock-step batch: inner tolerances differ"};
  const std::vector<int> ps = all();
  auto gkb_launch = [&](cudaStream_t s_, const int* G, int op, int first,
                        const std::function<dim3(int, JGkb&)>& fill) {
    const bool lin = (op == G_GK3 || op == G_GK4V);
    launch<JGkb>(s_, GKB_KC_GKB, ps, lin ? dim3(CB) : dim3(32, 8), [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.L = s.L64;
      j.len = s.L64.nvel;
      j.op = op;
      j.first = first;
      j.st = s.gkb_dev;
      j.red = s.red;
      j.out = (double*)((char*)s.gkb_dev + offsetof(GkbState, red));
      return fill(p, j);
    }, kb_gkb);
  };
  auto apply64 = [&](cudaStream_t s_, const int* G, std::function<const double*(int)> xin) {
    launch<JTile<double>>(s_, GKB_KC_APPLY, ps, dim3(BX, BY), [&](int p, JTile<double>& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.L = s.L64;
      j.x = xin(p);
      j.y = s.t.p;
      j.red = s.red;
      j.fin = FIN_STORE;
      j.st = (double*)((char*)s.gkb_dev + offsetof(GkbState, red));
      return face_grid(s.L64);
    }, kb_tile<double, 1, true>);
  };
  auto vec64 = [&](cudaStream_t s_, const int* G, int op, std::function<const double*(Solver&)> x,
                   std::function<double*(Solver&)> y, bool cells, double a = 0, double b = 0) {
    launch<JVec>(s_, op == 0 ? GKB_KC_BLAS : GKB_KC_LAYOUT, ps, dim3(RB), [&](int p, JVec& j) {
      Solver& s = *S[p];
      j.h.active = G ? G + p : nullptr;
      j.len = cells ? s.L64.ncell : s.L64.nvel;
      j.a = a;
      j.b = b;
      j.x = x ? x(s) : nullptr;
      j.y = y(s);
      j.op = op;
      return dim3((unsigned)blas_blocks(j.len));
    }, kb_vec64);
  };
  sect = 0;
  // Eq. (3): f = g + gamma A N^-1 r, then the inner solve y0 = M^-1 f
  launch<JGrad>(st, GKB_KC_LAYOUT, ps, dim3(BX, BY), [&](int p, JGrad& j) {
    Solver& s = *S[p];
    j.L = s.L64;
    j.pc = s.ctmp.p;
    j.y = s.f.p;
    j.s = s.gamma / s.n_scale;
    return face_grid(s.L64);
  }, kb_grad);
  vec64(st, nullptr, 0, [](Solver& s) { return (const double*)s.wtmp.p; }, [](Solver& s) { return s.f.p; }, false,
        1.0, 1.0);
  ctl(st, K_INIT);
  cg_prefix(st);
  cg_precond(st);
  // the batch's loop: one CG iteration per problem in an inner solve; the
  // GKB steps of problems whose inner solve has ended
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphConditionalHandle hw = new_handle(st);
  ctl(st, K_POST, {hw});
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  GKB_CUDA(cudaStreamGetCaptureInfo(st, &cst, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hw;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wn;
  GKB_CUDA(cudaGraphAddNode(&wn, g, deps, nullptr, nd, &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  GKB_CUDA(cudaStreamBeginCaptureToGraph(sb, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  sect = 1;
  const cudaGraphConditionalHandle h_fin = new_handle(sb), h_al = new_handle(sb), h_init = new_handle(sb),
                                   h_outer = new_handle(sb), h_next = new_handle(sb), h_start = new_handle(sb);
  ctl(sb, K_PRE, {h_fin, h_al, h_init, h_outer});
  cg_body(sb, sc);
  if_node(sb, sc, h_fin, 2, [&](cudaStream_t s_) { cg_suffix(s_); });
  // after the inner solve of Eq. (3): b = r - A^T y0, beta_1, q_1, f = A q_1
  if_node(sb, sc, h_al, 3, [&](cudaStream_t s_) {
    const int* G = F.al;
    vec64(s_, G, 2, [](Solver& s) { return (const double*)s.x.p; }, [](Solver& s) { return s.y0.p; }, false);
    gkb_launch(s_, G, G_B, 0, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.ctmp.p;
      j.b = s.y0.p;
      j.c = s.bc.p;
      return cgrid_ls(s.L64);
    });
    serial(s_, GKB_KC_GKB, G, P_SCALAR, S_BETA1);
    gkb_launch(s_, G, G_Q1, 0, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.bc.p;
      j.c = s.q.p;
      return cgrid_ls(s.L64);
    });
    launch<JGrad>(s_, GKB_KC_LAYOUT, ps, dim3(BX, BY), [&](int p, JGrad& j) {
      Solver& s = *S[p];
      j.h.active = G + p;
      j.L = s.L64;
      j.pc = s.q.p;
      j.y = s.f.p;
      j.s = 1.0;
      return face_grid(s.L64);
    }, kb_grad);
    vec64(s_, G, 1, nullptr, [](Solver& s) { return s.u.p; }, false);
    vec64(s_, G, 1, nullptr, [](Solver& s) { return s.pp.p; }, true);
  });
  // after the initialisation's inner solve: alpha_1, v_1, zeta_1, d_1, p, u
  if_node(sb, sc, h_init, 4, [&](cudaStream_t s_) {
    const int* G = F.init;
    apply64(s_, G, [&](int p) { return (const double*)S[p]->x.p; });
    serial(s_, GKB_KC_GKB, G, P_SCALAR, S_ALPHA1);
    gkb_launch(s_, G, G_GK4V, 1, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.x.p;
      j.c = s.v.p;
      j.d = s.u.p;
      return dim3(lin_blocks_ls(s.L64.nvel));
    });
    gkb_launch(s_, G, G_GK4C, 1, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.gq.p;
      j.c = s.q.p;
      j.d = s.d.p;
      j.e = s.pp.p;
      return cgrid_ls(s.L64);
    });
  });
  // after an outer step's inner solve: w, alpha, the stopping rule, v, u, q, d, p
  if_node(sb, sc, h_outer, 5, [&](cudaStream_t s_) {
    const int* G = F.outer;
    gkb_launch(s_, G, G_GK3, 0, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.x.p;
      j.b = s.v.p;
      j.c = s.w.p;
      return dim3(lin_blocks_ls(s.L64.nvel));
    });
    apply64(s_, G, [&](int p) { return (const double*)S[p]->w.p; });
    serial(s_, GKB_KC_GKB, G, P_SCALAR, S_ALPHA);
    gkb_launch(s_, G, G_GK4V, 0, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.w.p;
      j.c = s.v.p;
      j.d = s.u.p;
      return dim3(lin_blocks_ls(s.L64.nvel));
    });
    gkb_launch(s_, G, G_GK4C, 0, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.gq.p;
      j.c = s.q.p;
      j.d = s.d.p;
      j.e = s.pp.p;
      return cgrid_ls(s.L64);
    });
  });
  // the while test of Algorithm 1; the next outer step's N-step and A q
  ctl(sb, K_OUTER, {h_next});
  if_node(sb, sc, h_next, 6, [&](cudaStream_t s_) {
    const int* G = F.start_outer;
    gkb_launch(s_, G, G_GK1, 0, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.v.p;
      j.b = s.q.p;
      j.c = s.gq.p;
      return cgrid_ls(s.L64);
    });
    serial(s_, GKB_KC_GKB, G, P_SCALAR, S_BETA);
    gkb_launch(s_, G, G_GK2, 0, [&](int p, JGkb& j) {
      Solver& s = *S[p];
      j.a = s.gq.p;
      j.c = s.f.p;
      return face_grid(s.L64);
    });
  });
  // inner solves starting in this iteration, then the preconditioner step
  ctl(sb, K_START, {h_start});
  if_node(sb, sc, h_start, 7, [&](cudaStream_t s_) { cg_prefix(s_); });
  cg_precond(sb);
  ctl(sb, K_POST, {hw});
  sect = 0;
  GKB_CUDA(cudaStreamEndCapture(sb, &bodyg));
  GKB_CUDA(cudaStreamUpdateCaptureDependencies(st, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
}

Lockstep::Lockstep(Solver* const* S, int count, cudaStream_t cap1, cudaStream_t cap2, cudaStream_t cap3) {
  I = new Impl();
  Impl& M = *I;
  M.S.assign(S, S + count);
  M.n = count;
  M.mixed = S[0]->opt.precision == GKB_PREC_MIXED;
  M.state.alloc(11 * (size_t)count);
  M.counts.alloc(9);
  std::vector<GkbState*> sp(count);
  std::vector<CgState*> cp(count);
  for (int p = 0; p < count; ++p) {
    sp[p] = S[p]->gkb_dev;
    cp[p] = S[p]->cg_dev;
  }
  M.sp.alloc(count);
  M.cp.alloc(count);
  GKB_CUDA(cudaMemcpy(M.sp.p, sp.data(), count * sizeof(GkbState*), cudaMemcpyHostToDevice));
  GKB_CUDA(cudaMemcpy(M.cp.p, cp.data(), count * sizeof(CgState*), cudaMemcpyHostToDevice));
  int* a = M.state.p;
  Flat& f = M.F;
  f.S = M.sp.p;
  f.cg = M.cp.p;
  int** slots[11] = {&f.incg, &f.event, &f.ended, &f.body, &f.fin, &f.al, &f.init, &f.outer, &f.start_outer,
                     &f.start_cg, &f.pc};
  for (int k = 0; k < 11; ++k) *slots[k] = a + (size_t)k * count;
  f.counts = M.counts.p;
  cudaGraph_t g = nullptr;
  try {
    GKB_CUDA(cudaGraphCreate(&g, 0));
    GKB_CUDA(cudaStreamBeginCaptureToGraph(cap1, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    M.capture(cap1, cap2, cap3);
    GKB_CUDA(cudaStreamEndCapture(cap1, &g));
    GKB_CUDA(cudaGraphInstantiate(&M.exec, g, 0));
  } catch (...) {
    for (cudaStream_t st : {cap3, cap2, cap1}) {
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(st, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
      }
    }
    (void)cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    delete I;
    I = nullptr;
    throw;
  }
  cudaGraphDestroy(g);
}

Lockstep::~Lockstep() {
  if (I && I->exec) cudaGraphExecDestroy(I->exec);
  delete I;
}

void Lockstep::launch(cudaStream_t s) {
  GKB_CUDA(cudaMemsetAsync(I->counts.p, 0, 9 * sizeof(unsigned long long), s));
  GKB_CUDA(cudaGraphLaunch(I->exec, s));
}

void Lockstep::launch_counts(cudaStream_t s, long long out[GKB_KC_COUNT]) {
  unsigned long long c[9] = {};
  GKB_CUDA(cudaMemcpyAsync(c, I->counts.p, sizeof(c), cudaMemcpyDeviceToHost, s));
  GKB_CUDA(cudaStreamSynchronize(s));
  // section 0 once; 1 every iteration; 2..8 when taken (c[1..7])
  for (int k = 0; k < GKB_KC_COUNT; ++k) {
    long long v = I->cl[0][k] + (long long)c[0] * I->cl[1][k];
    for (int t = 2; t < 9; ++t) v += (long long)c[t - 1] * I->cl[t][k];
    out[k] = v;
  }
}

}  // namespace gkb
