// solver.cuh - host-side objects: levels, multigrid hierarchy, CG, GKB driver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <functional>
#include <string>
#include <vector>

#include "../../include/gkb.h"
#include "common.cuh"
#include "ops.h"
#include "prof.h"
#include "reduce.cuh"
#include "state.cuh"

namespace gkb {

// thrown inside the library only; converted to a status at the ABI
struct Error {
  int code;
  std::string msg;
};

void check_cuda(cudaError_t e, const char* what);
#define GKB_CUDA(x) ::gkb::check_cuda((x), #x)

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      throw Error{GKB_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed"};
    }
    n = count;
    GKB_CUDA(cudaMemset(p, 0, count * sizeof(T)));
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

struct Unet;
struct UnetAct;

// Geometry of one level (both precisions share it; mu pointers differ).
Lvl make_level(int dim, const int n[3], double h, const int nat[6], double gc);

// Compact ordering of include/gkb.h <-> padded layout of level L, on stream
// s. Packing writes only the active entries (the caller clears the rest).
void pack_velocity(const Lvl& L, const double* compact, double* padded, cudaStream_t s);
void unpack_velocity(const Lvl& L, const double* padded, double* compact, cudaStream_t s);
void pack_cells(const Lvl& L, const double* compact, double* padded, cudaStream_t s);
void unpack_cells(const Lvl& L, const double* padded, double* compact, cudaStream_t s);

// Multigrid hierarchy in precision T for an all-Dirichlet grid.
template <typename T>
struct Gmg {
  struct Level {
    Lvl L;
    DevBuf<T> x, b, r, d, mu;
    DevBuf<T> nw;               // coarsened grad-div weights (diagonal N)
    DevBuf<T> em;               // node / edge viscosity table
    DevBuf<T> t2;               // second restriction scratch (3D coarse levels)
    DevBuf<T> sl;               // coarse slopes for the 3D prolongation
    DevBuf<T> table;            // patch class inverses (constant viscosity)
    std::vector<double> ca, cb; // Chebyshev coefficients per step
    std::vector<double> fold_in; // constant viscosity: the interior class stencils (host copy)
    double lam_max = 0;
  };
  std::vector<Level> lev;
  DevBuf<T> coarse_inv;
  DevBuf<int> coarse_idx;
  int coarse_m = 0;
  int degree = 2;
  double cheb_lo = 0.1;    // interval [cheb_lo * lam, cheb_hi * lam]
  double cheb_hi = 1.1;
  RedBuf red{};
  // learned coarse correction (optional): at level net_level the V-cycle
  // stops descending and applies the network instead
  Unet* net = nullptr;
  int net_level = -1;
  bool net_composite = false;  // network, then the ordinary cycle from its level
  UnetAct* net_act = nullptr;  // owned: this hierarchy's activation workspace
  DevBuf<float> net_img;
  DevBuf<double> net_nrm;
  DevBuf<T> net_q;             // M z of the network's correction
  // the coarse end of the V-cycle as one cluster kernel (2D, constant
  // viscosity): levels from tail_level on (the first whose longer side is at
  // most tail_side) run inside k_vtail; -1: off
  int tail_side = 0;
  int tail_level = -1;
  int tail_cs = 0;
  DevBuf<unsigned char> tail_buf;
  void attach_net(Unet* u, int level, bool composite, cudaStream_t s);
  void detach_net();
  Gmg() = default;
  Gmg(const Gmg&) = delete;
  Gmg& operator=(const Gmg&) = delete;
  ~Gmg();

  // levels[0] geometry given; mu0_cells: fine padded cell viscosity (T) or null
  void build(const Lvl& fine, const T* fine_mu, int coarse_max, int degree, const RedBuf& red,
             double* scratch_dev, cudaStream_t s);
  // z = B r on the finest level (one V-cycle); r, z fine padded arrays
  void vcycle(const T* r, T* z, cudaStream_t s, bool use_net = true);
  void smooth(int l, const T* b, T* x, bool x_zero, cudaStream_t s);
};

// plan and launch of the fused coarse end (tail.cu)
template <typename T>
void gmg_tail_setup(Gmg<T>& G, int side, cudaStream_t s);
template <typename T>
void gmg_tail_launch(const Gmg<T>& G, cudaStream_t s);

// An instantiated graph of a whole solve with the launch counts of its
// parts recorded at capture time: [0] once, [1] per outer iteration,
// [2] per inner solve, [3] per inner loop-body execution, [4] per
// execution of the body of the flexible form's fallback loop.
struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  long long cl[5][GKB_KC_COUNT] = {};
  long long cu[5][GKB_KC_COUNT] = {};
  void destroy() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  ~SolveGraph() { destroy(); }
};

// Conjugate gradients for M x = f in precision T on one level, optionally
// preconditioned by a V-cycle.
template <typename T>
struct Cg {
  Lvl L;
  Gmg<T>* pre = nullptr;
  bool flex = false;          // flexible CG (FCG(1) beta), for a nonlinear preconditioner
  double rho2 = 0;            // flexible CG: fallback contraction threshold squared
  DevBuf<T> r, z, p, q;
  CgState* st = nullptr;      // device
  CgState* host = nullptr;    // pinned mirror
  RedBuf red{};
  void init(const Lvl& L_, Gmg<T>* pre_, const RedBuf& red_, CgState* st_dev, CgState* st_host);
  // x = M^-1 f to relative tolerance tol (zero start); returns status
  int solve(const T* f, T* x, double tol, int maxit, cudaStream_t s, int* iters);
};

// Work space of the FGMRES(m) inner solver (fgmres.cu): the Krylov basis
// V (m + 1 vectors), the preconditioned vectors Z (m), and small scratch.
struct Fgmres {
  int m = 0;
  long long len = 0;
  DevBuf<double> V, Z, w, r, h, h2, y, part;
  DevBuf<double> state;    // device-resident form: its state, H, cs, sn, g
  DevBuf<double> vin, zt;  // the current basis vector and its V-cycle (fixed graph arguments)
  void init(long long len, int m);
};

struct Solver;
// x = M^-1 f by FGMRES(m) with one V-cycle as right preconditioner (FP64),
// host-sequenced
int fgmres_solve(Solver& S, const double* f, double* x, int* iters);
// the same inner solve (S.f -> S.x) captured on the graph stream s capturing,
// device-resident: its restart loop's body on sb, the Arnoldi loop's on sc;
// the outcome goes to S.cg_dev as a CG solve's would
void capture_fgmres(Solver& S, cudaStream_t s, cudaStream_t sb, cudaStream_t sc);
// "pre; while (cond) body; post" on the graph stream s is capturing (body on
// sb; pre ends by setting the condition, body with the kernel that updates it)
void capture_while(cudaStream_t s, cudaStream_t sb, int body_phase,
                   const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& pre,
                   const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& body,
                   const std::function<void(cudaStream_t)>& post);
// [W A; A^T 0][w; p] = [g; r] by FGMRES(restart) with GKB to pc_tol as the
// preconditioner; stops at ||b - K z||_2 <= tol ||b||_2 (compact I/O)
int solve_preconditioned(Solver& S, const double* g, const double* r, double tol, int restart, int maxit,
                         double pc_tol, int delay, double* w_out, double* p_out, int* iters);

struct Solver {
  gkb_options opt{};
  cudaStream_t stream = nullptr;
  std::string last_error;
  bool have_problem = false;
  gkb_grid grid{};
  double gamma = 0, n_scale = 0, mu0 = 1;
  bool enclosed = false;
  int64_t m = 0, ncell = 0;      // compact sizes
  Lvl L64{}, L32{};              // finest level, FP64 / FP32 views
  DevBuf<double> mu64;
  DevBuf<float> mu32;
  DevBuf<double> em64;           // node / edge viscosity table of the finest FP64 level
  // diagonal N (gkb_set_problem_n): N per cell (padded, FP64), the relative
  // grad-div weights n_scale / N in both precisions, sum N and sum 1/N
  DevBuf<double> nd64, nw64;
  DevBuf<float> nw32;
  double nsum = 0, ninvsum = 0;
  bool diag_n = false;

  // reduction scratch and device scalars
  DevBuf<double> red_partial;
  DevBuf<unsigned int> red_ticket;
  RedBuf red{};
  DevBuf<double> scal;           // small scratch for FIN_STORE results
  DevBuf<unsigned char> state_mem;
  CgState* cg_dev = nullptr;
  GkbState* gkb_dev = nullptr;
  CgState* cg_host = nullptr;    // pinned
  GkbState* gkb_host = nullptr;  // pinned

  // multigrid and CG in both precisions (only the ones in use are built)
  Gmg<double> gmg64;
  Gmg<float> gmg32;
  Fgmres fgm;                     // inner FGMRES work space
  Fgmres fgo;                     // outer FGMRES work space (saddle vectors)
  void cell_sum(const double* p, double* out);  // out[0] = sum over the in-domain cells
  Cg<double> cg64;
  Cg<float> cg32;

  // FP64 vectors of the GKB recurrence (padded)
  DevBuf<double> u, v, x, w, t, f, y0, wtmp;   // velocity
  DevBuf<double> q, d, pp, gq, bc, ctmp;       // cells
  DevBuf<double> r64;                          // mixed refinement residual
  DevBuf<float> f32, x32;                      // mixed refinement FP32 rhs / correction
  DevBuf<double> hist;                         // alpha, beta, zeta, est histories
  DevBuf<double> stage_m, stage_n;             // compact staging for host I/O
  gkb_stats_t stats{};
  Profiler prof;
  cudaStream_t cap1 = nullptr, cap2 = nullptr, cap3 = nullptr, cap4 = nullptr;  // private capture streams
  SolveGraph sgraph;              // whole solve as one graph (use_graph, no profiling)
  DevBuf<int> hist_inner;         // CG iterations of each inner solve
  int generation = 0;             // bumped by every set_problem
  Unet* net = nullptr;            // learned correction (GKB_INNER_FCG_UNET[_MG])
  bool learned_inner() const { return opt.inner == GKB_INNER_FCG_UNET || opt.inner == GKB_INNER_FCG_UNET_MG; }
  void set_net(Unet* u);
  double tuned_ms = 0;            // inner-solve time of the tuned configuration
  void build_inner();
  double time_inner_solve(int* its = nullptr);  // device ms of one inner solve (best of 3)
  void autotune_inner(bool var_mu, int weighted);
  void attach_net_levels();
  void refresh_net();
  void ensure_capture_streams();
  void build_solve_graph();
  // emitters shared by the graph capture and the host-sequenced path
  void al_rhs(cudaStream_t s);
  void capture_core(cudaStream_t s, cudaStream_t sb1, cudaStream_t sb2);
  void capture_inner(cudaStream_t s, cudaStream_t sb);
  void stage_in(const double* g, const double* r, const double* w0, const double* p0);
  void init_state(double tol, int delay);
  void run_core_host();
  int finish(double* w_out, double* p_out, const double* w0, const double* p0, bool graph_run);

  void set_problem(const gkb_grid* g, const double* viscosity, double mu0, double gamma, double n_scale,
                   const double* n_diag = nullptr);
  int solve(const double* g, const double* r, double tol, int delay, double* w_out, double* p_out,
            const double* w0, const double* p0);
  void apply(int op, const double* x, double* y);
  void boundary_rhs(int side, const double* normal_velocity, double* g, double* r);
  void precond(const double* r, double* z);
  int harvest(const double* f, int max_pairs, float* x_img, float* t_img, int* n_pairs);
  // inner solve in FP64 padded layout: x = M^-1 f; returns status
  int inner_solve(const double* f, double* x);
  bool small_cg() const;
  void launch_cg_block(const double* f, double* x, cudaStream_t s);
  int mixed_solve(const double* f, double* x, int* iters);
  ~Solver();
};

// Solve independent problems (one handle each) in one CUDA graph launch: the
// whole solve of every problem is one branch of the graph, branches run
// concurrently. The graph is captured at the first call for a list of
// handles and reused while none of them is re-set or destroyed.
int solve_batched(Solver** S, int count, const double* const* g, const double* const* r, double tol, int delay,
                  double* const* w, double* const* p);
void forget_batches(const Solver* s);

}  // namespace gkb
