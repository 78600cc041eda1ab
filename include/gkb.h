/*
 * gkb.h - C ABI of the GB300 generalized Golub-Kahan bidiagonalization (GKB)
 * solver for MAC-discretised Stokes saddle-point systems
 *
 *     [ W   A ] [w]   [g]
 *     [ A^T 0 ] [p] = [r]                                   (Sec. 2, Eq. (1))
 *
 * with W the viscous operator, A the integrated gradient, N = n_scale * I and
 * the augmented block M = W + gamma A N^-1 A^T (Eq. (2)). The solver applies
 * the augmented-Lagrangian transform (Eq. (3)), runs the Craig-variant GKB
 * recurrence (Algorithm 1) with the lower-bound stopping rule of Sec. 2.2
 * (Eq. (5)) and solves every inner system M x = f with conjugate gradients,
 * optionally preconditioned by one geometric-multigrid V-cycle.
 *
 * Discretisation (shared definition with the independent CPU oracle):
 *   uniform spacing h; velocity component c on the faces normal to axis c,
 *   pressure in the cells; finite-volume integrated form, so W has entries of
 *   size mu h^(d-2) and A entries +-h^(d-1): (A p)_f = h^(d-1)(p_plus - p_minus),
 *   and A^T is minus the integrated divergence. Tangential links use the mean
 *   viscosity of the in-domain cells around the node (2D) / edge (3D). Walls
 *   are no-slip mirror walls; natural sides are do-nothing outflow with
 *   half control volumes.
 *
 * Vector layout of every m-vector (velocity) and n-vector (pressure) crossing
 * this boundary ("compact ordering"): all active u faces, then all active v
 * faces (then w), each block row-major with x fastest; a face normal to axis
 * c is active unless it lies on a Dirichlet side normal to c. Pressure is the
 * cell array, x fastest. gkb_layout() reports m and n.
 *
 * Memory: every array pointer may be host memory (pageable or pinned) or
 * device memory of the handle's device; the library detects which with
 * cudaPointerGetAttributes. Host arrays are staged through the handle's
 * device buffers (copies included in the call). The caller owns all arrays
 * it passes; the handle owns all workspace.
 *
 * Errors: every entry point returns a status code (GKB_OK or GKB_ERR_*);
 * nothing is thrown across the ABI. gkb_last_error() returns a message for
 * the last failing call on that handle. A handle is not thread safe.
 *
 * Calls are synchronous with respect to the host: they return after the
 * work queued on the handle's stream has completed.
 */
#ifndef GKB_H
#define GKB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GKB_OK                       0
#define GKB_ERR_INVALID_ARG          1  /* bad size, pointer, option or state */
#define GKB_ERR_NOT_SPD              2  /* w^T M w <= 0 or p^T M p <= 0 met     */
#define GKB_ERR_NOT_CONVERGED        3  /* outer maxit reached (Algorithm 1)     */
#define GKB_ERR_INNER_NOT_CONVERGED  4  /* an inner solve hit maxit_inner        */
#define GKB_ERR_NAN                  5  /* NaN or Inf met in a norm              */
#define GKB_ERR_TIMEOUT              6  /* a bounded device wait ran out         */
#define GKB_ERR_CUDA                 7  /* CUDA runtime error                    */
#define GKB_ERR_OOM                  8  /* device allocation failed              */

/* ---- enumerations ------------------------------------------------------ */
#define GKB_BC_DIRICHLET  0   /* velocity given on that side (no-slip wall) */
#define GKB_BC_NATURAL    1   /* do-nothing outflow                         */

#define GKB_PREC_FP64     0   /* everything in FP64                          */
#define GKB_PREC_MIXED    1   /* inner CG, V-cycles and stencils in FP32 with
                                 the solution accumulated and the residual
                                 periodically recomputed in FP64; GKB vectors,
                                 alpha, beta, zeta and the estimator in FP64 */

#define GKB_INNER_CG      0   /* unpreconditioned CG                         */
#define GKB_INNER_GMG_PCG 1   /* CG + one GMG V-cycle (all-Dirichlet grids)  */
#define GKB_INNER_FCG_UNET 2  /* flexible CG (FCG(1)) + a V-cycle whose coarse
                                 correction at the level of unet_side cells is
                                 a U-Net (gkb_set_unet; 2D all-Dirichlet);
                                 without a network: the plain V-cycle         */
#define GKB_INNER_FGMRES  4   /* restarted flexible GMRES (fgmres_restart
                                 vectors) with one GMG V-cycle as right
                                 preconditioner, FP64, host-sequenced (the
                                 paper's other inner Krylov method, Sec. 3)  */
#define GKB_INNER_FCG_UNET_MG 3  /* flexible CG + a V-cycle that takes the
                                 network's correction at the level of
                                 unet_side cells as the starting guess of the
                                 ordinary cycle from that level down           */

#define GKB_VISC_LAPLACE 0
#define GKB_VISC_SYMGRAD 1

#define GKB_OP_W   0          /* y = W x                 (m -> m) */
#define GKB_OP_A   1          /* y = A x (gradient)      (n -> m) */
#define GKB_OP_AT  2          /* y = A^T x (-divergence) (m -> n) */
#define GKB_OP_M   3          /* y = M x                 (m -> m) */

/* kernel classes counted (and, with gkb_options.profile, timed) per solve */
#define GKB_KC_APPLY     0    /* operator products with fused dot (CG, alpha)   */
#define GKB_KC_RESIDUAL  1    /* r = b - M x                                    */
#define GKB_KC_SMOOTH    2    /* patch-Chebyshev smoothing step                 */
#define GKB_KC_RESTRICT  3    /* residual restriction P^T                       */
#define GKB_KC_PROLONG   4    /* prolongation and correction x += P e          */
#define GKB_KC_COARSE    5    /* dense coarsest-level solve                     */
#define GKB_KC_BLAS      6    /* dots and vector updates of CG                  */
#define GKB_KC_GKB       7    /* GKB recurrence kernels (Algorithm 1 steps)     */
#define GKB_KC_LAYOUT    8    /* packing, precision conversion, gradients       */
#define GKB_KC_UNET      9    /* U-Net convolutions, pooling, loss, optimiser   */
#define GKB_KC_COUNT     10

typedef struct gkb_ctx* gkb_handle;

/* Grid: dim = 2 or 3, n[] cells per axis (n[2] ignored in 2D), spacing h,
 * bc[] per side in the order x-low, x-high, y-low, y-high, z-low, z-high. */
typedef struct {
  int dim;
  int n[3];
  double h;
  int bc[6];
} gkb_grid;

typedef struct {
  int precision;          /* GKB_PREC_*                                        */
  int inner;              /* GKB_INNER_*                                       */
  double tol_inner;       /* inner stop: ||f - M x||_2 <= tol_inner ||f||_2    */
  int maxit;              /* outer (Algorithm 1 while-loop) iteration limit    */
  int maxit_inner;        /* CG iteration limit per inner solve                */
  int smoother_degree;    /* Chebyshev degree of pre- and post-smoothing       */
  int coarse_max;         /* coarsen while every side is even, halves to >= 2
                             cells and the longest side exceeds coarse_max
                             (coarse_max / 2, at least 4, in 3D)              */
  double mixed_rtol;      /* GKB_PREC_MIXED: the FP32 CG recomputes its
                             residual in FP64 whenever it has dropped by this
                             factor since the last recomputation, and checks
                             convergence on that FP64 residual; 0: ablation
                             without replacement (the FP32 recursion's own
                             convergence claim ends each inner solve, and the
                             FP32 iterate is converted to FP64 once), for
                             measuring the error floor that the replacement
                             removes                                           */
  int use_graph;          /* 1: run every inner CG solve as one CUDA graph whose
                             while loop is a device-side conditional node;
                             0: host-sequenced loop (always used when
                             profiling)                                        */
  int profile;            /* 1: time every kernel launch with CUDA events on
                             the stream and report per-class totals in
                             gkb_stats (adds event overhead between kernels)  */
  int kernel_variant;     /* stencil kernels' deep-interior fast paths (same
                             values bit for bit as the general paths, except
                             the 3D constant-viscosity smoother's folded
                             stencil, which agrees to rounding):
                             0: on in FP32, off in FP64 (measured fastest);
                             1: off everywhere; 2: on everywhere               */
  int unet_side;          /* GKB_INNER_FCG_UNET: longer side (cells) of the
                             multigrid level where the network replaces the
                             rest of the V-cycle; 0: the finest level (the
                             network alone)                                   */
  double fcg_rho;         /* GKB_INNER_FCG_UNET: an inner solve whose residual
                             after k >= 5 iterations exceeds fcg_rho^k ||f||
                             (or whose preconditioned vector is not finite)
                             continues as plain GMG-PCG from its iterate;
                             0 disables the switch                            */
  int fgmres_restart;     /* GKB_INNER_FGMRES: Krylov vectors per cycle (1..64) */
  double cheb_lo;         /* Chebyshev smoothing interval [cheb_lo, cheb_hi] x
                             lambda_max(C M) (power-iteration estimate);   */
  double cheb_hi;         /* 0 < cheb_lo < cheb_hi; defaults 0.1 and 1.1     */
  int autotune;           /* 1: gkb_set_problem searches smoother_degree (1..3),
                             kernel_variant (0..2), coarse_max (8, 16, 32) and
                             cheb_lo (0.05, 0.1, 0.2, 0.3), one after another,
                             then tail_side (0, 64; with 64, coarse_max
                             again), for the fastest inner solve (device
                             time of one GMG-PCG solve to tol_inner, best of
                             three; within 2 % of each other, the candidate
                             with fewer iterations) and keeps it; results
                             are cached per device, grid, viscosity kind,
                             precision, inner solver and gamma decade in the
                             process and, when the environment variable
                             GKB_TUNE_CACHE names a file, in that file (read
                             once, appended). gkb_get_options returns the
                             choice. Multigrid inner solvers only.           */
  void* stream;           /* cudaStream_t to run on (NULL: legacy stream)     */
  int viscous_form;       /* GKB_VISC_LAPLACE (default): W is the component-
                             wise -div(mu grad u_c); GKB_VISC_SYMGRAD: W is
                             -div(2 mu eps(u)), eps(u) = (grad u + grad u^T)
                             / 2, coupling the components through the
                             node (2D) / edge (3D) viscosities; needs
                             Dirichlet velocity on every side                 */
  int batch_lockstep;     /* gkb_solve_batched, read from hs[0]: 0 (default)
                             captures every problem as one branch of the
                             batch's graph; 1 runs a batch that qualifies
                             (2D, GMG-PCG, Laplacian form, constant
                             viscosity per problem, N = n I, one precision,
                             smoother degree and iteration limits) in lock
                             step: each step one kernel launch over all
                             problems; other batches keep the branches     */
  int tail_side;          /* 2D constant viscosity, multigrid inner solvers:
                             the levels from the first one whose longer side
                             is at most tail_side down to the coarsest run
                             as one thread-block-cluster kernel (smoothing,
                             residuals, transfers and the dense coarse solve
                             with cluster barriers between the steps; the same
                             values as separate launches); 0 (default): off.
                             The autotuner tries 64 (on a GB300 it measured
                             slower than separate launches: each fused step
                             still pays its memory round trips, plus the
                             barrier, on 16 SMs).                           */
} gkb_options;

typedef struct {
  int status;                 /* status of the last gkb_solve                */
  int outer_iterations;       /* while-loop iterations of Algorithm 1        */
  int inner_solves;           /* inner M-solves (AL transform + init + loop) */
  int64_t inner_iterations;   /* total CG iterations over all inner solves   */
  double estimate;            /* final lower-bound estimate (Eq. (5))        */
  double setup_seconds;       /* gkb_set_problem wall time                   */
  double solve_seconds;       /* last gkb_solve wall time                    */
  int levels;                 /* multigrid levels (0 without GMG)            */
  int inner_fallbacks;        /* flexible inner solves that switched to GMG-PCG */
  double tuned_inner_ms;      /* autotune: inner-solve device time of the choice (0 if not tuned) */
  int64_t kernel_launches[GKB_KC_COUNT];  /* launches per class, last solve  */
  int64_t kernel_units[GKB_KC_COUNT];     /* work per class: velocity unknowns
                                             of the launch's level summed over
                                             launches (vector elements for
                                             BLAS, rows for the coarse solve) */
  double kernel_ms[GKB_KC_COUNT];         /* summed kernel time per class (ms)
                                             when profiling, else 0          */
  int64_t kernel_top_launches[GKB_KC_COUNT]; /* profiling: the class's timed
                                             launches of its largest work per
                                             launch (the finest level)       */
  int64_t kernel_top_units[GKB_KC_COUNT]; /* that work per launch            */
  double kernel_top_ms[GKB_KC_COUNT];     /* their summed kernel time (ms)   */
} gkb_stats_t;

/* Fill *opt with defaults: FP64, GMG-PCG, tol_inner 1e-10, maxit 1000,
 * maxit_inner 2000, degree 2, coarse_max 8, mixed_rtol 1e-3, graphs on. */
int gkb_default_options(gkb_options* opt);

/* Create a handle on the current CUDA device. *out receives the handle.
 * Errors: INVALID_ARG (null pointers, bad option values), CUDA. */
int gkb_create(gkb_handle* out, const gkb_options* opt);

/* Define the operator (Eq. (1)-(2)): grid, cell viscosity, gamma and
 * N = n_scale * I (n_scale <= 0 selects h^dim, the pressure mass matrix).
 * viscosity: NULL for the constant mu0, else n values in compact pressure
 * ordering (host or device; copied). Builds the multigrid hierarchy and the
 * coarse solver. Errors: INVALID_ARG (sizes < 2, non-positive h, mu <= 0,
 * natural sides with GMG, odd sizes that cannot coarsen), OOM, CUDA. */
int gkb_set_problem(gkb_handle h, const gkb_grid* grid, const double* viscosity,
                    double mu0, double gamma, double n_scale);

/* gkb_set_problem with a diagonal N = diag(n_diag) (Sec. 3: N may be any
 * symmetric positive definite matrix; e.g. n_diag = h^dim / mu, the
 * viscosity-weighted pressure mass matrix, which approximates the Schur
 * complement A^T W^-1 A and cuts the outer iterations when mu varies).
 * n_diag: n values > 0 in compact pressure ordering (host or device;
 * copied). M = W + gamma A N^-1 A^T; the N-step of Algorithm 1 divides by
 * N cell by cell and beta is the N-norm; on an enclosed grid the N-step
 * vector is centred by its N-weighted mean. The multigrid levels carry the
 * weights h^dim / N (coarsened by averaging), and the operator runs on the
 * variable-viscosity kernels even for a constant mu0. Errors: those of
 * gkb_set_problem, and INVALID_ARG for a NULL, non-positive or non-finite
 * n_diag. */
int gkb_set_problem_n(gkb_handle h, const gkb_grid* grid, const double* viscosity,
                      double mu0, double gamma, const double* n_diag);

/* Sizes of the compact velocity (m) and pressure (n) vectors. */
int gkb_layout(gkb_handle h, int64_t* m, int64_t* n);

/* The handle's effective options (after autotuning, if any). */
int gkb_get_options(gkb_handle h, gkb_options* out);

/* Fold a Dirichlet normal velocity on one side into (g, r) in place: for
 * every boundary face b of that side with value u_b, the momentum row of the
 * active face linked to it gets kappa * u_b and the adjacent cell's
 * continuity row gets -A[b, cell] * u_b. normal_velocity holds one value per
 * boundary face of the side (x fastest over the remaining axes). g (m) and
 * r (n) are compact vectors. Errors: INVALID_ARG (side not Dirichlet). */
int gkb_boundary_rhs(gkb_handle h, int side, const double* normal_velocity,
                     double* g, double* r);

/* Solve Eq. (1) for (w, p): AL transform (Eq. (3)), Algorithm 1 with the
 * lower-bound rule of Eq. (5): with zeta_1..zeta_K known, stop when
 * sqrt(sum_{j=K-d}^{K} zeta_j^2 / sum_{j=1}^{K} zeta_j^2) <= tol, delay d.
 * g (m), r (n): right-hand side; w_out (m), p_out (n): solution. w0 / p0:
 * optional initial guess (NULL for zero), handled by defect correction. With
 * every side Dirichlet the returned pressure has zero mean.
 * Returns OK, NOT_CONVERGED (maxit reached; w_out/p_out hold the last
 * iterate), INNER_NOT_CONVERGED, NOT_SPD, NAN, or an argument/CUDA error. */
int gkb_solve(gkb_handle h, const double* g, const double* r, double tol, int delay,
              double* w_out, double* p_out, const double* w0, const double* p0);

/* GKB as a preconditioner (Sec. 3: the method serves as solver or as
 * preconditioner): restarted flexible GMRES (restart 1..64 vectors, at most
 * maxit iterations) on [W A; A^T 0][w; p] = [g; r], each iteration applying
 * the handle's GKB solve (AL transform and Algorithm 1 with its inner solver)
 * to tolerance pc_tol and delay `delay` as the preconditioner; stops when
 * ||b - K z||_2 <= tol ||b||_2. Same layouts and host/device rules as
 * gkb_solve; *iterations (may be NULL) receives the outer iterations. Returns
 * GKB_ERR_NOT_CONVERGED when maxit is reached first. Host-sequenced. */
int gkb_solve_preconditioned(gkb_handle h, const double* g, const double* r, double tol, int restart, int maxit,
                             double pc_tol, int delay, double* w_out, double* p_out, int* iterations);

/* Solve `count` independent problems in one CUDA graph launch (the batched
 * form; same method as gkb_solve for each, and the same result bit for bit).
 * hs[i] is a handle set up with gkb_set_problem or gkb_set_problem_n, all on
 * one device, with use_graph = 1 and profile = 0. g[i], r[i] (inputs) and
 * w_out[i], p_out[i] (outputs) are problem i's compact vectors, host or device
 * memory. By default every problem's whole solve, with its device-side loops,
 * is one branch of a single graph; the branches run concurrently (one
 * problem's latency-bound coarse levels overlap another's fine levels) and
 * each stops on its own estimate. With hs[0]'s batch_lockstep = 1 a batch
 * that qualifies runs in lock step instead (see gkb_options). The graph for a
 * list of handles is captured at its first call and reused while none of the
 * handles is re-set or destroyed. Runs on the stream of hs[0]. Returns OK when
 * every problem returned OK, else the first non-OK status; per-problem
 * statistics via gkb_stats(hs[i]). */
int gkb_solve_batched(gkb_handle* hs, int count, const double* const* g, const double* const* r,
                      double tol, int delay, double* const* w_out, double* const* p_out);

/* Statistics of the last solve. */
int gkb_stats(gkb_handle h, gkb_stats_t* out);

/* Per-step history of the last solve, host arrays of `capacity` entries
 * (any may be NULL): alpha_k, beta_k (beta_1 first), zeta_k, the estimate
 * after each loop step, and the CG iterations of each inner solve. Returns
 * the number of entries written for zeta (negative on error). */
int gkb_history(gkb_handle h, double* alpha, double* beta, double* zeta,
                double* estimate, int* inner_its, int capacity);

/* Apply one operator (GKB_OP_*) in FP64 to compact vectors, y = op(x). */
int gkb_apply(gkb_handle h, int op, const double* x, double* y);

/* Apply the inner preconditioner once, z = B r (one V-cycle, or identity for
 * plain CG), in the handle's precision, to compact m-vectors. */
int gkb_precond(gkb_handle h, const double* r, double* z);

/* Allocation-free operator product (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory, e.g. because their
 * device memory belongs to another allocator or a fixed arena, or because
 * cudaMalloc / cudaFree would synchronise a latency-critical loop).
 *
 * y = op(x) as in gkb_apply, for a constant-viscosity grid described by the
 * arguments (no handle). x and y are compact vectors in device memory (host
 * pointers are rejected). The call allocates nothing: its two padded work
 * arrays live in one file-scope device array of 2 * GKB_NOALLOC_MAX_ELEMS
 * doubles (16 MiB), which every GPU that loads the library holds until the
 * process exits. A grid whose padded velocity or cell array exceeds
 * GKB_NOALLOC_MAX_ELEMS doubles returns GKB_ERR_INVALID_ARG. The padded
 * layout rounds every x row of n_x + 1 faces up to a multiple of 32
 * elements, so the largest squares and cubes accepted are 711 x 711 cells
 * (2 * 712 * 736 doubles) and 63^3 cells (190 * 64 * 64 doubles); a 64^3
 * grid needs 193 * 65 * 96 = 1,204,320. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it for the
 * process: make that first call before any stream capture, and do not use
 * this entry point across a cudaDeviceReset. All calls share the array and
 * each call clears what it needs, so calls that overlap on the GPU
 * (different streams or threads) race and must be serialised by the
 * caller. Runs on `stream` (cudaStream_t, NULL: legacy stream) and waits
 * for that stream (cudaStreamSynchronize) before it returns.
 * Errors: INVALID_ARG (bad grid, sizes above the limit, host pointers),
 * CUDA. */
#define GKB_NOALLOC_MAX_ELEMS 1048576
int gkb_apply_noalloc(const gkb_grid* grid, double mu0, double gamma, double n_scale, int op,
                      const double* x, double* y, void* stream);

/* ---- learned preconditioner: a convolutional U-Net ---------------------
 * (The paper has no learned component; the network is the learned part of
 * the variable-viscosity workload.) Architecture: 3 levels with 16 / 32 / 32
 * channels and 3x3 convolutions with zero padding; encoder a1, a2 (full
 * resolution), 2x2 mean pooling, b1, b2, pooling, c1, c2; decoder: bilinear
 * doubling (pixel-centre aligned, edges clamped) of c2 concatenated with the
 * b2 output -> d1; doubling of d1 concatenated with the a2 output -> e1; a
 * linear 3x3 output convolution.
 * ReLU after every convolution but the last. Images are NHWC float arrays
 * in device memory with sides divisible by 4. Parameters: one flat float
 * vector, per layer the weights w[ky][kx][cin][cout] then the bias, layers
 * in the order a1 a2 b1 b2 c1 c2 d1 e1 out. Training uses FP32 kernels; the
 * inference path can run the convolutions on BF16 tensor cores with FP32
 * accumulation. */
typedef struct gkb_unet_ctx* gkb_unet;

/* Create a network with c_in inputs (1..16), c1 = 16 and c2 = 32 channels and
 * c_out outputs (1..3); He-normal weights from `seed`, zero biases. Returns
 * GKB_ERR_INVALID_ARG for other shapes. The handle is bound to the current
 * device and to `stream` (NULL: the legacy default stream). */
int gkb_unet_create(gkb_unet* out, int c_in, int c1, int c2, int c_out, unsigned long long seed, void* stream);
int gkb_unet_num_params(gkb_unet u, int64_t* n);
/* Copy the flat parameter vector out of / into the network (host or device). */
int gkb_unet_get_params(gkb_unet u, float* params);
int gkb_unet_set_params(gkb_unet u, const float* params);
/* y = N(x), x (n, h, w, c_in) and y (n, h, w, c_out) device arrays;
 * tensor_cores = 1 runs the convolutions in BF16 with FP32 accumulation. */
int gkb_unet_forward(gkb_unet u, const float* x, int n, int h, int w, float* y, int tensor_cores);
/* loss = (1/n) sum over the n samples of ||N(x) - target||^2 (FP32 forward), and its
 * gradient w.r.t. the parameters (kept for gkb_unet_adam_step; copied to grad
 * when not NULL, host or device). */
int gkb_unet_loss_grad(gkb_unet u, const float* x, const float* target, int n, int h, int w, double* loss,
                       float* grad);
/* One Adam update with the last gradient (bias-corrected moments). */
int gkb_unet_adam_step(gkb_unet u, float lr, float beta1, float beta2, float eps);
/* Train: `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, rate lr) on
 * minibatches of `batch` pairs drawn without replacement from the count pairs
 * (x_img (count, h, w, c_in), t_img (count, h, w, c_out), device arrays),
 * reshuffled by a generator seeded with `seed` on every pass; the loss of
 * each step goes to losses[step] when losses (host) is not NULL. The targets
 * are multiplied by the network's target scale. */
int gkb_unet_train(gkb_unet u, const float* x_img, const float* t_img, int64_t count, int h, int w, int batch,
                   int steps, float lr, unsigned long long seed, double* losses);
/* The network is trained on s * e^ and used as e^ = N(r^) / s (default 1).
 * A handle's captured solve graph keeps the s of its last gkb_set_unet or
 * gkb_set_problem; call gkb_set_unet again after changing it. */
int gkb_unet_set_target_scale(gkb_unet u, float s);
int gkb_unet_get_target_scale(gkb_unet u, float* s);
const char* gkb_unet_last_error(gkb_unet u);
int gkb_unet_destroy(gkb_unet u);

/* Attach the network to a handle (NULL detaches): with GKB_INNER_FCG_UNET the
 * V-cycle descends to the level with unet_side cells per side and applies
 * z = (||b|| / sqrt(nx ny)) / s * N(b^, log mu) there, with b^ = b sqrt(nx ny) / ||b||
 * on the west u / south v face of every cell (z = 0 for b = 0). The network must
 * outlive its use by the handle; its weights are read at each solve (a BF16
 * copy is refreshed when they changed). Rebuilds the handle's solve graph. */
int gkb_set_unet(gkb_handle h, gkb_unet u);

/* Training pairs from the handle's problem (2D, sides divisible by 4, FP64
 * with GKB_INNER_GMG_PCG): GMG-PCG on M x = f (f: compact velocity vector,
 * host or device) from x = 0 to tol_inner; for every iteration k before
 * convergence, x_img[k] (ny, nx, 3) = (r_k^ u, r_k^ v, log mu) and t_img[k]
 * (ny, nx, 2) = e_k^ with r_k^ = r_k sqrt(nx ny) / ||r_k||, e_k^ = (x* - x_k)
 * sqrt(nx ny) / ||r_k||, on the west u / south v face of each cell (wall faces
 * 0); only the leading iterations with ||r_k|| >= 1e4 ||r_final|| (the error
 * of x* - x_k is about their ratio); at most max_pairs, the count in *n_pairs
 * (0 unless the solve converged); images past the count are zero.
 * The images are device arrays. */
int gkb_harvest_pairs(gkb_handle h, const double* f, int max_pairs, float* x_img, float* t_img, int* n_pairs);

/* Message for the last failing call (never NULL). */
const char* gkb_last_error(gkb_handle h);

/* Release the handle and all its device memory. */
int gkb_destroy(gkb_handle h);

#ifdef __cplusplus
}
#endif

#endif /* GKB_H */
