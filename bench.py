#!/usr/bin/env python
"""GKB time-to-1e-8 benchmark on one GB300 (or N independent replicas).

Default workload (``--workload stokes2d``): the enclosed 2D Stokes cavity on
the unit square, MAC grid 1024 x 1024 (2,095,104 velocity and 1,048,576
pressure unknowns), forcing g ~ N(0,1) per velocity unknown from the fixed
seed, r = 0, viscosity 1, N = h^2 I, delay d = 5, outer tolerance 1e-8, inner
CG preconditioned by one GMG V-cycle to 1e-10, plain FP64. One step solves
the system for gamma = 10 and for gamma = 1000 (two handles set up before
timing; setup is reported separately). ``value`` is the device time of one
step (seconds, lower is better) with inputs resident in HBM; L2 is flushed
between steps.

Other workloads: ``stokes3d`` (256^3 cavity, gamma 100, mixed FP32/FP64),
``poiseuille`` (32 x 32 channel, gamma 100, plain CG to 1e-12, seeded
initial guess), ``batched2d`` (256 cavities of side 32*U{2..16} with
per-problem viscosity, gamma 100, mixed, one graph launch per step; value
in solves/s), ``varvisc2d`` (2048 x 2048 cavity with log-normal viscosity
from a Gaussian random field, gamma 100, mixed; inner flexible CG whose
V-cycle takes a U-Net correction at the 512 x 512 level; the network is
trained before timing on pairs harvested from GMG-PCG on 512 x 512
instances of the same family, and the GMG-PCG forms are timed beside it).

``--impl reference`` times the CPU oracle (sparse-LU inner solves) on the
host cores instead, on a reduced member of the same family, scaled by the
unknown ratio.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
BF16_FALLBACK_TFLOPS = 1900.0
FP64_PEAK_TFLOPS = 1.258   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (probe: 1.25)
FP32_PEAK_TFLOPS = 80.6    # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz

# algorithmic work per velocity unknown of the launch's level, per kernel
# class: (flops, element accesses). Flops count the arithmetic of the
# definitions with constant viscosity: a W row is 2d+2 flops (2d-1 additions
# of the neighbours, 2d x_f - sum as one fused multiply-add, the viscosity
# scale); the divergence of a cell (2d-1 additions) is shared by its d
# faces; the grad-div term adds 3 per face (difference of the two cell
# divergences, scale, sum); the residual subtracts from b (1 more). The
# smoother's count depends on the Chebyshev step (see SMOOTH_FLOPS).
# Accesses count the compulsory reads and writes of the vectors.
PER_UNIT = {
    2: {"apply": (10.5, 2.0), "residual": (11.5, 3.0), "smooth": (None, 4.5), "restrict": (1.5, 1.25),
        "prolong": (1.5, 2.25), "blas": (2.0, 3.0)},
    3: {"apply": (8.0 + 5.0 / 3.0 + 3.0, 2.0), "residual": (9.0 + 5.0 / 3.0 + 3.0, 3.0), "smooth": (None, 4.5),
        "restrict": (1.5, 1.125), "prolong": (1.5, 2.125), "blas": (2.0, 3.0)},
}


def smooth_flops(dim, degree):
    """Flops per velocity unknown of one Chebyshev step of the patch
    smoother, averaged over the 2 * degree steps of a V-cycle's pre- and
    post-smoothing. A face lies in 2 patches (2D vertex patches) or 4 (3D
    edge patches); its share of each is one row of the 4 x 4 patch inverse
    (4 products, 3 sums), and the patches' contributions are summed:
    z = 15 (2D) / 31 (3D) flops. The first pre-smoothing step (x = 0, no
    previous direction) adds ca * z; the first post-smoothing step also adds
    x + d; every other step forms d = ca z + cb d and x + d (4 more)."""
    z = 15.0 if dim == 2 else 31.0
    steps = [z + 1.0, z + 2.0] + [z + 4.0] * (2 * degree - 2)
    return sum(steps) / len(steps)


# U-Net forward: flops per pixel of the image (9 convolutions: 4 at full,
# 3 at half, 2 at quarter resolution) and unit count per pixel of one
# forward as the launch counters record it (pixels of each convolution and
# of the two image conversions)
UNET_FLOP_PER_PX = (2 * 9 * (3 * 16 + 16 * 16 + 48 * 16 + 16 * 2)
                    + 2 * 9 * (16 * 32 + 32 * 32 + 64 * 32) / 4 + 2 * 9 * (2 * 32 * 32) / 16)
UNET_UNITS_PER_PX = 4 + 3 / 4 + 2 / 16 + 2

# variable viscosity: the smoother also reads the per-patch inverses (10
# entries per node in 2D, per edge of each orientation in 3D), in elements
# per velocity unknown
VARMU_SMOOTH_EXTRA = {2: 5.0, 3: 10.0}

# DRAM traffic (bytes, read + write) of one finest-level launch of the
# dominant kernel, from ncu captures of the current kernels (cold cache, one
# launch each), keyed by (workload, form, kernel class)
TRAFFIC = {
    # 1024^2 FP64: first Chebyshev step (smooth, k_cheb2) and residual of a
    # V-cycle (reads exactly the algorithmic vectors; the writes include
    # lines left dirty before the launch)
    ("stokes2d", "fp64", "smooth"): 16.79e6 + 45.57e6,
    ("stokes2d", "fp64", "residual"): 33.72e6 + 34.30e6,
    # 2048^2 log-normal viscosity, mixed form
    ("varvisc2d", "mixed", "smooth"): 203.02e6 + 48.94e6,
    ("varvisc2d", "mixed", "residual"): 84.25e6 + 12.06e6,
    # 3D smoother captured at 160^3 (12.21 M unknowns, 96.32 MB), scaled by
    # the unknowns to 256^3 (50.14 M); the step's bytes are per unknown
    ("stokes3d", "mixed", "smooth"): (50.48e6 + 45.84e6) * (3 * 255 * 256 ** 2) / (3 * 159 * 160 ** 2),
}
# algorithmic bytes of the captured finest-level launch per velocity unknown,
# in elements (first Chebyshev step: r read, d and x written; residual: x, b
# read, r written)
CAPTURED_ELEMS = {"smooth": 3.0, "residual": 3.0}


def host_cpu():
    """Model of the host CPU and its core count (for the CPU baseline)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                if key.strip().lower() in ("model name", "cpu part") and model is None:
                    model = val.strip()
    except Exception:
        pass
    import platform
    # Arm cores report a part number instead of a model name
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    model = arm_parts.get(model, model)
    return {"model": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "host_cores": os.cpu_count()}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def measured_bf16_sustained():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured"
    except Exception:
        return BF16_FALLBACK_TFLOPS * 0.9, "fallback"


def train_network(gk, torch, wk, args):
    """The learned part's setup (untimed, reported): harvest (r^, e^) pairs
    with FP64 GMG-PCG on 512 x 512 instances of the workload's family (own
    seeds, so the timed instance is held out), then train the U-Net with
    Adam on the device. Returns the network and a report."""
    import numpy as np

    import workloads as W
    side = wk.unet_side
    t0 = time.perf_counter()
    cap = 40
    x_img = torch.zeros((args.train_pairs + cap, side, side, 3), dtype=torch.float32, device="cuda")
    t_img = torch.zeros((args.train_pairs + cap, side, side, 2), dtype=torch.float32, device="cuda")
    count, inst = 0, 0
    opt = gk.gkb_default_options()
    opt.precision = gk.GKB_PREC_FP64
    opt.inner = gk.GKB_INNER_GMG_PCG
    opt.tol_inner = 1e-10
    opt.maxit_inner = 5000
    opt.stream = torch.cuda.current_stream().cuda_stream
    h = gk.gkb_create(opt)
    try:
        while count < args.train_pairs and time.perf_counter() - t0 < args.harvest_seconds:
            pr = W.varvisc2d(side, seed_offset=1000 + 2 * inst)
            visc = np.ascontiguousarray(np.asarray(pr["mu"]).ravel(order="F"))
            gk.gkb_set_problem(h, gk.make_grid(pr["n"], pr["h"], pr["bc"]), visc, 1.0, 100.0, 0.0)
            k = gk.gkb_harvest_pairs(h, pr["g"], cap, x_img[count:], t_img[count:])
            count += k
            inst += 1
    finally:
        gk.gkb_destroy(h)
    count = min(count, args.train_pairs)
    torch.cuda.synchronize()
    harvest_s = time.perf_counter() - t0
    x_img, t_img = x_img[:count], t_img[:count]
    rms = float(t_img.pow(2).mean().sqrt())
    net = gk.gkb_unet_create(3, 16, 32, 2, 20010424, torch.cuda.current_stream().cuda_stream)
    gk.gkb_unet_set_target_scale(net, 1.0 / rms)
    t1 = time.perf_counter()
    losses = gk.gkb_unet_train(net, x_img, t_img, count, side, side, args.train_batch, args.train_steps,
                               args.train_lr, seed=7)
    train_s = time.perf_counter() - t1
    del x_img, t_img
    torch.cuda.empty_cache()
    head = float(np.mean(losses[:10])) if len(losses) else None
    tail = float(np.mean(losses[-10:])) if len(losses) else None
    return net, {"instances": inst, "pairs": count, "harvest_s": harvest_s, "train_s": train_s,
                 "steps": args.train_steps, "batch": args.train_batch, "lr": args.train_lr,
                 "target_rms": rms, "loss_first10": head, "loss_last10": tail,
                 "samples_per_s": args.train_steps * args.train_batch / train_s if train_s > 0 else None}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws, device="cuda"):
    """The largest value over the ranks of the initialised process group
    (the step time of a multi-GPU run is its slowest rank's)."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_seed_offset(rank):
    """Seed offset of rank `rank`'s batch: every rank solves its own problems
    (weak scaling: per-GPU work fixed, no data-path collective)."""
    return 6 + 1000 * int(rank)


# ---------------------------------------------------------------------------
# workloads: the problems one step solves
# ---------------------------------------------------------------------------

class Workload:
    """name, problems (dicts: n, h, bc, mu, gamma, g, r, optional w0/p0 and
    inflow), handle options, and how a step runs (sequential or batched)."""

    def __init__(self, args):
        import workloads as W
        self.name = args.workload
        self.batched = False
        self.inner = 1          # GMG-PCG
        self.tol_inner = args.tol_inner
        self.form = args.form
        self.learned = None     # "replace" / "composite": flexible CG with the network
        self.net = None
        self.kernel_variant = getattr(args, "kernel_variant", None)
        if self.name == "stokes2d":
            base = W.stokes2d(args.n)
            self.problems = [dict(base, gamma=float(gm)) for gm in args.gammas]
            self.dim = 2
            self.label = "%dx%d MAC Stokes cavity, gamma in {%s}" % (args.n, args.n, ",".join("%g" % g for g in args.gammas))
            self.sample = ("cavity", 256, args.gammas)
        elif self.name == "stokes3d":
            n = args.n if args.n != 1024 else 256
            base = W.stokes3d(n)
            self.problems = [dict(base, gamma=100.0)]
            self.dim = 3
            self.form = "mixed" if args.form_default else args.form
            self.label = "%d^3 MAC Stokes cavity, gamma 100" % n
            self.sample = ("cavity3d", 24, [100.0])
        elif self.name == "poiseuille":
            pr = W.poiseuille(32, shifted=False, guess=True)
            self.problems = [dict(pr, gamma=100.0)]
            self.dim = 2
            self.inner = 0
            self.tol_inner = 1e-12
            self.label = "32x32 MAC Poiseuille channel, gamma 100, inner CG 1e-12"
            self.sample = ("poiseuille", 32, [100.0])
        elif self.name == "varvisc2d":
            n = args.n if args.n != 1024 else 2048
            base = W.varvisc2d(n)
            self.problems = [dict(base, gamma=100.0)]
            self.dim = 2
            self.form = "mixed" if args.form_default else args.form
            self.learned = args.learned_form
            self.unet_side = args.unet_side
            self.label = "%dx%d MAC Stokes cavity, log-normal GRF viscosity, gamma 100" % (n, n)
            self.sample = ("varvisc", 128, [100.0])
        elif self.name == "batched2d":
            count = args.batch
            self.problems = [dict(pr, gamma=100.0)
                             for pr in W.batched2d(count=count, seed_offset=batch_seed_offset(getattr(args, "rank", 0)))]
            self.dim = 2
            self.batched = True
            self.form = "mixed" if args.form_default else args.form
            self.label = "%d MAC Stokes cavities, side 32*U{2..16}, gamma 100, one graph launch" % count
            self.sample = ("batched", 48, [100.0])
        else:
            raise ValueError(self.name)

    def metric(self):
        if self.batched:
            return "GKB batched solves/s to 1e-8 error (%s, %s GMG-PCG)" % (self.label, self.form_text())
        inner = "GMG-PCG" if self.inner == 1 else "CG"
        if self.learned:
            inner = "flexible CG, V-cycle with U-Net at %d^2 (%s form)" % (self.unet_side, self.learned)
        return "GKB time-to-1e-8 error (%s, %s %s)" % (self.label, self.form_text(), inner)

    def form_text(self):
        return "plain FP64" if self.form == "fp64" else "mixed FP32/FP64"

    def unit(self):
        return "solves/s" if self.batched else "s"


def make_handle(gk, torch, pr, wk, form, profile=0, learned=None, autotune=0, inner=None, variant=None,
                mixed_rtol=None, maxit=1000, lockstep=0):
    """variant: None, or a combination of "ndiag" (N = h^d / mu, the
    viscosity-weighted pressure mass matrix) and "symgrad" (the
    symmetric-gradient viscous operator). mixed_rtol: the mixed form's
    replacement trigger (0: the ablation without FP64 replacement).
    lockstep: the batch_lockstep option of gkb_solve_batched."""
    opt = gk.gkb_default_options()
    opt.autotune = autotune
    opt.batch_lockstep = lockstep
    if wk.kernel_variant is not None:
        opt.kernel_variant = wk.kernel_variant
    opt.precision = gk.GKB_PREC_FP64 if form == "fp64" else gk.GKB_PREC_MIXED
    opt.inner = wk.inner
    opt.tol_inner = wk.tol_inner
    opt.maxit = maxit
    if mixed_rtol is not None:
        opt.mixed_rtol = mixed_rtol
    opt.maxit_inner = 20000 if wk.inner == 0 else 5000
    opt.profile = profile
    opt.stream = torch.cuda.current_stream().cuda_stream
    if learned:
        opt.inner = gk.GKB_INNER_FCG_UNET if learned == "replace" else gk.GKB_INNER_FCG_UNET_MG
        opt.unet_side = wk.unet_side
    if inner is not None:
        opt.inner = inner
    if variant and "symgrad" in variant:
        opt.viscous_form = gk.GKB_VISC_SYMGRAD
    h = gk.gkb_create(opt)
    if learned:
        gk.gkb_set_unet(h, wk.net)
    mu = pr["mu"]
    import numpy as np
    if np.isscalar(mu):
        gk.gkb_set_problem(h, gk.make_grid(pr["n"], pr["h"], pr["bc"]), None, float(mu), pr["gamma"], 0.0)
    elif variant and "ndiag" in variant:
        visc = np.ascontiguousarray(np.asarray(mu).ravel(order="F"))
        nd = np.ascontiguousarray(pr["h"] ** len(pr["n"]) / visc)
        gk.gkb_set_problem_n(h, gk.make_grid(pr["n"], pr["h"], pr["bc"]), nd, visc, 1.0, pr["gamma"])
    else:
        visc = np.ascontiguousarray(np.asarray(mu).ravel(order="F"))
        gk.gkb_set_problem(h, gk.make_grid(pr["n"], pr["h"], pr["bc"]), visc, 1.0, pr["gamma"], 0.0)
    return h


class Bound:
    """Handles plus device/host buffers of a workload, and its step."""

    def __init__(self, gk, torch, wk, form, profile=0, subset=None, learned="default", autotune=0, inner=None,
                 variant=None, mixed_rtol=None, maxit=1000, concurrent=True, lockstep=0):
        import numpy as np
        self.gk, self.torch, self.wk = gk, torch, wk
        probs = wk.problems if subset is None else [wk.problems[i] for i in subset]
        self.probs = probs
        lf = wk.learned if learned == "default" else learned
        self.hs = [make_handle(gk, torch, pr, wk, form, profile, lf, autotune, inner, variant, mixed_rtol, maxit,
                               lockstep) for pr in probs]
        self.g, self.r, self.w, self.p, self.w0, self.p0 = [], [], [], [], [], []
        for h, pr in zip(self.hs, probs):
            m, n = gk.gkb_layout(h)
            if "inflow" in pr:   # Dirichlet inflow folded by the library
                g0 = np.zeros(m)
                r0 = np.zeros(n)
                gk.gkb_boundary_rhs(h, 0, np.ascontiguousarray(pr["inflow"]), g0, r0)
                pr = dict(pr, g=g0, r=r0)
            self.g.append(torch.tensor(pr["g"], device="cuda"))
            self.r.append(torch.tensor(pr["r"], device="cuda"))
            self.w.append(torch.empty(m, dtype=torch.float64, device="cuda"))
            self.p.append(torch.empty(n, dtype=torch.float64, device="cuda"))
            self.w0.append(torch.tensor(pr["w0"], device="cuda") if "w0" in pr else None)
            self.p0.append(torch.tensor(pr["p0"], device="cuda") if "p0" in pr else None)
        self.host = None
        # several problems without initial guesses: one gkb_solve_batched
        # call (a graph branch per problem, run concurrently), else one
        # gkb_solve per problem in turn
        self.batched = wk.batched or (concurrent and not profile and len(self.hs) > 1
                                      and all(x is None for x in self.w0 + self.p0))

    def step(self, args, host=False):
        gk = self.gk
        g, r, w, p = (self.host if host else (self.g, self.r, self.w, self.p))
        w0 = [None if x is None else (x.cpu().pin_memory() if host else x) for x in self.w0] if host else self.w0
        p0 = [None if x is None else (x.cpu().pin_memory() if host else x) for x in self.p0] if host else self.p0
        status = []
        if self.batched:
            status.append(gk.gkb_solve_batched(self.hs, g, r, args.tol, args.delay, w, p))
        else:
            for i, h in enumerate(self.hs):
                status.append(gk.gkb_solve(h, g[i], r[i], args.tol, args.delay, w[i], p[i], w0[i], p0[i]))
        return status

    def pin_host(self):
        t = self.torch
        self.host = ([x.cpu().pin_memory() for x in self.g], [x.cpu().pin_memory() for x in self.r],
                     [t.empty(x.numel(), dtype=t.float64).pin_memory() for x in self.w],
                     [t.empty(x.numel(), dtype=t.float64).pin_memory() for x in self.p])
        return sum(x.numel() for x in self.g + self.r) * 8, sum(x.numel() for x in self.w + self.p) * 8

    def stats(self):
        return [self.gk.gkb_stats(h) for h in self.hs]

    def destroy(self):
        for h in self.hs:
            self.gk.gkb_destroy(h)
        self.hs = []


def roofline(gk, torch, wk, args, form, hbm_peak, peak_kind):
    """Profiled step (CUDA events around every launch on its stream): the
    dominant kernel class's algorithmic throughput, summed over its launches
    and divided by their durations."""
    import numpy as np
    subset = list(range(min(len(wk.problems), 16))) if wk.batched else None
    B = Bound(gk, torch, wk, form, profile=1, subset=subset, autotune=args.autotune)
    n_profiled = len(B.hs)
    ms, units, launches = {}, {}, {}
    smooth_fl = 0.0    # smoother flops of all profiled handles (degree per handle)
    # the profiled solves are the capture range of a profiler started with
    # its collection off (ncu --profile-from-start off); no-ops otherwise
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    # the launches of each class at its largest work per launch (the finest
    # level): count, summed work, summed time, smoother flops
    top_n, top_u, top_ms, top_sfl = {}, {}, {}, 0.0
    for i, h in enumerate(B.hs):
        gk.gkb_solve(h, B.g[i], B.r[i], args.tol, args.delay, B.w[i], B.p[i], B.w0[i], B.p0[i])
        st = gk.gkb_stats(h)
        sfl = smooth_flops(wk.dim, gk.gkb_get_options(h).smoother_degree)
        for k in gk.KERNEL_CLASSES:
            ms[k] = ms.get(k, 0.0) + st["kernel_ms"][k]
            units[k] = units.get(k, 0) + st["kernel_units"][k]
            launches[k] = launches.get(k, 0) + st["kernel_launches"][k]
            top_n[k] = top_n.get(k, 0) + st["kernel_top_launches"][k]
            top_u[k] = top_u.get(k, 0) + st["kernel_top_launches"][k] * st["kernel_top_units"][k]
            top_ms[k] = top_ms.get(k, 0.0) + st["kernel_top_ms"][k]
        smooth_fl += st["kernel_units"]["smooth"] * sfl
        top_sfl += st["kernel_top_launches"]["smooth"] * st["kernel_top_units"]["smooth"] * sfl
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    B.destroy()
    table = PER_UNIT[wk.dim]
    cand = {k: v for k, v in ms.items() if k in table or (k == "unet" and wk.learned)}
    top = max(cand, key=cand.get)
    s = 8.0 if form == "fp64" else 4.0
    t = ms[top] * 1e-3
    total_ms = sum(ms.values())
    if top == "unet":
        # BF16 tensor-core convolutions: algorithmic flops of the forwards
        flops = units[top] / UNET_UNITS_PER_PX * UNET_FLOP_PER_PX
        bf16_peak, bf16_kind = measured_bf16_sustained()
        rl = {"bound": "tensor", "achieved": flops / t / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
              "peak_kind": "%s bf16_tflops_sustained (kernel timed inside a long step)" % bf16_kind}
        rl["frac"] = rl["achieved"] / rl["peak"]
        rl["kernel_class"] = top
        rl["launches"] = launches[top]
        rl["avg_launch_us"] = ms[top] * 1e3 / max(1, launches[top])
        rl["share_of_kernel_time"] = ms[top] / total_ms if total_ms else None
        rl["traffic"] = TRAFFIC.get((wk.name, form, top))
        rl["class_ms"] = {k: round(v, 3) for k, v in ms.items()}
        rl["profiled"] = "%d problem(s), profiled host-sequenced solve" % n_profiled
        return rl
    varmu = any(not np.isscalar(p["mu"]) for p in wk.problems)
    per_unit_bytes = table[top][1] + (VARMU_SMOOTH_EXTRA[wk.dim] if (top == "smooth" and varmu) else 0.0)
    flops = smooth_fl if top == "smooth" else units[top] * table[top][0]
    byts = units[top] * per_unit_bytes * s
    alu_peak = (FP64_PEAK_TFLOPS if form == "fp64" else FP32_PEAK_TFLOPS) * 1e12
    if form == "fp64" and flops / alu_peak > byts / (hbm_peak * 1e9):
        rl = {"bound": "alu", "achieved": flops / t / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
              "peak_kind": "FP64 FMA rate: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (probe measured 1.25)"}
    else:
        rl = {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
              "peak_kind": "%s hbm_gbs (copy, burst)" % peak_kind}
    rl["frac"] = rl["achieved"] / rl["peak"]
    rl["kernel_class"] = top
    rl["launches"] = launches[top]
    rl["avg_launch_us"] = ms[top] * 1e3 / max(1, launches[top])
    rl["share_of_kernel_time"] = ms[top] / total_ms if total_ms else None
    rl["traffic"] = TRAFFIC.get((wk.name, form, top))
    if rl["traffic"] is not None:
        m0 = wk.problems[0]["m"]
        extra = VARMU_SMOOTH_EXTRA[wk.dim] if (top == "smooth" and varmu) else 0.0
        rl["traffic_basis"] = "ncu DRAM read+write of one finest-level launch (cold cache)"
        rl["traffic_algorithmic"] = m0 * (CAPTURED_ELEMS.get(top, table[top][1]) + extra) * s
    rl["class_ms"] = {k: round(v, 3) for k, v in ms.items()}
    rl["profiled"] = "%d problem(s), profiled host-sequenced solve" % n_profiled
    rl["flops_per_unit"] = flops / max(1, units[top])
    # the same class restricted to its finest-level launches (the level the
    # ncu captures look at; the class figure above averages every level,
    # coarse launches included), where they are a real share of the class
    if top_n.get(top) and top_ms.get(top) and ms[top] and top_ms[top] >= 0.25 * ms[top]:
        tf = top_ms[top] * 1e-3
        if rl["bound"] == "alu":
            ach = (top_sfl if top == "smooth" else top_u[top] * table[top][0]) / tf / 1e12
        else:
            ach = top_u[top] * per_unit_bytes * s / tf / 1e9
        rl["finest_level"] = {"launches": top_n[top], "unknowns_per_launch": top_u[top] // top_n[top],
                              "avg_launch_us": top_ms[top] * 1e3 / top_n[top],
                              "share_of_class_time": top_ms[top] / ms[top] if ms[top] else None,
                              "achieved": ach, "frac": ach / rl["peak"]}
    return rl


def _oracle_worker(conn, pr, inner, tol_inner):
    """Spawned process holding the oracle's operators of one problem and its
    inner solver (for ``inner="direct"`` the sparse LU of M, the oracle's
    setup); each request runs Eq. (3), Algorithm 1 and Eq. (5) once."""
    try:
        import numpy as np

        from oracle import gkb as ogkb
        from oracle import mac
        t0 = time.perf_counter()
        grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
        ops = mac.assemble(grid, pr["mu"], pr["gamma"])
        g, r = pr.get("g"), pr.get("r")
        if "inflow" in pr:
            g, r = mac.dirichlet_rhs(grid, ops, {0: pr["inflow"]})
        t1 = time.perf_counter()
        solver = ogkb.InnerSolver(ops["M"], inner, tol_inner)
        t2 = time.perf_counter()
        conn.send(("setup", t1 - t0, t2 - t1))
        while True:
            msg = conn.recv()
            if msg[0] == "stop":
                break
            _, tol, delay, want = msg
            ts = time.perf_counter()
            res = ogkb.solve(grid, ops, g, r, tol=tol, delay=delay, w0=pr.get("w0"), p0=pr.get("p0"),
                             solver=solver)
            secs = time.perf_counter() - ts
            out = {"seconds": secs, "outer_iterations": res["iterations"], "converged": bool(res["converged"]),
                   "inner_iterations": int(sum(res["inner_iterations"]))}
            if want:
                out["w"], out["p"] = np.asarray(res["w"]), np.asarray(res["p"])
            conn.send(("ok", out))
    except Exception as e:  # reported to the parent, which raises
        conn.send(("error", "%s: %s" % (type(e).__name__, e)))
    finally:
        conn.close()


class OracleWorkers:
    """The oracle on the workload's own problems at full size: one spawned
    process per problem (SciPy's sparse LU and products are single-threaded,
    so the problems run side by side, one host core each). Each process
    assembles its operators and factorises M once (the oracle's setup, timed
    apart like the GPU handles' setup); a step solves every problem once and
    takes the wall time until the last one finishes."""

    def __init__(self, problems, inner="direct", tol_inner=1e-12):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")   # never fork a process that holds a CUDA context
        self.conns, self.procs = [], []
        for pr in problems:
            a, b = ctx.Pipe()
            proc = ctx.Process(target=_oracle_worker, args=(b, pr, inner, tol_inner), daemon=True)
            proc.start()
            b.close()
            self.conns.append(a)
            self.procs.append(proc)
        msgs = [self._recv(c) for c in self.conns]
        self.assemble_s = [m[1] for m in msgs]
        self.factor_s = [m[2] for m in msgs]

    @staticmethod
    def _recv(c):
        msg = c.recv()
        if msg[0] == "error":
            raise RuntimeError("oracle worker: " + msg[1])
        return msg

    def step(self, tol, delay, want_solution=False):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(("solve", tol, delay, want_solution))
        outs = [self._recv(c)[1] for c in self.conns]
        return time.perf_counter() - t0, outs

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=30)
        self.conns, self.procs = [], []


# workloads whose oracle runs at the benchmark's own size (the others run it
# on a reduced member of the family and scale by the unknown ratio)
FULL_SIZE_ORACLE = {"stokes2d": ("direct", 1e-12), "poiseuille": ("cg", 1e-12)}
# tolerance of the oracle solution the GPU result is compared with
TRUTH_TOL = 1e-13


def oracle_full(wk, args, truth=False):
    """Time one oracle step on the workload's problems at full size (after
    its setup), and with ``truth`` also solve them to TRUTH_TOL; returns
    (step seconds, per-problem outputs, truth outputs or None, setup dict)."""
    inner, tol_inner = FULL_SIZE_ORACLE[wk.name]
    W = OracleWorkers(wk.problems, inner, tol_inner)
    try:
        secs, outs = W.step(args.tol, args.delay)
        ref = W.step(TRUTH_TOL, args.delay, want_solution=True)[1] if truth else None
        setup = {"assemble_s": W.assemble_s, "factor_s": W.factor_s}
    finally:
        W.close()
    return secs, outs, ref, setup


def error_vs_oracle(wk, ws, ps, ref):
    """Relative M-norm error of each GPU velocity against the oracle
    solution, and the largest pressure difference relative to the largest
    oracle pressure."""
    import numpy as np

    from oracle import mac
    ev, ep = [], []
    for pr, w, p, rf in zip(wk.problems, ws, ps, ref):
        grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
        M = mac.assemble(grid, pr["mu"], pr["gamma"])["M"]
        e = w - rf["w"]
        ev.append(float(np.sqrt(max(float(e @ (M @ e)), 0.0) / float(rf["w"] @ (M @ rf["w"])))))
        ep.append(float(np.abs(p - rf["p"]).max() / np.abs(rf["p"]).max()))
    return {"velocity_m_norm_rel": ev, "pressure_max_rel": ep, "oracle_tol": TRUTH_TOL,
            "oracle_inner": FULL_SIZE_ORACLE[wk.name][0], "size": "full (the timed problems)"}


def cpu_oracle_sample(wk, args):
    """The oracle (sparse-LU inner solves; plain CG for the Poiseuille case)
    on a reduced member of the workload's family; returns (seconds measured,
    unknown-ratio scale to the full step, description)."""
    import numpy as np

    import workloads as W
    from oracle import gkb as ogkb
    from oracle import mac
    kind, n_s, gammas = wk.sample
    t0 = time.perf_counter()
    if kind == "cavity":
        pr = W.stokes2d(n_s)
        grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
        for gm in gammas:
            ogkb.solve(grid, mac.assemble(grid, 1.0, gm), pr["g"], pr["r"], tol=args.tol, delay=args.delay, inner="direct")
        full = sum(p["m"] + p["ncells"] for p in wk.problems)
        part = len(gammas) * (pr["m"] + pr["ncells"])
        desc = "%dx%d cavity, gamma %s" % (n_s, n_s, gammas)
    elif kind == "cavity3d":
        pr = W.stokes3d(n_s)
        grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
        ogkb.solve(grid, mac.assemble(grid, 1.0, gammas[0]), pr["g"], pr["r"], tol=args.tol, delay=args.delay, inner="direct")
        full = sum(p["m"] + p["ncells"] for p in wk.problems)
        part = pr["m"] + pr["ncells"]
        desc = "%d^3 cavity, gamma %g" % (n_s, gammas[0])
    elif kind == "varvisc":
        pr = W.varvisc2d(n_s)
        grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
        ogkb.solve(grid, mac.assemble(grid, pr["mu"], gammas[0]), pr["g"], pr["r"], tol=args.tol, delay=args.delay,
                   inner="direct")
        full = sum(p["m"] + p["ncells"] for p in wk.problems)
        part = pr["m"] + pr["ncells"]
        desc = "%dx%d log-normal viscosity cavity, gamma %g" % (n_s, n_s, gammas[0])
    elif kind == "poiseuille":
        pr = W.poiseuille(32, shifted=False, guess=True)
        grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
        ops = mac.assemble(grid, 1.0, 100.0)
        g, r = mac.dirichlet_rhs(grid, ops, {0: pr["inflow"]})
        ogkb.solve(grid, ops, g, r, tol=args.tol, delay=args.delay, inner="cg", tol_inner=1e-12,
                   w0=pr["w0"], p0=pr["p0"])
        full = part = 1
        desc = "the full 32x32 channel (plain CG inner solves)"
    else:  # batched: the n_s smallest problems solved one by one
        order = np.argsort([p["ncells"] for p in wk.problems])[:n_s]
        part = 0
        for i in order:
            pr = wk.problems[int(i)]
            grid = mac.MacGrid(pr["n"], pr["h"], pr["bc"])
            ogkb.solve(grid, mac.assemble(grid, pr["mu"], pr["gamma"]), pr["g"], pr["r"], tol=args.tol,
                       delay=args.delay, inner="direct")
            part += pr["m"] + pr["ncells"]
        full = sum(p["m"] + p["ncells"] for p in wk.problems)
        desc = "%d smallest of the %d cavities, one by one" % (n_s, len(wk.problems))
    secs = time.perf_counter() - t0
    return secs, full / part, desc


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    wk = Workload(args)
    times, one_core, extra = [], [], {}
    if wk.name in FULL_SIZE_ORACLE:
        # the oracle at the benchmark's own size: setup (assembly, LU of M)
        # once, then every step a whole solve of every problem
        t0 = time.perf_counter()
        inner, tol_inner = FULL_SIZE_ORACLE[wk.name]
        W = OracleWorkers(wk.problems, inner, tol_inner)
        extra["setup_s"] = time.perf_counter() - t0
        try:
            for i in range(args.warmup + args.steps):
                t, outs = W.step(args.tol, args.delay)
                if i >= args.warmup:
                    times.append(t)
                    one_core.append(sum(o["seconds"] for o in outs))
            extra["outer_iterations"] = [o["outer_iterations"] for o in outs]
            extra["converged"] = [o["converged"] for o in outs]
            extra["factor_s"] = W.factor_s
        finally:
            W.close()
        cores = len(wk.problems)
        sample = ("oracle GKB (Eq. (3), Algorithm 1, Eq. (5); %s inner solves) on the workload's own %d "
                  "problem(s) at full size, one process and host core per problem; every step a whole solve; "
                  "assembly and factorisation are setup" % (inner, len(wk.problems)))
    else:
        for i in range(args.warmup + args.steps):
            t, scale, desc = cpu_oracle_sample(wk, args)
            if i >= args.warmup:
                times.append(t * scale)
        cores = 1
        sample = "oracle GKB on %s, extrapolated: scaled x%.0f by the unknown ratio per step" % (desc, scale)
    step_s = statistics.mean(times)
    val = len(wk.problems) / step_s if wk.batched else step_s
    cpu = {"value": val, "unit": wk.unit(), "cores": cores, "kind": "oracle", "host": host_cpu(), "sample": sample}
    if one_core:
        cpu["one_core_s"] = statistics.mean(one_core)
    line = {
        "impl": "reference", "metric": wk.metric(), "value": val, "unit": wk.unit(), "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": bool(wk.batched), "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(args, wk), "cpu_baseline": cpu,
        "e2e": {"value": val, "unit": wk.unit(), "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    line.update(extra)
    print(json.dumps(line))
    return 0


def config(args, wk):
    sizes = sorted(set(tuple(p["n"]) for p in wk.problems))
    c = {"workload": wk.name, "problems": len(wk.problems), "tol": args.tol, "delay": args.delay,
         "tol_inner": wk.tol_inner, "form": wk.form, "inner": "gmg_pcg" if wk.inner == 1 else "cg",
         "n_scale": "h^d", "l2": "flushed between steps (1 GiB write)",
         "parallelism": "replicas" if args.gpus > 1 else "single",
         "autotune": bool(getattr(args, "autotune", 0) > 0)}
    if len(wk.problems) > 1:
        c["solve"] = ("problems solved concurrently (GPU: gkb_solve_batched, one graph launch with a branch per "
                      "problem; CPU oracle: one process per problem)"
                      if (wk.batched or all("w0" not in p and "p0" not in p for p in wk.problems))
                      else "problems solved in turn")
    if len(sizes) <= 4:
        c["grid"] = [list(s) for s in sizes]
    else:
        c["grid_sides"] = [int(s[0]) for s in sizes]
    c["gammas"] = sorted(set(p["gamma"] for p in wk.problems))
    return c


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2001_10424_gb300 as gk

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gk.build.build()
    gk.load()
    hbm_peak, peak_kind = measured_peaks()
    wk = Workload(args)
    if args.autotune < 0:
        args.autotune = 0 if wk.batched else 1
    training = None
    if wk.learned:
        wk.net, training = train_network(gk, torch, wk, args)
    t0 = time.perf_counter()
    B = Bound(gk, torch, wk, wk.form, autotune=args.autotune)
    setup_s = time.perf_counter() - t0
    tuned = []
    if args.autotune:
        for h in B.hs[:8]:
            o = gk.gkb_get_options(h)
            tuned.append({"smoother_degree": o.smoother_degree, "kernel_variant": o.kernel_variant,
                          "coarse_max": o.coarse_max, "cheb_lo": o.cheb_lo, "tail_side": o.tail_side})
    flush = torch.empty(1 << 28, dtype=torch.float32, device="cuda")  # 1 GiB > L2
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        B.step(args)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, launches_total, status = [], 0, None
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status = B.step(args)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        launches_total += sum(sum(st["kernel_launches"].values()) for st in B.stats())
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(step_ms), ws)
    stats = B.stats()
    outer = [st["outer_iterations"] for st in stats]
    inner = [st["inner_iterations"] for st in stats]
    # end to end through the C ABI with pinned host buffers (copies inside)
    h2d, d2h = B.pin_host()
    e2e = []
    for i in range(args.steps + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        B.step(args, host=True)
        t2 = time.perf_counter()
        if i > 0:
            e2e.append(t2 - t1)
    e2e_s = statistics.mean(e2e)
    finite = bool(all(np.isfinite(x.numpy()).all() for x in B.host[2]))
    gpu_w = [x.numpy().copy() for x in B.host[2]]   # this run's solutions, for the oracle comparison
    gpu_p = [x.numpy().copy() for x in B.host[3]]
    B.destroy()
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    rl = roofline(gk, torch, wk, args, wk.form, hbm_peak, peak_kind)
    forms = {}

    keep = wk.name in FULL_SIZE_ORACLE and not args.no_cpu_baseline
    form_solutions = {}

    def time_form(form, learned, autotune=None, inner=None, variant=None, mixed_rtol=None, maxit=1000, name=None,
                  concurrent=True, lockstep=0):
        autotune = args.autotune if autotune is None else autotune
        t_setup = time.perf_counter()
        B2 = Bound(gk, torch, wk, form, learned=learned, autotune=autotune, inner=inner, variant=variant,
                   mixed_rtol=mixed_rtol, maxit=maxit, concurrent=concurrent, lockstep=lockstep)
        t_setup = time.perf_counter() - t_setup
        for _ in range(2):
            B2.step(args)
        vals = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B2.step(args)
            e1.record(stream)
            e1.synchronize()
            vals.append(e0.elapsed_time(e1) / 1e3)
        st2 = B2.stats()
        out = {"s_per_step": statistics.mean(vals)}
        if wk.batched:
            out["solves_per_s"] = len(st2) / out["s_per_step"]
            out["inner_iterations_sum"] = sum(s["inner_iterations"] for s in st2)
            out["launches_per_step"] = sum(sum(s["kernel_launches"].values()) for s in st2)
        else:
            out.update({"outer_iterations": [s["outer_iterations"] for s in st2],
                        "inner_iterations": [s["inner_iterations"] for s in st2],
                        "inner_fallbacks": [s["inner_fallbacks"] for s in st2],
                        "status": [s["status"] for s in st2]})
        if len(st2) > 1:
            out["problems_concurrent"] = B2.batched
        if keep and name:
            torch.cuda.synchronize()
            form_solutions[name] = ([x.cpu().numpy() for x in B2.w], [x.cpu().numpy() for x in B2.p])
        if autotune:
            out["setup_s_with_tuning"] = t_setup
            out["tuned"] = []
            for h in B2.hs:
                o = gk.gkb_get_options(h)
                out["tuned"].append({"smoother_degree": o.smoother_degree, "kernel_variant": o.kernel_variant,
                                     "coarse_max": o.coarse_max, "cheb_lo": o.cheb_lo, "tail_side": o.tail_side})
        B2.destroy()
        return out

    if not args.no_forms and wk.batched:
        # the lock-step batched form on the same problems
        forms["lockstep"] = time_form(wk.form, None, lockstep=1)
    if not args.no_forms and not wk.batched and wk.inner == 1:
        head = {"s_per_step": ms / 1e3, "outer_iterations": outer, "inner_iterations": inner,
                "inner_fallbacks": [s["inner_fallbacks"] for s in stats]}
        if wk.learned:
            forms["learned_" + wk.learned + "_" + wk.form] = head
            other = "composite" if wk.learned == "replace" else "replace"
            forms["learned_" + other + "_" + wk.form] = time_form(wk.form, other)
            forms["gmg_pcg_" + wk.form] = time_form(wk.form, None)
            forms["gmg_pcg_fp64"] = time_form("fp64", None)
            # general N and the symmetric-gradient operator on the same instance
            forms["gmg_pcg_" + wk.form + "_ndiag"] = time_form(wk.form, None, variant="ndiag")
            forms["gmg_pcg_" + wk.form + "_symgrad"] = time_form(wk.form, None, variant="symgrad")
            forms["gmg_pcg_" + wk.form + "_symgrad_ndiag"] = time_form(wk.form, None, variant="symgrad+ndiag")
        else:
            other = "mixed" if wk.form == "fp64" else "fp64"
            forms[other] = time_form(other, None, name=other)
            forms[wk.form] = head
            # ablation: FP32 inner solves without the FP64 residual
            # replacement (their error floor; the outer loop may not reach tau)
            forms["mixed_no_replacement"] = time_form("mixed", None, mixed_rtol=0.0, maxit=100,
                                                      name="mixed_no_replacement")
            if wk.dim == 2:   # the paper's other inner Krylov method (FGMRES(30), device-resident)
                forms["fgmres_fp64"] = time_form("fp64", None, inner=gk.GKB_INNER_FGMRES, name="fgmres_fp64")
            if len(wk.problems) > 1:   # the same problems solved one after another
                forms[wk.form + "_sequential"] = time_form(wk.form, None, concurrent=False)
        if args.autotune:
            forms[wk.form + "_default_options"] = time_form(wk.form, None if not wk.learned else wk.learned, autotune=0,
                                                            name=wk.form + "_default_options")
        else:
            forms[wk.form + "_autotuned"] = time_form(wk.form, None if not wk.learned else wk.learned, autotune=1)
    cpu = None
    err = None
    if not args.no_cpu_baseline:
        if wk.name in FULL_SIZE_ORACLE:
            # the oracle on the timed problems themselves: one whole solve
            # (timed), then a solve to TRUTH_TOL that the GPU solutions are
            # compared with
            secs, outs, ref, setup = oracle_full(wk, args, truth=True)
            cpu = {"value": secs, "unit": wk.unit(), "cores": len(wk.problems), "host": host_cpu(), "kind": "oracle",
                   "one_core_s": sum(o["seconds"] for o in outs),
                   "outer_iterations": [o["outer_iterations"] for o in outs],
                   "setup_s": setup,
                   "sample": "oracle GKB (Eq. (3), Algorithm 1, Eq. (5); %s inner solves) on the timed problems at "
                             "full size, one process and host core per problem, one whole solve; assembly and "
                             "factorisation are setup" % FULL_SIZE_ORACLE[wk.name][0]}
            err = error_vs_oracle(wk, gpu_w, gpu_p, ref)
            for nm, (fw, fp) in form_solutions.items():
                e2 = error_vs_oracle(wk, fw, fp, ref)
                forms[nm]["error_vs_oracle"] = {"velocity_m_norm_rel": e2["velocity_m_norm_rel"],
                                                "pressure_max_rel": e2["pressure_max_rel"]}
        else:
            t_cpu, scale, desc = cpu_oracle_sample(wk, args)
            cpu_step = t_cpu * scale
            cpu = {"value": len(wk.problems) / cpu_step if wk.batched else cpu_step, "unit": wk.unit(), "cores": 1,
                   "host": host_cpu(),
                   "kind": "oracle",
                   "sample": "oracle GKB on %s: %.1f s measured, extrapolated x%.0f (unknown ratio) to the full "
                             "step" % (desc, t_cpu, scale)}
    step_s = ms / 1e3
    value = args.gpus * len(wk.problems) / step_s if wk.batched else step_s
    e2e_val = args.gpus * len(wk.problems) / e2e_s if wk.batched else e2e_s
    line = {
        "metric": wk.metric(), "value": value, "unit": wk.unit(), "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": bool(wk.batched), "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if wk.form == "fp64" else "f32+f64", "data": "synthetic",
        "config": config(args, wk),
        "e2e": {"value": e2e_val, "unit": wk.unit(), "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches_total),
        "roofline": rl, "cpu_baseline": cpu, "clocks": clk,
        "solves_per_s": args.gpus * len(wk.problems) / step_s,
        "inner_iterations_per_s": args.gpus * sum(inner) / step_s,
        "outer_iterations": outer if len(outer) <= 8 else {"min": min(outer), "max": max(outer), "sum": sum(outer)},
        "inner_iterations": inner if len(inner) <= 8 else {"min": min(inner), "max": max(inner), "sum": sum(inner)},
        "status": status, "setup_s": setup_s, "forms": forms, "finite_output": finite,
        "error_vs_oracle": err,
    }
    if tuned:
        line["tuned_options"] = tuned
    if training:
        line["training"] = training
    if wk.net is not None:
        gk.gkb_unet_destroy(wk.net)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_probe(args, local):
    """Short run for ncu captures: setup, then one V-cycle or one solve."""
    import torch

    import paper_2001_10424_gb300 as gk
    torch.cuda.set_device(local)
    gk.build.build()
    gk.load()
    wk = Workload(args)
    wk.problems = wk.problems[:1]
    if wk.learned:   # untrained weights: the launches are the same
        wk.net = gk.gkb_unet_create(3, 16, 32, 2, 1, torch.cuda.current_stream().cuda_stream)
    B = Bound(gk, torch, wk, wk.form)
    if args.probe == "precond":
        gk.gkb_precond(B.hs[0], B.g[0], B.w[0])
    else:
        B.step(args)
    torch.cuda.synchronize()
    B.destroy()
    print("probe done")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["stokes2d", "stokes3d", "poiseuille", "batched2d", "varvisc2d"],
                    default="stokes2d")
    ap.add_argument("--unet-side", type=int, default=512, help="varvisc2d: level (cells per side) of the network")
    ap.add_argument("--train-pairs", type=int, default=10000)
    ap.add_argument("--harvest-seconds", type=float, default=120.0)
    ap.add_argument("--train-steps", type=int, default=800)
    ap.add_argument("--train-batch", type=int, default=8)
    ap.add_argument("--train-lr", type=float, default=1e-3)
    ap.add_argument("--learned-form", choices=["replace", "composite"], default="replace")
    ap.add_argument("--kernel-variant", type=int, choices=[0, 1, 2], default=None,
                    help="deep-interior fast paths: 0 FP32 only (default), 1 none, 2 everywhere (untuned handles)")
    ap.add_argument("--form", choices=["fp64", "mixed"], default=None)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--gammas", type=str, default="10,1000")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--tol-inner", type=float, default=1e-10)
    ap.add_argument("--delay", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--autotune", type=int, default=-1,
                    help="1: the timed handles are autotuned at setup (reported in setup_s); 0: default options; "
                         "-1 (default): 1 for single problems, 0 for the batched form (its tuning times one "
                         "problem alone, which misjudges the coarse-level cost of 256 concurrent problems)")
    ap.add_argument("--probe", choices=["precond", "solve"], default=None,
                    help="profiling target: set up one handle and run one V-cycle or one solve")
    args = ap.parse_args()
    args.form_default = args.form is None
    if args.form is None:
        args.form = "fp64"
    args.gammas = [float(x) for x in args.gammas.split(",")]
    args.warmup = max(args.warmup, 0)
    ws, rank, local = dist_setup()
    args.rank = rank
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.probe:
        return run_probe(args, local)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
