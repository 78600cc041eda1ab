#!/usr/bin/env python
"""GKB time-to-1e-8 benchmark on one GB300 (or N independent replicas).

Workload (default): the enclosed 2D Stokes cavity on the unit square, MAC grid
1024 x 1024 (2,095,104 velocity and 1,048,576 pressure unknowns), forcing
g ~ N(0,1) per velocity unknown from the fixed seed, r = 0, viscosity 1,
N = h^2 I, delay d = 5, outer tolerance 1e-8, inner CG preconditioned by one
GMG V-cycle to 1e-10, plain FP64. One step solves the system for both
gamma = 10 and gamma = 1000 (two handles set up before timing; setup is
reported separately). ``value`` is the device time of one step (seconds,
lower is better) with inputs resident in HBM; L2 is flushed between steps.

``--impl reference`` times the CPU oracle (sparse-LU inner solves) on the
host cores instead, on a 256 x 256 member of the same family, extrapolated
by the unknown ratio.
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
FP64_PEAK_TFLOPS = 1.258   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (probe: 1.25)
FP32_PEAK_TFLOPS = 80.6    # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz

# algorithmic work per velocity unknown of the launch's level (2D), per class:
# (flops, element accesses); see DESIGN.md "Roofline accounting"
PER_UNIT_2D = {
    "apply": (14.0, 2.0),      # M x with fused dot: read x, write y
    "residual": (14.0, 3.0),   # r = b - M x: read x, b, write r
    "smooth": (20.0, 4.5),     # z = C r (2 patch rows), d, x updates; mean of first/other steps
    "restrict": (1.5, 1.25),   # read fine r, write coarse (1/4)
    "prolong": (1.5, 2.25),    # read coarse (1/4), read + write x
    "blas": (2.0, 3.0),        # per element: mean of dot / update kernels
}
PER_UNIT_3D = {
    "apply": (19.0, 2.0),
    "residual": (19.0, 3.0),
    "smooth": (35.0, 4.5),
    "restrict": (1.5, 1.125),
    "prolong": (1.5, 2.125),
    "blas": (2.0, 3.0),
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


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


def cpu_oracle_sample(n_sample, gammas, tol, delay):
    """Oracle (sparse-LU inner solves) on the n_sample^2 member of the family."""
    import workloads
    from oracle import gkb as ogkb
    from oracle import mac
    wl = workloads.stokes2d(n_sample)
    grid = mac.MacGrid(wl["n"], wl["h"], wl["bc"])
    t0 = time.perf_counter()
    iters = []
    for gm in gammas:
        ops = mac.assemble(grid, 1.0, gm)
        res = ogkb.solve(grid, ops, wl["g"], wl["r"], tol=tol, delay=delay, inner="direct")
        iters.append(res["iterations"])
    return time.perf_counter() - t0, iters


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    n_s = 256
    scale = (args.n / n_s) ** 2
    times = []
    for i in range(args.warmup + args.steps):
        t, _ = cpu_oracle_sample(n_s, args.gammas, args.tol, args.delay)
        if i >= args.warmup:
            times.append(t * scale)
    val = statistics.mean(times)
    line = {
        "impl": "reference", "metric": metric_name(args), "value": val, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config(args),
        "cpu_baseline": {"value": val, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": "oracle GKB with sparse-LU inner solves on the %dx%d cavity, gamma %s, "
                                   "time x%.0f (unknown ratio) per step" % (n_s, n_s, args.gammas, scale)},
        "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def metric_name(args):
    return "GKB time-to-1e-8 error (%dx%d MAC Stokes cavity, gamma in {%s}, %s GMG-PCG)" % (
        args.n, args.n, ",".join("%g" % g for g in args.gammas), "plain FP64" if args.form == "fp64" else "mixed FP32/FP64")


def config(args):
    return {"workload": "stokes2d_cavity_%d_gamma_%s" % (args.n, "_".join("%g" % g for g in args.gammas)),
            "grid": [args.n, args.n], "gammas": args.gammas, "tol": args.tol, "delay": args.delay,
            "tol_inner": args.tol_inner, "form": args.form, "inner": "gmg_pcg", "n_scale": "h^2",
            "l2": "flushed between steps (1 GiB write)", "parallelism": "replicas" if args.gpus > 1 else "single"}


def make_handles(gk, torch, wl, args, form, profile=0):
    hs = []
    for gm in args.gammas:
        opt = gk.gkb_default_options()
        opt.precision = gk.GKB_PREC_FP64 if form == "fp64" else gk.GKB_PREC_MIXED
        opt.inner = gk.GKB_INNER_GMG_PCG
        opt.tol_inner = args.tol_inner
        opt.maxit = 1000
        opt.maxit_inner = 5000
        opt.profile = profile
        opt.stream = torch.cuda.current_stream().cuda_stream
        h = gk.gkb_create(opt)
        gk.gkb_set_problem(h, gk.make_grid(wl["n"], wl["h"], wl["bc"]), None, 1.0, float(gm), 0.0)
        hs.append(h)
    return hs


def roofline(gk, torch, wl, args, form, hbm_peak, peak_kind):
    """Profiled step: the dominant kernel class's algorithmic throughput,
    summed over its launches and divided by their CUDA-event durations."""
    hs = make_handles(gk, torch, wl, args, form, profile=1)
    m, n = gk.gkb_layout(hs[0])
    g = torch.tensor(wl["g"], device="cuda")
    r = torch.tensor(wl["r"], device="cuda")
    w = torch.empty(m, dtype=torch.float64, device="cuda")
    p = torch.empty(n, dtype=torch.float64, device="cuda")
    ms, units, launches = {}, {}, {}
    for h in hs:
        gk.gkb_solve(h, g, r, args.tol, args.delay, w, p)
        st = gk.gkb_stats(h)
        for k in gk.KERNEL_CLASSES:
            ms[k] = ms.get(k, 0.0) + st["kernel_ms"][k]
            units[k] = units.get(k, 0) + st["kernel_units"][k]
            launches[k] = launches.get(k, 0) + st["kernel_launches"][k]
    for h in hs:
        gk.gkb_destroy(h)
    table = PER_UNIT_2D
    cand = {k: v for k, v in ms.items() if k in table}
    top = max(cand, key=cand.get)
    s = 8.0 if form == "fp64" else 4.0
    flops = units[top] * table[top][0]
    byts = units[top] * table[top][1] * s
    t = ms[top] * 1e-3
    alu_peak = (FP64_PEAK_TFLOPS if form == "fp64" else FP32_PEAK_TFLOPS) * 1e12
    alu_time, mem_time = flops / alu_peak, byts / (hbm_peak * 1e9)
    total_ms = sum(ms.values())
    if alu_time > mem_time:
        rl = {"bound": "alu", "achieved": flops / t / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
              "peak_kind": "FP64 FMA rate derived from SM count and clock (probe measured 1.25)"
              if form == "fp64" else "FP32 FMA rate derived from SM count and clock"}
    else:
        rl = {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
              "peak_kind": "%s hbm_gbs" % peak_kind}
    rl["frac"] = rl["achieved"] / rl["peak"]
    rl["kernel_class"] = top
    rl["launches"] = launches[top]
    rl["avg_launch_us"] = ms[top] * 1e3 / max(1, launches[top])
    rl["share_of_kernel_time"] = ms[top] / total_ms if total_ms else None
    rl["traffic"] = None
    rl["class_ms"] = {k: round(v, 3) for k, v in ms.items()}
    return rl


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2001_10424_gb300 as gk
    import workloads

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gk.build.build()
    gk.load()
    hbm_peak, peak_kind = measured_peaks()
    wl = workloads.stokes2d(args.n)
    t0 = time.perf_counter()
    hs = make_handles(gk, torch, wl, args, args.form)
    setup_s = time.perf_counter() - t0
    m, n = gk.gkb_layout(hs[0])
    g = torch.tensor(wl["g"], device="cuda")
    r = torch.tensor(wl["r"], device="cuda")
    w = torch.empty(m, dtype=torch.float64, device="cuda")
    p = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(1 << 28, dtype=torch.float32, device="cuda")  # 1 GiB > L2
    stream = torch.cuda.current_stream()

    def step():
        outer, inner, launches, status = [], [], 0, []
        for h in hs:
            rc = gk.gkb_solve(h, g, r, args.tol, args.delay, w, p)
            st = gk.gkb_stats(h)
            status.append(rc)
            outer.append(st["outer_iterations"])
            inner.append(st["inner_iterations"])
            launches += sum(st["kernel_launches"].values())
        return outer, inner, launches, status

    for _ in range(args.warmup):
        step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, launches_total, outer, inner, status = [], 0, None, None, None
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outer, inner, nl, status = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        launches_total += nl
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = statistics.mean(step_ms)
    if ws > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    # end to end through the C ABI with pinned host buffers
    gh = torch.tensor(wl["g"]).pin_memory()
    rh = torch.tensor(wl["r"]).pin_memory()
    wh = torch.empty(m, dtype=torch.float64).pin_memory()
    ph = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e = []
    for i in range(args.steps + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for h in hs:
            gk.gkb_solve(h, gh, rh, args.tol, args.delay, wh, ph)
        t2 = time.perf_counter()
        if i > 0:
            e2e.append(t2 - t1)
    e2e_s = statistics.mean(e2e)
    correct = bool(np.isfinite(wh.numpy()).all())
    for h in hs:
        gk.gkb_destroy(h)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0
    rl = roofline(gk, torch, wl, args, args.form, hbm_peak, peak_kind)
    rl["traffic"] = TRAFFIC.get((args.form, rl["kernel_class"]))
    forms = {}
    if not args.no_forms:
        other = "mixed" if args.form == "fp64" else "fp64"
        hs2 = make_handles(gk, torch, wl, args, other)
        for _ in range(2):
            for h in hs2:
                gk.gkb_solve(h, g, r, args.tol, args.delay, w, p)
        vals = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for h in hs2:
                gk.gkb_solve(h, g, r, args.tol, args.delay, w, p)
            e1.record(stream)
            e1.synchronize()
            vals.append(e0.elapsed_time(e1) / 1e3)
        its = [gk.gkb_stats(h)["outer_iterations"] for h in hs2]
        inn = [gk.gkb_stats(h)["inner_iterations"] for h in hs2]
        for h in hs2:
            gk.gkb_destroy(h)
        forms[other] = {"s_per_step": statistics.mean(vals), "outer_iterations": its, "inner_iterations": inn}
        forms[args.form] = {"s_per_step": ms / 1e3, "outer_iterations": outer, "inner_iterations": inner}
    cpu = None
    if not args.no_cpu_baseline:
        n_s = 256
        t_cpu, _ = cpu_oracle_sample(n_s, args.gammas, args.tol, args.delay)
        scale = (args.n / n_s) ** 2
        cpu = {"value": t_cpu * scale, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": "oracle GKB (sparse-LU inner solves) on the %dx%d cavity, gamma %s, %.1f s measured, "
                         "x%.0f (unknown ratio) to the %dx%d step" % (n_s, n_s, args.gammas, t_cpu, scale, args.n, args.n)}
    value = ms / 1e3
    line = {
        "metric": metric_name(args), "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(args),
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(len(args.gammas) * (m + n) * 8),
                "d2h_bytes_per_step": int(len(args.gammas) * (m + n) * 8)},
        "gpu_launches": int(launches_total),
        "roofline": rl, "cpu_baseline": cpu, "clocks": clk,
        "solves_per_s": args.gpus * len(args.gammas) / value,
        "inner_iterations_per_s": args.gpus * sum(inner) / value,
        "outer_iterations": outer, "inner_iterations": inner, "status": status,
        "setup_s": setup_s, "forms": forms, "finite_output": correct,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_probe(args, local):
    """Short run for ncu captures: setup, then one V-cycle or one solve."""
    import torch

    import paper_2001_10424_gb300 as gk
    import workloads
    torch.cuda.set_device(local)
    gk.build.build()
    gk.load()
    wl = workloads.stokes2d(args.n)
    args.gammas = args.gammas[:1]
    h = make_handles(gk, torch, wl, args, args.form)[0]
    m, n = gk.gkb_layout(h)
    g = torch.tensor(wl["g"], device="cuda")
    r = torch.tensor(wl["r"], device="cuda")
    w = torch.empty(m, dtype=torch.float64, device="cuda")
    p = torch.empty(n, dtype=torch.float64, device="cuda")
    if args.probe == "precond":
        gk.gkb_precond(h, g, w)
    else:
        gk.gkb_solve(h, g, r, args.tol, args.delay, w, p)
    torch.cuda.synchronize()
    gk.gkb_destroy(h)
    print("probe done")
    return 0


# per-launch DRAM traffic (bytes) of the dominant kernel from ncu captures,
# keyed by (form, kernel class); summarised under profiles/
TRAFFIC = {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--gammas", type=str, default="10,1000")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--tol-inner", type=float, default=1e-10)
    ap.add_argument("--delay", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--probe", choices=["precond", "solve"], default=None,
                    help="profiling target: set up one handle (first gamma) and run one V-cycle or one solve")
    args = ap.parse_args()
    args.gammas = [float(x) for x in args.gammas.split(",")]
    args.warmup = max(args.warmup, 0)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.probe:
        return run_probe(args, local)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
