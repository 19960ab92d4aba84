#!/usr/bin/env python
"""Throughput of the ICWF time step (arXiv 1805.11169) on one GB300, as one JSON line.

Workload: the Shin-Metiu proton-coupled electron transfer model at the paper's scale, electron grid
1024 points on [-100, 100], proton grid 512 points on [-9.5, 9.5], N = 1024 trajectories,
dt = 0.05 a.u., initial state sampled from |Psi0|^2 with seed 0 (synthetic inputs: model potential
and BO states computed here).  A step is one full ICWF update of all N trajectories (velocities,
positions, CWF propagation, matrix assembly, regularised Cholesky + RK4); observables are
evaluated every 100 steps inside the timed region.  Metric: trajectory-steps/s = N * steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fp64|bf16x3|tf32x3]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores (same metric)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OBS_EVERY = 100
# mode -> (precision enum, dtype label, SVD cutoff, regulariser eps).  Every mode solves with
# eps = 1e-6: the mixed modes' overlap is an exact Gram of fixed-point CWFs (positive
# semidefinite to rounding), so they need no larger shift than FP64.
MODES = {"fp64": (0, "f64", 1e-12, 1e-6), "bf16x3": (1, "mixed-bf16x3", 1e-8, 1e-6),
         "tf32x3": (2, "mixed-tf32x3", 1e-8, 1e-6)}
NOMINAL_FP64_TFLOPS = 1.25   # GB300 FP64 (vector and DMMA alike), nominal
# FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz = 40.3e12 lane operations/s.  The mixed modes factorise
# in double-float arithmetic on it: one complex multiply-add (8 flops) costs 39 FP32 operations
# (three real compensated products of 13 operations each), so the FP64-equivalent ceiling is
# 40.3e12 * 8 / 39 = 8.26 TFLOP/s.
FP32_LANE_OPS = 152 * 128 * 2.07e9
DF64_CMAC_OPS = 39
DF64_TFLOPS = FP32_LANE_OPS * 8 / DF64_CMAC_OPS / 1e12
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rates
# DRAM bytes (read + write) per family call from one ncu capture, with the profile that gives them;
# keyed by (family, mode, N).  Valid only while the kernels are the ones profiled.
TRAFFIC = {("cholesky", "tf32x3", 1024): (193.6e6, "profiles/k_chol_step_df_mixed_N1024.md")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="tf32x3", choices=list(MODES))
    ap.add_argument("--vs-exact", type=int, default=0, metavar="STEPS",
                    help="also run ICWF and the exact 2D propagation side by side for STEPS steps "
                         "and report density and population errors ('vs_exact'); not timed")
    ap.add_argument("--vs-exact-every", type=int, default=2000)
    ap.add_argument("--coeff-scheme", default="interpolated", choices=["interpolated", "frozen"],
                    help="RK4 with S, Heff linear over the step (two factorisations per step, "
                         "default) or frozen at t_n (one)")
    ap.add_argument("--no-exact2d", action="store_true",
                    help="skip the exact 2D propagation measurement on the same grid")
    ap.add_argument("--solve", default="df64", choices=["df64", "fp64"],
                    help="mixed modes: Cholesky and triangular solves in double-float (default) "
                         "or FP64")
    ap.add_argument("--n-traj", type=int, default=1024)
    ap.add_argument("--nx", type=int, default=1024, help="electron grid points (profiling cases)")
    ap.add_argument("--nR", type=int, default=512, help="nuclear grid points (profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--serving-jobs", type=int, default=24,
                    help="jobs in the serving stream measured beside the throughput (0: skip)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-mode comparison run")
    ap.add_argument("--workload", default="shin_metiu", choices=["shin_metiu", "cavity"],
                    help="Shin-Metiu 1024 x 512 (default) or the cavity 2048 x 256")
    ap.add_argument("--lam", type=float, default=0.5, help="cavity coupling lambda")
    ap.add_argument("--eps", type=float, default=None, help="override the mode's regulariser")
    ap.add_argument("--no-step-graphs", action="store_true",
                    help="launch the step's kernels directly instead of replaying captured graphs")
    ap.add_argument("--workload-cache", default=None, metavar="NPZ",
                    help="read the Shin-Metiu tables (V, Psi0, BO states) from this file if it "
                         "holds the grid, else build and save them (for profiling runs)")
    ap.add_argument("--overlap-split", action="store_true",
                    help="mixed modes: S from the split products (FP32 accumulation) instead of "
                         "the exact fixed-point Gram")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the rank-error, mixed-vs-FP64 and cavity reports")
    return ap.parse_args()


_WORKLOADS = {}


CAVITY_EPS = 1e-4   # the cavity's regulariser in every mode (its coefficient equation is stiff)
_CACHE = None       # --workload-cache: .npz file the Shin-Metiu tables are read from / saved to
_T0 = time.perf_counter()


def log(msg):
    sys.stderr.write("[bench %.1fs] %s\n" % (time.perf_counter() - _T0, msg))
    sys.stderr.flush()


def _sm_paper_cached(nx, nR):
    """The Shin-Metiu paper-scale workload, its tables (V, Psi0, BO states) read from the cache
    file when it holds this grid, else built (and saved there)."""
    import dataclasses
    import numpy as np
    import workloads
    tag = np.array([nx, nR])
    if os.path.exists(_CACHE):
        z = np.load(_CACHE, allow_pickle=False)
        if np.array_equal(z["grid"], tag):
            fields = {k: (z[k].item() if z[k].ndim == 0 else z[k]) for k in z.files
                      if k not in ("grid", "model_keys", "model_vals")}
            model = dict(zip(z["model_keys"].tolist(), z["model_vals"].tolist()))
            model["kind"] = "shin_metiu"
            return workloads.Workload(model=model, **fields)
    w = workloads.WORKLOADS["sm_paper"](nx=nx, nR=nR)
    d = {f.name: getattr(w, f.name) for f in dataclasses.fields(w) if f.name != "model"}
    mk = [k for k in w.model if k != "kind"]
    np.savez(_CACHE, grid=tag, model_keys=np.array(mk),
             model_vals=np.array([float(w.model[k]) for k in mk]), **d)
    return w


def make_workload(n_traj, cutoff, eps, nx=1024, nR=512, kind="shin_metiu", lam=0.5):
    """The synthetic workload (tables built once per grid and model, then re-parameterised).
    The cavity keeps its own dt (0.01) and eps (CAVITY_EPS)."""
    from workloads import WORKLOADS
    key = (kind, nx, nR, lam)
    if key not in _WORKLOADS:
        if kind == "cavity":
            _WORKLOADS[key] = WORKLOADS["cavity"](lam=lam)
        elif _CACHE:
            _WORKLOADS[key] = _sm_paper_cached(nx, nR)
        else:
            _WORKLOADS[key] = WORKLOADS["sm_paper"](nx=nx, nR=nR)
        log(f"workload {kind} {nx}x{nR} ready")
    if kind == "cavity":
        eps = max(eps, CAVITY_EPS)
    return _WORKLOADS[key].with_(n_traj=n_traj, svd_rel_cutoff=cutoff, s_reg_eps=eps)


def workload_name(w):
    if w.model.get("kind") == "cavity":
        return f"cavity_{w.nx}x{w.nR}_lambda{w.model['lam']}_N{w.n_traj}_dt{w.dt}"
    return f"shin_metiu_{w.nx}x{w.nR}_N{w.n_traj}_dt{w.dt}"


# ---------------------------------------------------------------- distributed plumbing

def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    dist.init_process_group("nccl" if os.environ.get("ICWF_BENCH_GLOO") is None else "gloo")
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, units_per_rank, slowest_s):
    """Whole-job throughput of ws independent replicas: all ranks' units over the slowest rank's
    time (every rank runs the same workload; the job ends when the last one does)."""
    return ws * units_per_rank / slowest_s


# ---------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.f:
            return None
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline bookkeeping

def algorithmic_work(fam, w, K, mode, nfact=2):
    """(amount, unit, bound) of algorithmic work per launch of a kernel family."""
    N, nx, nR = w.n_traj, w.nx, w.nR
    c = 16 if mode == "fp64" else 8
    if fam == "assemble":
        # Hermitian half of (K+1) Grams per side: 4 N^2 (K+1)(nx+nR) real flops
        return 4.0 * N * N * (K + 1) * (nx + nR), "flop", "alu" if mode == "fp64" else "tensor"
    if fam == "propagate":
        return 2.0 * N * (nx + nR) * c, "byte", "hbm"
    if fam == "cholesky":
        # one call factors S(t+dt/2) and S(t+dt) together (interpolated scheme; the frozen one
        # factors S(t+dt) alone): nfact x (4/3) N^3 (complex Cholesky)
        return nfact * 4.0 / 3.0 * N ** 3, "flop", "alu"
    if fam == "velocity":
        return 2.0 * 4 * N * N * c, "byte", "hbm"
    if fam == "rk4_matvec":
        return 16.0 * N * N * (1 if True else 2), "byte", "hbm"
    if fam == "chol_solve":
        return 2 * 8.0 * N * N, "flop", "alu"
    return None


def roofline(prof, w, K, mode, peaks, solve="df64", nfact=2):
    fam = max(prof, key=lambda f: prof[f][0])
    ms, n = prof[fam]
    work = algorithmic_work(fam, w, K, mode, nfact)
    out = {"kernel": fam, "launches": n, "avg_ms": ms / max(n, 1)}
    if work is None or n == 0:
        return out
    amount, unit, bound = work
    rate = amount / (ms / n / 1e3)
    if unit == "byte":
        out.update(bound="hbm", achieved=rate / 1e9, peak=peaks.get("hbm_gbs"), unit="GB/s",
                   peak_source="measured (MEASURED_PEAKS.json hbm_gbs)")
    elif bound == "tensor":
        # algorithmic Gram flops against the split-product ceiling: three products per Gram in the
        # operand type (TF32 at the nominal TF32/BF16 ratio of the measured BF16 peak)
        bf16 = peaks.get("bf16_tflops_sustained")
        ratio = TF32_PER_BF16 if mode == "tf32x3" else 1.0
        out.update(bound="tensor", achieved=rate / 1e12,
                   peak=bf16 * ratio / 3 if bf16 else None, unit="TFLOP/s",
                   peak_source=("measured bf16 sustained (MEASURED_PEAKS.json) x %.3f (nominal "
                                "%s/BF16) / 3 split products" % (ratio, "TF32" if ratio < 1 else "BF16")))
    elif mode == "fp64" or solve == "fp64":
        out.update(bound="alu", achieved=rate / 1e12, peak=NOMINAL_FP64_TFLOPS, unit="TFLOP/s",
                   peak_source="nominal FP64 (152 SMs x 2 FP64 FMA/clk x 2.07 GHz)")
    else:
        out.update(bound="alu", achieved=rate / 1e12, peak=DF64_TFLOPS, unit="TFLOP/s",
                   peak_source="double-float on the FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz, "
                               "8 flops per 39 FP32 operations (FP64-equivalent flops)")
    if out.get("peak"):
        out["frac"] = out["achieved"] / out["peak"]
    tr = TRAFFIC.get((fam, mode if solve == "df64" else "fp64-solve", w.n_traj))
    out["traffic"] = tr[0] if tr else None
    if tr:
        out["traffic_unit"] = "bytes per call (DRAM read + write, ncu)"
        out["traffic_source"] = tr[1]
    return out


# ---------------------------------------------------------------- our arm

def n_obs_calls(steps):
    """Observables calls in a timed region of `steps` steps: one every OBS_EVERY steps, and at
    least one, so that a short timed region still pays for them (never fewer than the metric's
    rate of one per 100 steps)."""
    return max(1, steps // OBS_EVERY)


def timed_steps(sim, steps, warmup, local, ws=1, prof_steps=20):
    """W untimed steps, then `steps` steps timed one by one with CUDA events on the library's
    stream (L2 flushed before each), observables n_obs_calls(steps) times inside the timed
    region, clocks sampled meanwhile.  The library replays each step as a captured CUDA graph
    there; the per-family kernel times come from a separate pass of `prof_steps` steps with the
    library's timing events on (direct launches)."""
    import torch
    import paper_1805_11169_gb300 as g
    stream = torch.cuda.ExternalStream(sim.stream())
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(warmup):
        sim.step(1)
    launches0 = sim.info()["kernel_launches"]
    n_obs = n_obs_calls(steps)
    obs_at = {steps - 1 - k * (steps // n_obs) for k in range(n_obs)}
    barrier(ws)
    torch.cuda.synchronize()
    step_ms = []
    with Clocks(local) as clk:
        for s in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(1)
            if s in obs_at:
                sim.observables()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(ws)
    launches = sim.info()["kernel_launches"] - launches0 + 4 * n_obs
    # per-family breakdown (direct launches, timing events on), scaled to per-step values below
    g.icwf_profile_reset(sim.h)
    g.icwf_profile_enable(sim.h, True)
    for s in range(prof_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        sim.step(1)
    sim.observables()
    g.icwf_profile_enable(sim.h, False)
    raw = g.icwf_profile_read(sim.h)
    prof = {f: (ms * steps / prof_steps, int(round(n * steps / prof_steps))) for f, (ms, n) in raw.items()}
    prof["observables"] = (raw["observables"][0] * n_obs, raw["observables"][1] * n_obs)
    return sum(step_ms), prof, launches, clk.summary(), n_obs


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def run_ours(args, rank, ws, local):
    import numpy as np
    import torch
    import paper_1805_11169_gb300 as g

    torch.cuda.set_device(local)
    prec, dtype_name, cutoff, eps = MODES[args.mode]
    if args.eps is not None:
        eps = args.eps
    w = make_workload(args.n_traj, cutoff, eps, args.nx, args.nR, args.workload, args.lam)
    params = g.params_from(w, precision=prec, solve_fp64=int(args.solve == "fp64"),
                           coeff_scheme=int(args.coeff_scheme == "frozen"),
                           overlap_split=int(args.overlap_split))

    sim = g.Icwf(params, w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, w.seed)
    if args.no_step_graphs:
        sim.set_step_graphs(False)
    info = sim.info()
    log("handle created and initialised")
    total_ms, prof, launches, clocks, n_obs = timed_steps(sim, args.steps, args.warmup, local, ws)
    log("timed steps done")
    total_s = max_over_ranks(total_ms / 1e3, ws)
    value = whole_job_rate(ws, w.n_traj * args.steps, total_s)
    sim.close()

    peaks, _ = load_peaks()
    prof_step = {f: v for f, v in prof.items() if v[1] > 0 and f != "observables"}
    rl = roofline(prof_step, w, info["rank"], args.mode, peaks, args.solve,
                  1 if args.coeff_scheme == "frozen" else 2)

    out = {
        "metric": "ICWF trajectory-steps/s at N=1024",
        "value": value,
        "unit": "trajectory-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype_name,
        "data": ("synthetic (%s potential, BO states and |Psi0|^2 sampling computed here)"
                 % ("cavity" if args.workload == "cavity" else "Shin-Metiu")),
        "config": {"workload": workload_name(w), "nx": w.nx, "nR": w.nR, "n_traj": w.n_traj,
                   "dt": w.dt, "rank_k": info["rank"], "svd_rel_cutoff": cutoff, "s_reg_eps": eps,
                   "svd_tail_rel": info["tail_rel"], "coeff_scheme": "rk4-" + args.coeff_scheme,
                   "overlap": ("fp64" if args.mode == "fp64" else
                               "split products, FP32 accumulation" if args.overlap_split else
                               "exact Gram of 4-digit fixed-point CWFs (BF16 tensor cores)"),
                   "solve": ("fp64" if args.mode == "fp64" or args.solve == "fp64"
                             else "double-float (FP32 pairs)"),
                   "obs_every": OBS_EVERY, "obs_calls_timed": n_obs,
                   "step_launch": ("direct kernel launches" if args.no_step_graphs else
                                   "one captured CUDA graph per step"),
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "replicas" if ws > 1 else "single-gpu"},
        "roofline": rl,
        "kernels_ms_per_step": {f: v[0] / args.steps for f, v in prof.items() if v[1]},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_e2e:
        record(out, "e2e", run_e2e, args, w, params, g)
    if rank == 0 and not args.no_fp64 and args.mode != "fp64":
        if record(out, "fp64", run_fp64_comparison):
            out["speedup_vs_fp64"] = value / out["fp64"]["value"]
    if rank == 0 and not args.no_extras and args.workload == "shin_metiu":
        record(out, "rank_error", run_rank_error, args.mode)
        if args.mode != "fp64":
            record(out, "mixed_vs_fp64", run_mixed_vs_fp64, args.mode, eps)
            if args.solve != "fp64":
                record(out, "solve_fp64", run_solve_fp64, args.mode, eps, local)
        record(out, "cavity", run_cavity_line, args, local, peaks)
    if rank == 0 and not args.no_exact2d:
        record(out, "exact2d", run_exact2d, w)
    if rank == 0 and args.vs_exact > 0:
        record(out, "vs_exact", run_vs_exact, w, prec, args.vs_exact, args.vs_exact_every, w.seed,
               int(args.overlap_split))
    if rank == 0 and args.serving_jobs > 0:
        record(out, "serving", run_serving, args.serving_jobs,
               args.mode if args.mode != "fp64" else "tf32x3")
    if rank == 0 and not args.no_cpu:
        record(out, "cpu_baseline", run_cpu_baseline, w, args.cpu_budget_s)
    return out


def record(out, key, fn, *fargs):
    """out[key] = fn(*fargs); a record that fails is reported in the line as {"error": ...} (and
    on stderr) instead of losing the headline measured before it.  True if it succeeded."""
    try:
        out[key] = fn(*fargs)
        return True
    except Exception as e:  # noqa: BLE001 -- any failure of an extra record is reported, not raised
        out[key] = {"error": f"{type(e).__name__}: {e}"}
        log(f"{key} failed: {type(e).__name__}: {e}")
        return False


def run_e2e(args, w, params, g):
    """The same metric through the public C ABI with host buffers: create (V), projectors,
    init (Psi0), K steps with observables every 100 steps copied back, destroy."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = g.Icwf(params, w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, w.seed)
    t1 = time.perf_counter()
    n_obs = 0
    done = 0
    while done < args.steps:
        k = min(OBS_EVERY, args.steps - done)
        sim.step(k)
        done += k
        if done % OBS_EVERY == 0 or done == args.steps:
            sim.observables()
            n_obs += 1
    t2 = time.perf_counter()
    sim.close()
    dt = time.perf_counter() - t0
    h2d = w.V.nbytes + w.phi.nbytes + w.psi0.nbytes
    d2h = n_obs * 8 * (w.nx + w.nR + 4 + 64 + 8)
    return {"value": w.n_traj * args.steps / dt, "unit": "trajectory-steps/s",
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "wall_s": dt, "includes": "create (host SVD of V), init (sampling, slices, C0), steps, "
                                      "observables copies, destroy",
            "setup_s": t1 - t0,
            "steps_value": w.n_traj * args.steps / (t2 - t1),
            "steps_value_includes": "icwf_step and icwf_observables (results copied to host "
                                    "arrays) only, after create and init"}


def run_cpu_baseline(w, budget_s):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the same workload:
    the first M steps of the same job (M chosen to fit the budget)."""
    import numpy as np
    from oracle.icwf import Icwf as Oracle, Params
    p = Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
               w.n_traj, w.svd_rel_cutoff, w.s_reg_eps)
    o = Oracle(p, w.V)
    st = o.init_from_density(w.psi0, w.seed)
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(st)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    threads = os.environ.get("OMP_NUM_THREADS")
    return {"value": w.n_traj * n / dt, "unit": "trajectory-steps/s",
            "cores": int(threads) if threads else (os.cpu_count() or 1), "kind": "oracle",
            "sample": f"first {n} steps of the same N={w.n_traj} job (factorised Heff, same rank)",
            "s_per_step": dt / n}


# ---------------------------------------------------------------- FP64 comparison and serving

def run_exact2d(w, steps=50, warmup=2):
    """The exact Strang propagation of Psi(x, R) on the GPU (FP64) on the bench grid: grid
    points x steps / s, with its FP64 roofline (two 2D FFTs of 5 n log2 n flops and ~24 flops of
    phases per point and step)."""
    import paper_1805_11169_gb300 as g
    e = g.Exact2D(g.params_from(w), w.V)
    e.set_state(w.psi0)
    e.step(warmup)
    t0 = time.perf_counter()
    e.step(steps)
    dt = time.perf_counter() - t0
    e.close()
    n = w.nx * w.nR
    flops = 2 * 5.0 * n * math.log2(n) + 24.0 * n
    return {"value": n * steps / dt, "unit": "grid-point-steps/s", "ms_per_step": 1e3 * dt / steps,
            "grid": [w.nx, w.nR], "steps": steps, "dtype": "f64",
            "roofline": {"bound": "alu", "achieved": flops * steps / dt / 1e12,
                         "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops * steps / dt / 1e12 / NOMINAL_FP64_TFLOPS}}


def run_vs_exact(w, prec, steps, every, seed, overlap_split=0):
    """ICWF against the exact propagation of the full Psi(x, R) from the same Psi0 on the same
    grid (the paper's comparison in Figs. 1-2): L1 errors of the reduced densities and the largest
    BO-population error at every `every` steps.  ICWF starts from the sampled trajectories, so
    the t = 0 row shows the error of the initial representation."""
    import numpy as np
    import paper_1805_11169_gb300 as g
    sim = g.Icwf(g.params_from(w, precision=prec, overlap_split=overlap_split), w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, seed)
    ex = g.Exact2D(g.params_from(w), w.V)
    ex.set_projectors(w.phi)
    ex.set_state(w.psi0)
    rows = []
    t0 = time.perf_counter()
    for k in range(0, steps + 1, every):
        if k:
            sim.step(every)
            ex.step(every)
        a, b = sim.observables(), ex.observables()
        rows.append({"t_au": round(a["t"], 6),
                     "rho_x_L1": float(w.dx * np.sum(np.abs(a["rho_x"] - b["rho_x"]))),
                     "rho_R_L1": float(w.dR * np.sum(np.abs(a["rho_R"] - b["rho_R"]))),
                     "pop_max_err": float(np.max(np.abs(a["pop"] - b["pop"]))),
                     "pop_icwf": [float(v) for v in a["pop"]],
                     "pop_exact": [float(v) for v in b["pop"]],
                     "norm_icwf": float(a["norm"])})
    wall = time.perf_counter() - t0
    sim.close()
    ex.close()
    return {"n_traj": w.n_traj, "steps": steps, "dt": w.dt, "s_reg_eps": w.s_reg_eps,
            "checkpoints": rows,
            "max_rho_x_L1": max(r["rho_x_L1"] for r in rows),
            "max_rho_R_L1": max(r["rho_R_L1"] for r in rows),
            "max_pop_err": max(r["pop_max_err"] for r in rows), "wall_s": wall}


def init_residual(sim, w):
    """||(S + eps I) C - b|| / ||b|| of an FP64-mode handle right after initialisation, with
    b_a = <psi_a chi_a | Psi0> formed here from the handle's own FP64 CWFs (the slices the
    library projected) and S as stored."""
    import numpy as np
    st = sim.state()
    S = sim.matrices()["S"]
    b = w.dx * w.dR * np.sum(st["psi"].conj() * (w.psi0 @ st["chi"].conj()), axis=0)
    r = (S + w.s_reg_eps * np.eye(w.n_traj)) @ st["C"] - b
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def run_fp64_comparison(steps=10, warmup=2):
    """The same workload in FP64 mode (same GB300, same process): trajectory-steps/s, and the
    residual of the initial solve (FP64 solver, emulated-FP64 trailing updates)."""
    import torch
    import paper_1805_11169_gb300 as g
    prec, dtype_name, cutoff, eps = MODES["fp64"]
    w = make_workload(1024, cutoff, eps)
    sim = g.Icwf(g.params_from(w, precision=prec), w.V)
    sim.init_from_density(w.psi0, w.seed)
    resid = init_residual(sim, w)
    stream = torch.cuda.ExternalStream(sim.stream())
    for _ in range(warmup):
        sim.step(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    k = sim.info()["rank"]
    sim.close()
    return {"value": w.n_traj * steps / (ms / 1e3), "unit": "trajectory-steps/s",
            "ms_per_step": ms / steps, "dtype": dtype_name, "rank_k": k, "steps": steps,
            "svd_rel_cutoff": cutoff, "s_reg_eps": eps, "init_solve_residual": resid}


def run_solve_fp64(mode, eps, local, steps=30, warmup=3):
    """The headline configuration with the FP64 solver (solve_fp64 = 1): trajectory-steps/s and the
    factorisation's time per call, with its trailing updates in emulated FP64 on the tensor cores
    (the default) and with FP64 FMAs; plus the initial-solve residual of the same solver in FP64
    mode on this workload."""
    import paper_1805_11169_gb300 as g
    prec, _, cutoff, _ = MODES[mode]
    w = make_workload(1024, cutoff, eps)
    out = {"s_reg_eps": eps}
    for name, emu, n in (("emulated_update", 1, steps), ("fma_update", 0, max(5, steps // 3))):
        sim = g.Icwf(g.params_from(w, precision=prec, solve_fp64=1), w.V)
        sim.set_emulated_update(emu)
        sim.set_projectors(w.phi)
        sim.init_from_density(w.psi0, w.seed)
        total_ms, prof, _, clocks, _ = timed_steps(sim, n, warmup, local, prof_steps=10)
        sim.close()
        ch = prof.get("cholesky", (0.0, 0))
        out[name] = {"value": w.n_traj * n / (total_ms / 1e3), "ms_per_step": total_ms / n,
                     "steps": n, "cholesky_ms_per_call": ch[0] / max(ch[1], 1) if ch[1] else None,
                     "clocks": clocks}
    sim = g.Icwf(g.params_from(w, precision=MODES["fp64"][0]), w.V)
    sim.init_from_density(w.psi0, w.seed)
    out["init_solve_residual_fp64_mode"] = init_residual(sim, w)
    sim.close()
    out["value"] = out["emulated_update"]["value"]
    out["unit"] = "trajectory-steps/s"
    return out


def run_rank_error(mode, steps=10, n_cols=16):
    """Error of the factorised Heff (rank k from the SVD cutoff) against the full
    O(N^2 nx nR) contraction, on sampled columns at the bench configuration (N = 1024,
    1024 x 512, after `steps` steps): the full double sum comes from icwf_heff_direct (FP64,
    same CWFs and positions).  Reported for the FP64 mode at cutoffs 1e-8 and 1e-12 (rank
    truncation alone) and for the mixed mode at its cutoff (truncation + tensor-core rounding)."""
    import numpy as np
    import paper_1805_11169_gb300 as g
    rng = np.random.default_rng(7)
    cols = np.sort(rng.choice(1024, n_cols, replace=False)).astype(np.int32)
    out = {"n_cols": n_cols, "steps": steps, "metric": "max over sampled columns b of "
           "||Heff_factorised[:, b] - Heff_direct[:, b]|| / ||Heff_direct[:, b]||"}
    runs = [("fp64", 0, 1e-8), ("fp64", 0, 1e-12)]
    if mode != "fp64":
        runs.append((mode, MODES[mode][0], MODES[mode][2]))
    for name, prec, cutoff in runs:
        w = make_workload(1024, cutoff, MODES[name][3])
        sim = g.Icwf(g.params_from(w, precision=prec), w.V)
        sim.init_from_density(w.psi0, w.seed)
        sim.step(steps)
        Hd = sim.heff_direct(cols)
        Hf = sim.matrices()["Heff"][:, cols]
        errs = np.linalg.norm(Hf - Hd, axis=0) / np.linalg.norm(Hd, axis=0)
        info = sim.info()
        out[f"{name}_cutoff{cutoff:g}"] = {"rank_k": info["rank"], "svd_tail_rel": info["tail_rel"],
                                           "max_rel": float(errs.max()),
                                           "median_rel": float(np.median(errs))}
        sim.close()
    return out


def run_mixed_vs_fp64(mode, eps_mixed, steps=100):
    """Mixed mode at its own eps against the FP64 mode at eps 1e-6 (both on the GPU, same
    N = 1024 job, same seed) after `steps` steps: L1 distances of rho_x, rho_R and the BO
    populations, and the norms."""
    import numpy as np
    import paper_1805_11169_gb300 as g
    res = {}
    for name in ("fp64", mode):
        prec, _, cutoff, eps = MODES[name]
        w = make_workload(1024, cutoff, eps)
        sim = g.Icwf(g.params_from(w, precision=prec), w.V)
        sim.set_projectors(w.phi)
        sim.init_from_density(w.psi0, w.seed)
        sim.step(steps)
        res[name] = sim.observables()
        sim.close()
    a, b = res[mode], res["fp64"]
    return {"steps": steps, "mixed_eps": eps_mixed, "fp64_eps": MODES["fp64"][3],
            "rho_x_L1": float(w.dx * np.sum(np.abs(a["rho_x"] - b["rho_x"]))),
            "rho_R_L1": float(w.dR * np.sum(np.abs(a["rho_R"] - b["rho_R"]))),
            "pop_L1": float(np.sum(np.abs(a["pop"] - b["pop"]))),
            "norm_mixed": float(a["norm"]), "norm_fp64": float(b["norm"])}


def run_cavity_line(args, local, peaks, steps=50, warmup=3):
    """Throughput of the same mode on the cavity workload (2048 x 256, lambda 0.5, N = 1024,
    dt = 0.01, eps = 1e-4; V_c exactly rank 1), timed like the headline, with its own roofline
    entry."""
    import paper_1805_11169_gb300 as g
    prec, _, cutoff, eps = MODES[args.mode]
    w = make_workload(1024, cutoff, eps, kind="cavity", lam=args.lam)
    sim = g.Icwf(g.params_from(w, precision=prec), w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, w.seed)
    k = sim.info()["rank"]
    total_ms, prof, launches, clocks, n_obs = timed_steps(sim, steps, warmup, local)
    sim.close()
    prof_step = {f: v for f, v in prof.items() if v[1] > 0 and f != "observables"}
    return {"workload": workload_name(w), "s_reg_eps": w.s_reg_eps,
            "value": w.n_traj * steps / (total_ms / 1e3),
            "unit": "trajectory-steps/s", "ms_per_step": total_ms / steps, "steps": steps,
            "rank_k": k, "obs_calls_timed": n_obs, "gpu_launches": int(launches),
            "roofline": roofline(prof_step, w, k, args.mode, peaks, args.solve),
            "kernels_ms_per_step": {f: v[0] / steps for f, v in prof.items() if v[1]},
            "clocks": clocks}


def _model_library(rng):
    """A few synthetic model instances (grids and parameters drawn like the mixed-size stream:
    Shin-Metiu with R_f ~ U[4, 6], R0 ~ U[-5, -3]; cavity with lambda ~ U[0.1, 1]).  Shin-Metiu
    runs at dt 0.05 with eps 1e-6, the cavity at dt 0.01 with eps 1e-4 (its product initial state
    makes the coefficient equation stiff)."""
    from workloads import cavity, shin_metiu
    lib = []
    for nx, nR in ((256, 128), (512, 128), (512, 256)):
        lib.append(shin_metiu(nx=nx, x_range=(-60.0, 60.0), nR=nR, R_range=(-9.0, 9.0),
                              Rf=float(rng.uniform(4, 6)), R0=float(rng.uniform(-5, -3)),
                              dt=0.05, n_traj=64, svd_rel_cutoff=1e-8, s_reg_eps=1e-6))
    for nx, nq in ((512, 128), (1024, 128)):
        lib.append(cavity(nx=nx, x_range=(-60.0, 60.0), nq=nq, q_range=(-20.0, 20.0),
                          lam=float(rng.uniform(0.1, 1.0)), dt=0.01, n_traj=64,
                          svd_rel_cutoff=1e-8, s_reg_eps=1e-4))
    return lib


def _serving_jobs(n_jobs, seed):
    import numpy as np
    rng = np.random.default_rng(seed)
    lib = _model_library(rng)
    Ns = (64, 128, 256, 512, 1024, 2048)
    jobs = [dict(model=int(rng.integers(len(lib))), N=int(rng.choice(Ns)),
                 steps=int(rng.integers(100, 401)), seed=int(rng.integers(1 << 31)))
            for _ in range(n_jobs)]
    return lib, jobs


def _make_job(lib, job, precision):
    import paper_1805_11169_gb300 as g
    w = lib[job["model"]].with_(n_traj=job["N"])
    sim = g.Icwf(g.params_from(w, precision=precision), w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, job["seed"])
    return sim, w


def _run_stream(lib, jobs, arrivals, graphs, max_live, precision, grouping=True):
    """Feed the jobs at their arrival times into a pool and tick it until all are done."""
    import numpy as np
    import paper_1805_11169_gb300 as g
    n_jobs = len(jobs)
    pool = g.icwf_pool_create(64 << 30, max_live)
    g.icwf_pool_set_graphs(pool, graphs)
    g.icwf_pool_set_grouping(pool, grouping, 0)
    t_start = time.perf_counter()
    submitted, lat, ids, grids, results = 0, {}, {}, {}, {}
    done = set()
    while len(done) < n_jobs:
        now = time.perf_counter() - t_start
        while submitted < n_jobs and arrivals[submitted] <= now:
            sim, w = _make_job(lib, jobs[submitted], precision)
            ids[submitted] = g.icwf_pool_submit(pool, sim.release(), jobs[submitted]["steps"])
            grids[submitted] = (w.nx, w.nR)
            submitted += 1
        if submitted == len(done) and submitted < n_jobs:
            time.sleep(max(0.0, min(0.01, arrivals[submitted] - now)))
            continue
        g.icwf_pool_tick(pool)
        for j, jid in ids.items():
            if j in done:
                continue
            st, obs = g.icwf_pool_poll(pool, jid, *grids[j])
            if st in (2, 3):
                done.add(j)
                lat[j] = time.perf_counter() - t_start - arrivals[j]
                results[j] = obs if st == 2 else None
    makespan = time.perf_counter() - t_start
    stats = g.icwf_pool_get_stats(pool)
    g.icwf_pool_destroy(pool)
    L = np.array([lat[j] for j in range(n_jobs)])
    ts = sum(j["N"] * j["steps"] for j in jobs)
    stepping_ticks = max(1, stats["graph_launches"] + (stats["ticks"] if not graphs else 0))
    return {"p50_s": float(np.percentile(L, 50)), "p99_s": float(np.percentile(L, 99)),
            "traj_steps_per_s": ts / makespan, "makespan_s": makespan,
            "failed": sum(1 for r in results.values() if r is None),
            "ticks": stats["ticks"], "graph_launches": stats["graph_launches"],
            "graph_builds": stats["graph_builds"],
            "kernels_per_graph_launch": (stats["kernel_nodes"] / stats["graph_launches"]
                                         if stats["graph_launches"] else None),
            "grouped_kernels_per_graph_launch": (stats["group_nodes"] / stats["graph_launches"]
                                                 if stats["graph_launches"] else None),
            "host_launches_per_tick": (stats["graph_launches"] / stats["ticks"] if graphs else
                                       None),
            "eager_job_steps": stats["eager_job_steps"]}, results


def _run_saturated(lib, jobs, max_live, precision, grouping):
    """Capacity: every job created first, all submitted at once, the pool ticked until all are
    done; aggregate trajectory-steps/s over the makespan of the ticks."""
    import paper_1805_11169_gb300 as g
    made = [_make_job(lib, job, precision) for job in jobs]
    pool = g.icwf_pool_create(64 << 30, max_live)
    g.icwf_pool_set_grouping(pool, grouping, 0)
    ids = [g.icwf_pool_submit(pool, sim.release(), job["steps"])
           for (sim, _w), job in zip(made, jobs)]
    grids = [(w.nx, w.nR) for _sim, w in made]

    def states():
        return [g.icwf_pool_poll(pool, i, *grid)[0] for i, grid in zip(ids, grids)]

    t0 = time.perf_counter()
    while True:
        live, _ = g.icwf_pool_tick(pool)
        if live == 0 and all(st in (2, 3) for st in states()):
            break
    makespan = time.perf_counter() - t0
    failed = sum(1 for st in states() if st == 3)
    stats = g.icwf_pool_get_stats(pool)
    g.icwf_pool_destroy(pool)
    ts = sum(j["N"] * j["steps"] for j in jobs)
    return {"traj_steps_per_s": ts / makespan, "makespan_s": makespan, "failed": failed,
            "ticks": stats["ticks"],
            "kernels_per_graph_launch": (stats["kernel_nodes"] / stats["graph_launches"]
                                         if stats["graph_launches"] else None),
            "grouped_kernels_per_graph_launch": (stats["group_nodes"] / stats["graph_launches"]
                                                 if stats["graph_launches"] else None)}


def run_serving(n_jobs, mode="tf32x3", seed=0, load=0.7, max_live=16, n_checked=4):
    """Poisson stream of mixed-size jobs (N up to 2048) through the pool (continuous batching),
    with captured tick graphs and grouped velocity/propagation kernels over all live jobs (the
    default) and with direct launches: job latency p50/p99 (arrival -> result on the host),
    aggregate trajectory-steps/s and launches per tick.  The stream's first 12 jobs submitted all at
    once measure the pool's capacity, with and without the grouped kernels (`saturated`).
    Jobs' mixed-precision results are checked against FP64 runs of the same jobs (a sample of the
    small ones: the FP64 path is ~50x slower)."""
    import numpy as np
    prec = MODES[mode][0]
    lib, jobs = _serving_jobs(n_jobs, seed)
    # isolated service time of the mean job: the arrival rate is `load` times the rate at which
    # the GPU serves jobs one at a time
    t_iso = []
    for job in jobs[: min(4, n_jobs)]:
        t0 = time.perf_counter()
        sim, _ = _make_job(lib, job, prec)
        sim.step(job["steps"])
        sim.observables()
        sim.close()
        t_iso.append((time.perf_counter() - t0) / job["steps"] / job["N"])
    mean_service = float(np.mean(t_iso)) * float(np.mean([j["steps"] * j["N"] for j in jobs]))
    rate = load / mean_service
    arrivals = np.cumsum(np.random.default_rng(seed + 1).exponential(1.0 / rate, n_jobs))
    graphs, res = _run_stream(lib, jobs, arrivals, True, max_live, prec)
    eager, _ = _run_stream(lib, jobs, arrivals, False, max_live, prec)
    sat_jobs = jobs[:min(12, n_jobs)]   # the stream's first jobs (the same for any stream length)
    saturated = {("grouped" if gr else "ungrouped"): _run_saturated(lib, sat_jobs, max_live, prec, gr)
                 for gr in (True, False)}
    saturated["jobs"] = len(sat_jobs)
    # precision check: the first n_checked jobs with N <= 256, in FP64, same seed, alone
    checks = []
    for j, job in enumerate(jobs):
        if len(checks) >= n_checked:
            break
        if job["N"] > 256 or res.get(j) is None:
            continue
        sim, w = _make_job(lib, job, 0)
        sim.step(job["steps"])
        ref = sim.observables()
        sim.close()
        ob = res[j]
        checks.append({"job": j, "model": lib[job["model"]].model["kind"], "N": job["N"],
                       "steps": job["steps"],
                       "rho_x_L1": float(w.dx * np.sum(np.abs(ob["rho_x"] - ref["rho_x"]))),
                       "rho_R_L1": float(w.dR * np.sum(np.abs(ob["rho_R"] - ref["rho_R"]))),
                       "pop_L1": float(np.sum(np.abs(ob["pop"] - ref["pop"])))})
    return {"jobs": n_jobs, "p50_s": graphs["p50_s"], "p99_s": graphs["p99_s"],
            "traj_steps_per_s": graphs["traj_steps_per_s"], "graphs": graphs, "eager": eager,
            "saturated": saturated,
            "arrival_rate_per_s": rate, "max_live": max_live, "precision": MODES[mode][1],
            "vs_fp64": checks,
            "stream": "Poisson arrivals; Shin-Metiu (3 grids, dt 0.05, eps 1e-6) and cavity "
                      "(2 grids, dt 0.01, eps 1e-4) models; N in {64..2048}; 100-400 steps; "
                      "CI-sized stand-in for 2000 jobs"}


# ---------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, rank, ws):
    if rank != 0:
        return None
    prec, dtype_name, cutoff, eps = MODES[args.mode]
    w = make_workload(args.n_traj, cutoff, eps, args.nx, args.nR)
    from oracle.icwf import Icwf as Oracle, Params
    p = Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
               w.n_traj, w.svd_rel_cutoff, w.s_reg_eps)
    o = Oracle(p, w.V)
    st = o.init_from_density(w.psi0, w.seed)
    budget = 150.0
    t_start = time.perf_counter()
    for _ in range(args.warmup):
        o.step(st)
        if time.perf_counter() - t_start > budget / 3:
            break
    t0 = time.perf_counter()
    n = 0
    while n < args.steps:
        o.step(st)
        n += 1
        if (n % OBS_EVERY) == 0:
            o.observables(st, w.phi)
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    value = w.n_traj * n / dt
    cores = os.cpu_count() or 1
    return {
        "impl": "reference", "metric": "ICWF trajectory-steps/s at N=1024", "value": value,
        "unit": "trajectory-steps/s", "n_gpus": ws, "steps": n, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / n, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(w), "nx": w.nx, "nR": w.nR, "n_traj": w.n_traj,
                   "dt": w.dt, "rank_k": len(o.fac.s), "svd_rel_cutoff": cutoff},
        "cpu_baseline": {"value": value, "unit": "trajectory-steps/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{n} of the requested {args.steps} steps (time budget)"},
        "e2e": {"value": value, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    global _CACHE
    args = parse()
    _CACHE = args.workload_cache
    rank, ws, local = dist_init()
    if args.impl == "reference":
        out = run_reference(args, rank, ws)
    else:
        out = run_ours(args, rank, ws, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
