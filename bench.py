"""Benchmark of the shared-LHS batched solve on GB300.

Workload (one "step"): one batched solve of the FP64 pentadiagonal hyperdiffusion
system A = I + 0.25 D4 (hinged closure), N = 1024 unknowns, 65536 right-hand
sides drawn i.i.d. N(0, 1), interleaved layout; the shared factors are computed
once before timing (the paper times only the solve loop, section 3.4).  The
inputs (2 x 512 MiB) exceed the 126 MiB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--extras a,b] [--coarsening-systems M] [--table3-max-n N]
Under torchrun (N > 1) each rank solves its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.

--impl reference times the plain FP64 CPU oracle on the host cores on a bounded
sample of the same workload (there is no reference GPU implementation to run).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shared-LHS batched solves/s & HBM GB/s vs peak; fused/adjoint step/s vs plain"
UNIT = "batched solves/s"
WORKLOAD = "penta_hyper: FP64 pentadiagonal A=I+0.25*D4 (hinged), N=1024, M=65536 RHS ~ N(0,1), interleaved"
N_ROWS = 1024
M_SYS = 65536
R_COEF = 0.25
SEED = 2
# FP64 flops per element of one pentadiagonal solve: forward 2 FMA + 1 MUL, backward 2 FMA.
FLOPS_PER_ELT = 9
BYTES_PER_ELT = 16  # read the RHS once, write the solution once (FP64)
SM_COUNT = 152
SM_MAX_GHZ = 2.07
# FP64 FMA issue rate of GB300: 2 per clock per SM (nominal 1.25 TFLOP/s); peak in TFLOP/s.
FP64_PEAK_TFLOPS = 2 * 2 * SM_COUNT * SM_MAX_GHZ / 1e3
# sizes of the paper-workload extras (set from the command line)
OPTIONS = {"extras": [], "coarsening_systems": 1 << 16, "table3_max_n": 1024}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def hbm_peak():
    p = measured_peaks()
    if "hbm_gbs" in p:
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------- clocks sampler

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.device_index = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU baseline

def cpu_baseline(target_seconds=10.0, sample_systems=8192):
    """The FP64 oracle (NumPy, one core) on a bounded sample of the workload: the
    first `sample_systems` systems, full N, repeated until ~target_seconds.
    Returns (batched solves/s scaled to the full M, description)."""
    import numpy as np

    import synth
    from oracle import banded, matrices

    diags = matrices.hyperdiffusion_matrix(N_ROWS, R_COEF, "hinged")
    fac = banded.penta_factor(*diags)
    rhs = synth.rhs_normal(seed=SEED, N=N_ROWS, M=sample_systems)
    runs = 0
    t0 = time.perf_counter()
    while True:
        banded.penta_solve(*fac, rhs)
        runs += 1
        el = time.perf_counter() - t0
        if el >= target_seconds:
            break
    value = runs * (sample_systems / M_SYS) / el
    desc = (f"{runs} oracle solves of {sample_systems} of the {M_SYS} systems (full N={N_ROWS}) "
            f"in {el:.1f} s; solves/s scaled by {sample_systems}/{M_SYS}")
    _ = np
    return value, desc, el


def _oracle_worker(args):
    """One host process of the all-core oracle timing: the single-core timing on a
    sample of its own; returns (batched solves scaled to the full M, seconds)."""
    target, sample = args
    v, _, el = cpu_baseline(target_seconds=target, sample_systems=sample)
    return v * el, el


def cpu_baseline_all_cores(target_seconds=6.0, sample_systems=2048):
    """The same oracle run by one process per host core at once (spawned, so the
    parent's CUDA context is not inherited); returns (solves/s scaled to the full M,
    processes)."""
    import multiprocessing as mp
    n = max(1, os.cpu_count() or 1)
    env_keep = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"  # one thread per process
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.map(_oracle_worker, [(target_seconds, sample_systems)] * n)
    finally:
        if env_keep is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = env_keep
    solves = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return solves / wall, n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    total_runs = 0
    t_all = 0.0
    desc = ""
    for _ in range(args.warmup):
        cpu_baseline(target_seconds=0.0, sample_systems=1024)
    for _ in range(args.steps):
        v, desc, el = cpu_baseline(target_seconds=min(10.0, 60.0 / max(args.steps, 1)),
                                   sample_systems=4096)
        total_runs += v * el
        t_all += el
    value = total_runs / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_ROWS, "M": M_SYS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU timing

def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("sweep.cu", "sweep_tile.cuh", "arith.cuh", "two_ended.h"):
        with open(os.path.join(ROOT, "paper_2107_05395_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def time_launches(step, stream, steps, warmup):
    """Per-launch CUDA-event durations (ms) of `step` on `stream`, after warm-up."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def profiled_traffic():
    """DRAM bytes per launch of the timed kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "penta_sweep_f64_N1024_M65536.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


# ------------------------------------------------------- the other workloads

def _events_ms(fn, reps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_tri_latency(sb, torch, stream):
    """Tridiagonal backward-Euler solve, N=256, M=1024 (4 MiB): latency per solve
    from a CUDA graph of 100 solves (native FP64 and double-float)."""
    import synth
    w = synth.WORKLOADS["tri_dirichlet"]
    N, M = w["N"], w["M"]
    fac = sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", N, w["r"]))
    rhs = synth.torch_uniform(w["seed"], N, M, -1.0, 1.0, torch.float64, "cuda")
    x = torch.empty_like(rhs)
    out = {}
    for arith in ("native", "df32"):
        sb.sb_autotune(fac, rhs, x, arith=arith)
        sb.sb_solve_batched_ex(fac, rhs, x, arith=arith)  # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            for _ in range(100):
                sb.sb_solve_batched_ex(fac, rhs, x, arith=arith)
        g.replay()
        ms = _events_ms(g.replay, 5, torch.cuda.current_stream()) / 100
        out[arith] = {"us_per_solve": ms * 1e3, "solves_per_s": 1e3 / ms}
    return {"workload": "tri N=256, M=1024, r=0.5, U[-1,1]", **out}


def extra_multigroup(sb, torch, stream):
    """Three tridiagonal groups (N=128/512/2048, r=0.1/0.5/2.0), 2^21 FP32 RHS split
    4:2:1, FP64 solutions: two refinements (FP64 and double-float residual) against
    a single double-float pass, all groups per launch.  Error: max relative L2 on
    256 systems per group against the native FP64 solve of the promoted RHS."""
    import synth
    w = synth.WORKLOADS["multigroup_fp32"]
    Ms = synth.group_split(w["total"], w["ratio"], w["N"])
    facs, rhs, xs, work, ref = [], [], [], [], []
    for g, (N, r, M) in enumerate(zip(w["N"], w["r"], Ms)):
        facs.append(sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", N, r)))
        rhs.append(synth.torch_uniform(w["seed"] + g, N, M, -1.0, 1.0, torch.float32, "cuda"))
        xs.append(torch.empty((N, M), dtype=torch.float64, device="cuda"))
        work.append(torch.empty((N, M), dtype=torch.float32, device="cuda"))
        cols = torch.as_tensor([int(v) for v in __import__("numpy").linspace(0, M - 1, 256)], device="cuda")
        b64 = rhs[-1][:, cols].double().contiguous()
        xr = torch.empty_like(b64)
        sb.sb_solve_batched(facs[-1], b64, xr)
        ref.append((cols, xr))
    elts = sum(N * M for N, M in zip(w["N"], Ms))

    def err():
        worst = []
        for g in range(3):
            cols, xr = ref[g]
            d = xs[g][:, cols] - xr
            worst.append(float((d.norm(dim=0) / xr.norm(dim=0)).max().item()))
        return worst

    out = {"workload": "3 tri groups N=128/512/2048, 2^21 FP32 RHS 4:2:1 -> FP64",
           "elements": elts}
    variants = [("refine2_fp64_residual", dict(arith="native", n_refine=2, residual_arith="native")),
                ("refine2_df32_residual", dict(arith="native", n_refine=2, residual_arith="df32")),
                ("df32_direct", dict(arith="df32", n_refine=0)),
                ("fp32_only", dict(arith="native", n_refine=0))]
    for name, kw in variants:
        fn = lambda: sb.sb_solve_batched_groups(facs, rhs, xs, work=work, **kw)
        fn()
        ms = _events_ms(fn, 3, torch.cuda.current_stream())
        out[name] = {"ms_per_call": ms, "launches": 1,  # every pass of every group in one launch
                     "algorithmic_gbs": 12.0 * elts / (ms * 1e-3) / 1e9, "max_rel_err_per_group": err()}
    return out


def extra_cahn_hilliard(sb, torch, stream):
    """Cahn-Hilliard, N=256, 2^20 simulations: ms per step for the fused + graphed
    step (FP64 and double-float), the unfused two-kernel step, and the FP32 sweeps +
    2 refinement passes step (with its error against the FP64 step)."""
    import synth
    w = synth.WORKLOADS["cahn_hilliard"]
    N, M = w["N"], w["M"]
    st = sb.sb_stepper_create("cahn_hilliard", "be", "noflux", N, w["gamma"], w["dt"])
    C = synth.torch_uniform(w["seed"], N, M, -w["amp"], w["amp"], torch.float64, "cuda")
    work = torch.empty_like(C)
    out = {"workload": "CH N=256, M=2^20, gamma'=16.6, dt'=1e-3 (64 steps timed)"}
    for name, arith, mode in (("fused_graph_fp64", "native", "graph"), ("fused_graph_df32", "df32", "graph"),
                              ("unfused_fp64", "native", "unfused"), ("unfused_df32", "df32", "unfused")):
        sb.sb_stepper_run(st, C, 64, arith=arith, mode=mode, work=work)
        ms = _events_ms(lambda: sb.sb_stepper_run(st, C, 64, arith=arith, mode=mode, work=work), 2,
                        torch.cuda.current_stream()) / 64
        out[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms,
                     "algorithmic_gbs": 16.0 * N * M / (ms * 1e-3) / 1e9}
    # FP32 sweeps + 2 refinement passes per step (FP64 or double-float residual),
    # against the fused FP64 step from the same state after 64 steps
    rwork = torch.empty(sb.sb_stepper_refined_workspace_bytes(st, M), dtype=torch.uint8, device="cuda")
    C64 = C.clone()
    sb.sb_stepper_run(st, C64, 64)
    for name, res in (("fp32_refine2_fp64res", "native"), ("fp32_refine2_df32res", "df32")):
        Cr = C.clone()
        sb.sb_stepper_run_refined(st, Cr, 64, rwork, n_refine=2, residual_arith=res)
        err = float(((Cr - C64).norm(dim=0) / C64.norm(dim=0)).max().item())
        ms = _events_ms(lambda: sb.sb_stepper_run_refined(st, Cr, 64, rwork, n_refine=2, residual_arith=res), 2,
                        torch.cuda.current_stream()) / 64
        out[name] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms,
                     "max_rel_l2_vs_fp64_after_64_steps": err}
        del Cr
    del C64, rwork
    return out


def extra_periodic_cn(sb, torch, stream):
    """The paper's own tridiagonal benchmark (Table 1): 1000 Crank-Nicolson steps of
    1D periodic diffusion (sections 3.2-3.3), M = 2^16 systems, N = 64, 256, 1024,
    here in FP64 with the right-hand side built inside the fused step and the
    Sherman-Morrison correction inside the sweep, 64-step CUDA graphs.  The paper's
    V100 seconds (which include its separate stencil kernel) are quoted as context."""
    import synth
    paper_v100_s = {64: 1.278, 256: 5.015, 1024: 20.268}  # Table 1, M = 2^16 rows
    M, steps, sigma = 1 << 16, 1000, 0.5
    out = {"workload": "periodic CN diffusion, M=2^16, 1000 steps, sigma=0.5, U[-1,1], FP64"}
    for N in (64, 256, 1024):
        st = sb.sb_stepper_create("diffusion", "cn", "periodic", N, sigma, 0.0)
        C = synth.torch_uniform(11, N, M, -1.0, 1.0, torch.float64, "cuda")
        sb.sb_stepper_run(st, C, 64)  # builds the graph
        ms = _events_ms(lambda: sb.sb_stepper_run(st, C, steps), 1, torch.cuda.current_stream())
        out[f"N{N}"] = {"s_per_1000_steps": ms * 1e-3 * 1000 / steps, "ms_per_step": ms / steps,
                        "algorithmic_gbs": 16.0 * N * M / (ms / steps * 1e-3) / 1e9,
                        "paper_v100_s_per_1000_steps": paper_v100_s[N]}
        del C
    return out


def extra_coarsening(sb, torch, stream):
    """Section 5.3's batched coarsening study with the paper's periodic ends, on both
    of its domains: L = 2 pi (N = 256) and L = 4 pi (N = 512), dx = 2 pi / 256,
    gamma = 0.01, dt = 0.1 dx, T = 100 (40 744 steps), C(x, 0) ~ U[-0.1, 0.1];
    OPTIONS["coarsening_systems"] simulations (the paper: 2^20).  ell(t) is recorded
    after every step; reported: the run time and the correlation coefficient r of
    the least-squares line ell(t) ~ log t (the paper: r = 0.9989 and 0.9996)."""
    import math
    import numpy as np
    import synth
    M = OPTIONS["coarsening_systems"]
    dx = 2.0 * math.pi / 256
    gamma_grid = 0.01 / dx ** 2
    dt_phys = 0.1 * dx
    dt_grid = dt_phys / dx ** 2
    steps = int(round(100.0 / dt_phys))
    t = dt_phys * np.arange(1, steps + 1)
    out = {"workload": f"periodic CH, dx=2pi/256, gamma=0.01, dt=0.1dx, T=100 ({steps} steps), "
                       f"M={M}, C0~U[-0.1,0.1], FP64 (fused steps, ell reduced every step)"}
    for name, N, paper_r in (("L_2pi", 256, 0.9989), ("L_4pi", 512, 0.9996)):
        st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, gamma_grid, dt_grid)
        C = synth.torch_uniform(4, N, M, -0.1, 0.1, torch.float64, "cuda")
        ell = torch.zeros(steps, dtype=torch.float64, device="cuda")
        work = torch.empty(M + 256, dtype=torch.float64, device="cuda")
        ms = _events_ms(lambda: sb.sb_stepper_run_coarsening(st, C, steps, ell, work), 1,
                        torch.cuda.current_stream())
        e = ell.cpu().numpy()
        r = {"N": N, "s_total": ms / 1e3, "ms_per_step": ms / steps,
             "finite": bool(np.all(np.isfinite(e))),
             "ell_at_t": {str(tt): float(e[int(round(tt / dt_phys)) - 1]) for tt in (1, 10, 50, 100)}}
        for lo in (1.0, 10.0):
            sel = t >= lo
            r[f"r_log_fit_t{int(lo)}_100"] = float(np.corrcoef(np.log(t[sel]), e[sel])[0, 1])
        r["paper_r"] = paper_r
        out[name] = r
        del C, ell, work
        torch.cuda.empty_cache()
    return out


def extra_convergence(sb, torch, stream):
    """The paper's convergence study of the periodic CH scheme (section 5.2, Table 3):
    gamma = 0.01, L = 2 pi, dt = 0.1 dx, C(x, 0) = 1e-6 cos(5 x), T = 20, one
    simulation per grid, N = 64 .. OPTIONS["table3_max_n"].  E_N = mean over the N/2
    shared points of |C^(N/2) - C^(N)|, with the paper's printed E_N beside it."""
    import math
    import numpy as np
    import synth
    paper = {128: (0.0310, 3.7932), 256: (0.0022, 2.0376), 512: (5.45e-4, 2.0089),
             1024: (1.35e-4, 2.0022), 2048: (3.38e-5, 2.0005), 4096: (8.45e-6, 0.8947),
             8192: (4.54e-6, None)}
    Ns = [n for n in synth.WORKLOADS["ch_convergence"]["N"] if n <= OPTIONS["table3_max_n"]]
    runs, secs = {}, {}
    for N in Ns:
        gamma, dt, steps, _, C0 = synth.ch_convergence_case(N)
        st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, gamma, dt)
        d = torch.from_numpy(np.ascontiguousarray(C0)).cuda()
        secs[N] = _events_ms(lambda: sb.sb_stepper_run(st, d, steps), 1, torch.cuda.current_stream()) / 1e3
        runs[N] = d.cpu().numpy()[:, 0]
    rows = {}
    for N in Ns[1:]:
        e = float(np.mean(np.abs(runs[N // 2] - runs[N][::2])))
        rows[N] = {"E_N": e, "paper_E_N": paper[N][0], "s_run": secs[N]}
    for N in Ns[1:-1]:
        rows[N]["order"] = math.log2(rows[N]["E_N"] / rows[2 * N]["E_N"])
        rows[N]["paper_order"] = paper[N][1]
    return {"workload": "periodic CH, L=2pi, gamma=0.01, dt=0.1dx, C0=1e-6 cos(5x), T=20, M=1, FP64",
            "rows": {str(k): v for k, v in rows.items()}}


def extra_forced(sb, torch, stream):
    """The travelling-wave forced CH scheme of section 6.1 (WENO advection and forcing
    fused into the periodic CH step): (a) the paper's forced convergence study
    (Table 4) on N = 128 .. OPTIONS["table3_max_n"], one simulation per grid, with the
    printed E_N beside ours; (b) the flow-pattern batch of section 6.3: N = 512 on
    L = 2 pi, 768 x 768 = 589 824 simulations over f0 in [0, 2] and <C> in [0, 1.5],
    k = 1, v = 0.5, gamma = 0.01, dt = 0.1 dx, C0 = <C> + U[-0.1, 0.1]: the time per
    step over 2 graphs of 64 steps, and that rate applied to the paper's T = 50."""
    import math
    import numpy as np
    import synth
    out = {}
    w = synth.WORKLOADS["forced_ch_convergence"]
    paper = {256: (0.0013, 2.8363), 512: (1.8e-4, 1.9869), 1024: (4.54e-5, 2.0086), 2048: (1.13e-5, 1.9673),
             4096: (2.88e-5, None)}
    Ns = [n for n in w["N"] if n <= OPTIONS["table3_max_n"]]
    runs = {}
    for N in Ns:
        gamma, dt, steps, dtp, C0 = synth.forced_ch_convergence_case(N)
        dx = 2.0 * math.pi / N
        st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, gamma, dt)
        sb.sb_stepper_set_forcing(st, dtp * w["v"] / dx, dtp * w["k"] * np.cos(w["k"] * dx * np.arange(N)))
        d = torch.from_numpy(np.ascontiguousarray(C0)).cuda()
        a = torch.full((1,), w["f0"], dtype=torch.float64, device="cuda")
        sb.sb_stepper_run_forced(st, d, a, steps)
        runs[N] = d.cpu().numpy()[:, 0]
    rows = {}
    for N in Ns[1:]:
        rows[N] = {"E_N": float(np.mean(np.abs(runs[N // 2] - runs[N][::2]))), "paper_E_N": paper[N][0]}
    for N in Ns[1:-1]:
        rows[N]["order"] = math.log2(rows[N]["E_N"] / rows[2 * N]["E_N"])
        rows[N]["paper_order"] = paper[N][1]
    out["table4"] = {"workload": "forced periodic CH, L=2pi, gamma=0.01, k=1, v=0.5, f0=1, dt=0.1dx, "
                                 "C0=1e-6 cos(5x), T=20, M=1, FP64",
                     "rows": {str(k): v for k, v in rows.items()}}
    m = synth.WORKLOADS["forced_ch_map"]
    N, side = m["N"], m["side"]
    M = side * side
    dx = 2.0 * math.pi / N
    dtp = m["dt_over_dx"] * dx
    st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, m["gamma"] / dx ** 2, dtp / dx ** 2)
    sb.sb_stepper_set_forcing(st, dtp * m["v"] / dx, dtp * m["k"] * np.cos(m["k"] * dx * np.arange(N)))
    f0 = torch.linspace(m["f0"][0], m["f0"][1], side, dtype=torch.float64, device="cuda")
    mean = torch.linspace(m["mean"][0], m["mean"][1], side, dtype=torch.float64, device="cuda")
    amp = f0.repeat_interleave(side).contiguous()          # system a*side + b: f0[a], mean[b]
    C = synth.torch_uniform(m["seed"], N, M, -m["amp"], m["amp"], torch.float64, "cuda")
    C += mean.repeat(side)[None, :]
    sb.sb_stepper_run_forced(st, C, amp, 64)  # warm-up and graph capture
    ms = _events_ms(lambda: sb.sb_stepper_run_forced(st, C, amp, 128), 1, torch.cuda.current_stream()) / 128
    steps_T = int(math.ceil(m["T"] / dtp))
    out["flow_pattern_batch"] = {
        "workload": f"forced periodic CH, N={N}, M={M} (768 x 768 grid of f0 in [0,2], <C> in [0,1.5]), "
                    f"k=1, v=0.5, gamma=0.01, dt=0.1dx, FP64, fused + graph",
        "ms_per_step": ms, "elements_per_s": N * M / (ms / 1e3),
        "projected_s_for_T50": ms * steps_T / 1e3, "steps_T50": steps_T,
        "finite": bool(torch.isfinite(C).all().item())}
    del C, amp
    return out


def _load_cusparse():
    import ctypes
    import glob
    import torch
    names = ["libcusparse.so.12", "libcusparse.so"]
    base = os.path.dirname(os.path.dirname(torch.__file__))
    names += sorted(glob.glob(os.path.join(base, "nvidia", "*", "lib", "libcusparse.so*")))
    names += sorted(glob.glob("/usr/local/cuda*/lib*/libcusparse.so*"))
    for n in names:
        try:
            return ctypes.CDLL(n), n
        except OSError:
            continue
    return None, "libcusparse not found"


def extra_cusparse_context(sb, torch, stream):
    """Same-box context, not a target: cuSPARSE's interleaved batched solvers, which
    need a full copy of the matrix per system (the design the paper's constant-matrix
    kernels replace, section 1): gtsvInterleavedBatch (algorithm 0, no pivoting) on
    the tridiagonal Table 1 shape (N = 1024, M = 2^16, FP64) and gpsvInterleavedBatch
    on the pentadiagonal headline workload (N = 1024, M = 2^16, FP64), each timed per
    solve with CUDA events (the per-system matrix copies are restored before every
    call, outside the timed region), beside this library's shared-matrix solve of the
    same systems."""
    import ctypes
    import numpy as np
    import synth
    lib, where = _load_cusparse()
    if lib is None:
        return {"unavailable": where}
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    h = vp()
    if lib.cusparseCreate(ctypes.byref(h)) != 0:
        return {"unavailable": "cusparseCreate failed"}
    cur = torch.cuda.current_stream()
    lib.cusparseSetStream(h, vp(cur.cuda_stream))
    out = {"library": os.path.basename(where)}
    N, M = 1024, 1 << 16

    def timed(fn, restore, reps=10):
        ts = []
        for _ in range(reps + 2):
            restore()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(cur)
            fn()
            b.record(cur)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts[2:]))

    for kind in ("tri", "penta"):
        if kind == "tri":
            diags = sb.sb_build_matrix("diffusion", N, 0.5)
            fac = sb.sb_factor_shared_tri(*diags)
        else:
            diags = sb.sb_build_matrix("hinged", N, 0.25)
            fac = sb.sb_factor_shared_penta(*diags)
        rhs = synth.torch_normal(SEED, N, M, torch.float64, "cuda")
        full = [torch.from_numpy(np.ascontiguousarray(d)).cuda()[:, None].expand(N, M).contiguous() for d in diags]
        work = [t.clone() for t in full]
        xs = rhs.clone()
        ptr = lambda t: vp(t.data_ptr())

        def restore():
            for w, f in zip(work, full):
                w.copy_(f)
            xs.copy_(rhs)
        size = ctypes.c_size_t()
        if kind == "tri":
            st = lib.cusparseDgtsvInterleavedBatch_bufferSizeExt(h, i32(0), i32(N), ptr(work[0]), ptr(work[1]),
                                                                 ptr(work[2]), ptr(xs), i32(M), ctypes.byref(size))
        else:
            st = lib.cusparseDgpsvInterleavedBatch_bufferSizeExt(h, i32(0), i32(N), ptr(work[0]), ptr(work[1]),
                                                                 ptr(work[2]), ptr(work[3]), ptr(work[4]), ptr(xs),
                                                                 i32(M), ctypes.byref(size))
        if st != 0:
            out[kind] = {"unavailable": f"bufferSizeExt status {st}"}
            continue
        buf = torch.empty(max(1, size.value), dtype=torch.uint8, device="cuda")
        if kind == "tri":
            call = lambda: lib.cusparseDgtsvInterleavedBatch(h, i32(0), i32(N), ptr(work[0]), ptr(work[1]),
                                                             ptr(work[2]), ptr(xs), i32(M), ptr(buf))
        else:
            call = lambda: lib.cusparseDgpsvInterleavedBatch(h, i32(0), i32(N), ptr(work[0]), ptr(work[1]),
                                                             ptr(work[2]), ptr(work[3]), ptr(work[4]), ptr(xs),
                                                             i32(M), ptr(buf))
        ms_lib = timed(call, restore)
        restore()
        call()
        x = torch.empty_like(rhs)
        sb.sb_solve_batched(fac, rhs, x)
        torch.cuda.synchronize()
        agree = float(((xs - x).norm(dim=0) / x.norm(dim=0)).max().item())
        ms_ours = timed(lambda: sb.sb_solve_batched(fac, rhs, x), lambda: None)
        out[kind] = {"workload": f"{'tridiagonal diffusion r=0.5' if kind == 'tri' else 'pentadiagonal hinged r=0.25'}, "
                                 f"N={N}, M=2^16, FP64",
                     "cusparse_routine": "Dgtsv" if kind == "tri" else "Dgpsv",
                     "cusparse_ms_per_solve": ms_lib, "ours_ms_per_solve": ms_ours,
                     "speedup": ms_lib / ms_ours, "max_rel_diff_per_system": agree,
                     "cusparse_matrix_bytes": sum(t.numel() * 8 for t in full)}
        del full, work, xs, buf, x, rhs
        torch.cuda.empty_cache()
    lib.cusparseDestroy(h)
    return out


def extra_rollout(sb, torch, stream):
    """Adjoint rollout, N=512, 2^16 systems, 200 steps, checkpoints every 20 (CH
    and diffusion, FP64): forward and backward step rates against the plain
    per-step solve of the same stepper."""
    import synth
    w = synth.WORKLOADS["adjoint_rollout"]
    N, M, T, k = w["N"], w["M"], w["steps"], w["ckpt_every"]
    out = {"workload": "rollout N=512, M=2^16, 200 steps, ckpt 20, FP64"}
    for kind, p, dt, bc in (("cahn_hilliard", w["gamma"], w["dt"], "noflux"), ("diffusion", w["r"], 0.0, "dirichlet")):
        st = sb.sb_stepper_create(kind, "be", bc, N, p, dt)
        x0 = synth.torch_uniform(w["seed"], N, M, -0.1, 0.1, torch.float64, "cuda")
        work = torch.empty(sb.sb_rollout_workspace_bytes(st, M, T, k) // 8, dtype=torch.float64, device="cuda")
        CT = torch.empty_like(x0)
        g = torch.empty_like(x0)
        gC0 = torch.empty_like(x0)
        dp = torch.zeros((), dtype=torch.float64, device="cuda")
        fwd = lambda: sb.sb_rollout_forward(st, x0, CT, T, k, work)
        bwd = lambda: sb.sb_rollout_backward(st, g, gC0, T, k, work, grad_param=dp)
        fwd()
        g.copy_(CT)
        bwd()
        f_ms = _events_ms(fwd, 1, torch.cuda.current_stream())
        b_ms = _events_ms(bwd, 1, torch.cuda.current_stream())
        C = x0.clone()
        plain = _events_ms(lambda: sb.sb_stepper_run(st, C, 20, mode="direct"), 1,
                           torch.cuda.current_stream()) / 20
        out[kind] = {"forward_ms": f_ms, "backward_ms": b_ms,
                     "forward_steps_per_s": T / (f_ms * 1e-3), "backward_steps_per_s": T / (b_ms * 1e-3),
                     "plain_step_ms": plain, "backward_vs_plain_step": (b_ms / T) / plain}
    return out


def _r(v, digits=4):
    """v rounded to `digits` significant digits (None and non-numbers pass through)."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}")
    return v


def _get(d, *keys):
    for k in keys:
        if not isinstance(d, dict) or k not in d:
            return None
        d = d[k]
    return d


def summary(extras, fp32, df32, cpu, timeouts, link=None, fp64_fma_per_s=None):
    """Compact numeric record of every figure the workload extras report (kept at
    the end of the JSON line): times in ms (table1 in s per 1000 steps), fractions
    of the measured HBM peak, ratios against the plain per-step solve, the host
    link's copy rates (GB/s) beside the end-to-end figure, and the refined
    multi-group solve against its FP64-pipe bound (8 FP64 operations per element:
    3 FMAs per residual row and 1 addition per correction, two passes)."""
    ch = extras.get("cahn_hilliard", {})
    mg = extras.get("multigroup_refine", {})
    ro = extras.get("adjoint_rollout", {})
    fused = _get(ch, "fused_graph_fp64", "ms_per_step")
    out = {
        "fp32_solve_ms": _r(fp32.get("ms_per_solve")), "fp32_hbm_frac": _r(fp32.get("hbm_frac")),
        "fp32_kernel": fp32.get("kernel"),
        "df32_solve_ms": _r(df32.get("ms_per_solve")),
        "tri_latency_us": {k: _r(_get(extras, "tri_latency", k, "us_per_solve")) for k in ("native", "df32")},
        "multigroup_ms": {k: _r(_get(mg, k, "ms_per_call"))
                          for k in ("refine2_fp64_residual", "refine2_df32_residual", "df32_direct", "fp32_only")},
        "multigroup_launches": {k: _get(mg, k, "launches") for k in ("refine2_fp64_residual", "refine2_df32_residual")},
        "multigroup_max_err": _r(max([e for k in ("refine2_fp64_residual", "refine2_df32_residual")
                                      for e in (_get(mg, k, "max_rel_err_per_group") or [])], default=None)),
        "ch_step_ms": {k: _r(_get(ch, k, "ms_per_step"))
                       for k in ("fused_graph_fp64", "fused_graph_df32", "unfused_fp64", "fp32_refine2_fp64res",
                                 "fp32_refine2_df32res")},
        "fused_vs_plain": _r(_get(ch, "unfused_fp64", "ms_per_step") / fused) if fused and
        _get(ch, "unfused_fp64", "ms_per_step") else None,
        "refined_vs_plain": _r(_get(ch, "fp32_refine2_fp64res", "ms_per_step") / fused) if fused and
        _get(ch, "fp32_refine2_fp64res", "ms_per_step") else None,
        "adjoint_vs_plain": {k: _r(_get(ro, k, "backward_vs_plain_step")) for k in ("cahn_hilliard", "diffusion")},
        "rollout_ms": {k: [_r(_get(ro, k, "forward_ms")), _r(_get(ro, k, "backward_ms"))]
                       for k in ("cahn_hilliard", "diffusion")},
        "table1_s": {k: _r(_get(extras, "paper_table1_periodic_cn", k, "s_per_1000_steps"))
                     for k in ("N64", "N256", "N1024")},
        "cusparse_speedup": {k: _r(_get(extras, "cusparse_context", k, "speedup")) for k in ("tri", "penta")},
        "cpu_all_cores": {"value": _r(_get(cpu, "all_cores", "value")), "cores": _get(cpu, "all_cores", "cores")}
        if cpu else None,
        "partition_timeouts": timeouts,
        "host_link_gbs": {k: link.get(k) for k in ("h2d", "d2h", "both")} if link else None,
    }
    elts = mg.get("elements")
    t = _get(mg, "refine2_fp64_residual", "ms_per_call")
    if elts and t and fp64_fma_per_s:
        bound_ms = elts * 8 / fp64_fma_per_s * 1e3
        out["multigroup_fp64_bound_ms"] = _r(bound_ms)
        out["multigroup_of_fp64_bound"] = _r(bound_ms / t)
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_2107_05395_gb300 as sb
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    fac = sb.sb_factor_shared_penta(*sb.sb_build_matrix("hinged", N_ROWS, R_COEF))
    rhs = synth.torch_normal(SEED + 1000 * rank, N_ROWS, M_SYS, torch.float64, "cuda")
    x = torch.empty_like(rhs)
    stream = torch.cuda.current_stream()

    arith = args.arith
    # pick the launch shape of each arithmetic mode with the library's autotuner
    shapes = {}
    for mode in ("native", "df32"):
        if mode == arith and args.shape:
            # a pinned shape (e.g. for a profiler run, whose serialised launches can
            # change the autotuner's ranking)
            shp = tuple(int(v) for v in args.shape.split(","))
            sb.sb_shape_set(fac, shp, arith=mode)
            shapes[mode] = (shp, None)
        else:
            shapes[mode] = sb.sb_autotune(fac, rhs, x, arith=mode)

    def step():
        sb.sb_solve_batched_ex(fac, rhs, x, arith=arith, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    from paper_2107_05395_gb300.distributed import max_over_ranks
    total_ms = max_over_ranks(total_ms, device="cuda")  # the slowest rank's time
    ms_per_step = total_ms / args.steps
    value = world * args.steps / (total_ms / 1e3)

    # end to end through the public API with host buffers (pinned), copies timed
    h_rhs = torch.empty((N_ROWS, M_SYS), dtype=torch.float64, pin_memory=True)
    h_rhs.copy_(rhs)
    h_x = torch.empty_like(h_rhs, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 10))
    # the public host-memory call: chunked H2D / solve / D2H overlapped on the
    # library's internal streams, ordered on `stream`
    hwork = torch.empty(sb.sb_host_workspace_bytes(fac, M_SYS), dtype=torch.uint8, device="cuda")

    def e2e_step():
        sb.sb_solve_batched_host(fac, h_rhs, h_x, hwork, arith=arith, stream=stream)

    # the same workload stored and solved in FP32 (8 B per element): the path whose
    # bound is HBM rather than the FP64 pipe
    rhs32 = rhs.float()
    x32 = torch.empty_like(rhs32)
    n32 = max(5, min(args.steps, 20))
    # each algorithm with its own best shape, then the autotuner's overall choice
    per_algo = {}
    for algo, name in ((sb.SB_ALGO_SEQUENTIAL, "sequential"), (sb.SB_ALGO_PARTITIONED, "partitioned")):
        best = None
        for shp in ([(t, c, 1, algo) for t in (128, 256, 512) for c in (0, 1)] if algo == 0
                    else [(t, 0, 1, algo) for t in (256, 512, 1024)]):
            sb.sb_shape_set(fac, shp, rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32)
            try:
                t = float(np.min(time_launches(lambda: sb.sb_solve_batched(fac, rhs32, x32, stream=stream),
                                               stream, 3, 1)))
            except sb.SbError:
                continue
            if best is None or t < best[1]:
                best = (shp, t)
        if best is not None:
            sb.sb_shape_set(fac, best[0], rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32)
            ms = float(np.mean(time_launches(lambda: sb.sb_solve_batched(fac, rhs32, x32, stream=stream),
                                             stream, n32, 3)))
            per_algo[name] = {"shape": list(best[0]), "ms_per_solve": ms,
                              "hbm_frac": 8.0 * N_ROWS * M_SYS / (ms / 1e3) / 1e9 / hbm_peak()[0]}
    shape32 = sb.sb_autotune(fac, rhs32, x32)
    ms32 = time_launches(lambda: sb.sb_solve_batched(fac, rhs32, x32, stream=stream), stream, n32, 3)
    s32 = float(np.mean(ms32)) / 1e3
    timeouts = sb.sb_device_timeouts(local)  # partitioned CTAs that gave up waiting (must be 0)
    fp32_extra = {"shape": list(shape32[0]), "ms_per_solve": s32 * 1e3,
                  "kernel": ({256: "part_kernel2s (two systems per thread, stores spread through TMEM)",
                              512: "part_kernel", 1024: "part_kernel"}.get(shape32[0][0], "part_kernel")
                             if shape32[0][3] == sb.SB_ALGO_PARTITIONED else "sweep_kernel"),
                  "timeouts": timeouts,
                  "batched_solves_per_s": 1.0 / s32,
                  "hbm_gbs": 8.0 * N_ROWS * M_SYS / s32 / 1e9,
                  "hbm_frac": 8.0 * N_ROWS * M_SYS / s32 / 1e9 / hbm_peak()[0],
                  "by_algorithm": per_algo}
    del rhs32, x32

    # the other arithmetic mode on the same workload, timed the same way
    other = "native" if arith == "df32" else "df32"
    other_ms = time_launches(lambda: sb.sb_solve_batched_ex(fac, rhs, x, arith=other, stream=stream),
                             stream, max(5, min(args.steps, 20)), 3)

    e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, device="cuda")

    # the host link on this machine, for reading e2e: the same pinned buffers copied
    # whole, one direction at a time and both at once (copy engines, no kernel)
    def link_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        for _ in range(reps):
            fn()
        l1.record(stream)
        torch.cuda.synchronize()
        return l0.elapsed_time(l1) / reps

    side = torch.cuda.Stream()

    def both():
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            h_x.copy_(x, non_blocking=True)
        with torch.cuda.stream(stream):
            rhs.copy_(h_rhs, non_blocking=True)
        stream.wait_stream(side)

    with torch.cuda.stream(stream):
        nbytes = N_ROWS * M_SYS * 8
        link = {"h2d": nbytes / link_ms(lambda: rhs.copy_(h_rhs, non_blocking=True)) / 1e6,
                "d2h": nbytes / link_ms(lambda: h_x.copy_(x, non_blocking=True)) / 1e6,
                "both": 2 * nbytes / link_ms(both) / 1e6}
    link = {k: round(v, 1) for k, v in link.items()}
    link["e2e_bound_solves_per_s"] = round(link["both"] * 1e9 / (2 * nbytes), 1)

    extras = {}
    # the paper-workload extras run on one GPU (a multi-GPU run measures the scaling
    # of the headline step only, unless extras are named explicitly)
    if not args.no_extras and (world == 1 or OPTIONS["extras"]):
        for name, fn in (("tri_latency", extra_tri_latency), ("multigroup_refine", extra_multigroup),
                         ("cahn_hilliard", extra_cahn_hilliard), ("adjoint_rollout", extra_rollout),
                         ("paper_table1_periodic_cn", extra_periodic_cn), ("coarsening", extra_coarsening),
                         ("paper_table3_convergence", extra_convergence), ("forced_ch", extra_forced),
                         ("cusparse_context", extra_cusparse_context)):
            if OPTIONS["extras"] and name not in OPTIONS["extras"]:
                continue
            try:
                extras[name] = fn(sb, torch, stream)
            except Exception as exc:  # report, do not hide, a failing extra
                extras[name] = {"error": repr(exc)}
            torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    rates = sb.sb_measure_rates(local)  # the FP64 pipe's measured ceiling
    fp64_peak = 2.0 * rates["fp64_fma_per_s"] / 1e12
    avg_launch_s = float(np.mean(launch_ms)) / 1e3
    elts = N_ROWS * M_SYS
    flops = FLOPS_PER_ELT * elts
    achieved_tflops = flops / avg_launch_s / 1e12
    hbm, hbm_src = hbm_peak()
    achieved_gbs = BYTES_PER_ELT * elts / avg_launch_s / 1e9
    traffic = profiled_traffic()

    def headline_kernel(policy, what):
        # the kernel the autotuner's shape for this arithmetic launches
        shp = shapes[arith][0]
        if shp[3] == sb.SB_ALGO_TWO_ENDED:
            return (f"sweep_two_ended_kernel<P=2> ({what}; each system eliminated from both ends, "
                    f"16 systems per warp, {shp[0]} threads)")
        if shp[3] == sb.SB_ALGO_STAGED:
            return f"sweep_staged_kernel<{policy},P=2> ({what}; rows staged through shared memory, {shp[0]} threads)"
        return f"sweep_kernel<{policy},P=2> ({what}; {shp[0]} threads, {shp[2]} system(s) per thread)"

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, desc, _ = cpu_baseline()
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        try:
            va, na = cpu_baseline_all_cores()
            cpu["all_cores"] = {"value": va, "unit": UNIT, "cores": na,
                                "sample": "one process per core, each the oracle on 2048 of the systems "
                                          "for ~6 s, scaled to the full batch"}
        except Exception as exc:  # report, do not hide
            cpu["all_cores"] = {"error": repr(exc)}
    other_s = float(np.mean(other_ms)) / 1e3
    if arith == "df32":
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                "frac": achieved_gbs / hbm, "traffic": traffic,
                "kernel": headline_kernel("DFArith", "double-float arithmetic, FP64 I/O"),
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)",
                "alu_fp64_equiv": {"achieved": achieved_tflops, "unit": "TFLOP/s"}}
        dtype = "f64 (double-float arithmetic)"
    else:
        roof = {"bound": "alu", "achieved": achieved_tflops, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved_tflops / fp64_peak,
                "traffic": traffic,
                "kernel": headline_kernel("NativeArith<double>", "native FP64"),
                "peak_source": "measured: sb_measure_rates FP64 FMA throughput x 2 flop, this run "
                               f"(derived nominal {FP64_PEAK_TFLOPS:.3f} TFLOP/s = 2 FMA/clk/SM x 152 SMs x 2.07 GHz)",
                "rates": {k: rates[k] for k in ("fp64_fma_per_s", "fp32_fma_per_s", "f64_f32_conversions_per_s")},
                "hbm": {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                        "frac": achieved_gbs / hbm, "peak_source": hbm_src}}
        dtype = "f64"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_ROWS, "M": M_SYS, "closure": "hinged",
                   "r": R_COEF, "arith": arith, "l2": "inputs (2 x 512 MiB) exceed L2; no flush",
                   "shape": {"threads_ctas_per_sm_spt_algo": list(shapes[arith][0]),
                             "autotune_ms": shapes[arith][1]},
                   "parallelism": f"replicas x{world} (independent batches)"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": world * 1e3 / e2e_ms, "unit": UNIT,
                "h2d_bytes_per_step": elts * 8, "d2h_bytes_per_step": elts * 8,
                "host_link_gbs": link},
        "extras": {
            **extras,
            "solve_fp32": fp32_extra,
            f"solve_{other}": {"shape": list(shapes[other][0]),
                               "ms_per_solve": float(np.mean(other_ms)),
                               "batched_solves_per_s": 1.0 / other_s,
                               "hbm_gbs": BYTES_PER_ELT * elts / other_s / 1e9},
        },
        "gpu_launches": args.steps,
        "clocks": clocks,
        "launch_ms": {"mean": float(np.mean(launch_ms)), "min": float(np.min(launch_ms)),
                      "max": float(np.max(launch_ms))},
    }
    # last key of the line: the compact record of every extra's figures
    line["summary"] = summary(extras, fp32_extra, line["extras"][f"solve_{other}"] if other == "df32" else {},
                              cpu, timeouts, link, rates["fp64_fma_per_s"])
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--arith", choices=["native", "df32"], default="native")
    ap.add_argument("--no-extras", action="store_true", help="time the headline workload only")
    ap.add_argument("--shape", default="",
                    help="threads,ctas_per_sm,systems_per_thread,algorithm of the headline solve instead of "
                         "the autotuner's choice")
    ap.add_argument("--extras", default="", help="comma-separated names of the extras to run (default: all)")
    ap.add_argument("--coarsening-systems", type=int, default=1 << 16,
                    help="simulations per domain in the coarsening extra (the paper: 1048576)")
    ap.add_argument("--table3-max-n", type=int, default=1024,
                    help="largest grid of the convergence extra (the paper's table: 8192)")
    args = ap.parse_args()
    OPTIONS.update(extras=[e for e in args.extras.split(",") if e], coarsening_systems=args.coarsening_systems,
                   table3_max_n=args.table3_max_n)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
