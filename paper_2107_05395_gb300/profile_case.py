"""Runs a few launches of one solver kernel on a chosen size, for profilers.

    python -m paper_2107_05395_gb300.profile_case --kind penta --N 1024 --M 32768 --launches 3
    python -m paper_2107_05395_gb300.profile_case --kind forced_ch --N 512 --M 65536 --launches 3
    python -m paper_2107_05395_gb300.profile_case --kind ch_step --step refined --N 256 --M 65536 --launches 3
    python -m paper_2107_05395_gb300.profile_case --kind groups --total 131072 --launches 3

Everything goes through the C ABI; inputs are seeded N(0, 1) drawn on the device.
The default case keeps the inputs above the L2 size (so DRAM counters mean
something) while holding well under a GB on the device.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", choices=["tri", "penta", "forced_ch", "ch_step", "groups"], default="penta")
    ap.add_argument("--step", choices=["fp64", "refined"], default="fp64",
                    help="ch_step: the fused FP64 step or the FP32 + 2 refinements step")
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--M", type=int, default=32768)
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--arith", choices=["native", "df32"], default="native")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--total", type=int, default=131072,
                    help="groups: right-hand sides over the three tridiagonal groups (N = 128/512/2048, 4:2:1)")
    ap.add_argument("--n-refine", type=int, default=2, help="groups: correction passes")
    ap.add_argument("--residual", choices=["native", "df32"], default="native", help="groups: residual arithmetic")
    ap.add_argument("--autotune", action="store_true", help="pick the launch shape first")
    ap.add_argument("--shape", default=None, help="threads,ctas_per_sm,systems_per_thread[,algorithm]")
    args = ap.parse_args()

    import torch

    import paper_2107_05395_gb300 as sb
    import synth

    dt = torch.float64 if args.dtype == "f64" else torch.float32
    if args.kind == "forced_ch":
        # one direct (ungraphed) launch per step of the travelling-wave forced CH
        # scheme with the flow-pattern batch's parameters (k = 1, v = 0.5, gamma = 0.01,
        # dt = 0.1 dx on L = 2 pi), amplitudes f0 spread over [0, 2]
        import math
        N, M = args.N, args.M
        dx = 2.0 * math.pi / N
        dtp = 0.1 * dx
        st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, 0.01 / dx ** 2, dtp / dx ** 2)
        sb.sb_stepper_set_forcing(st, dtp * 0.5 / dx, [dtp * math.cos(dx * i) for i in range(N)])
        C = synth.torch_uniform(6, N, M, -0.1, 0.1, torch.float64, "cuda") + 0.5
        amp = torch.linspace(0.0, 2.0, M, dtype=torch.float64, device="cuda")
        sb.sb_stepper_run_forced(st, C, amp, args.launches, mode="direct")
        torch.cuda.synchronize()
        print(f"ok: {args.launches} forced CH steps N={N} M={M}")
        return
    if args.kind == "ch_step":
        # direct (ungraphed) no-flux Cahn-Hilliard steps with the workload's parameters
        w = synth.WORKLOADS["cahn_hilliard"]
        N, M = args.N, args.M
        st = sb.sb_stepper_create("cahn_hilliard", "be", "noflux", N, w["gamma"], w["dt"])
        C = synth.torch_uniform(w["seed"], N, M, -w["amp"], w["amp"], torch.float64, "cuda")
        if args.step == "fp64":
            sb.sb_stepper_run(st, C, args.launches, mode="direct")
        else:
            work = torch.empty(sb.sb_stepper_refined_workspace_bytes(st, M), dtype=torch.uint8, device="cuda")
            sb.sb_stepper_run_refined(st, C, args.launches, work, n_refine=2, mode="direct")
        torch.cuda.synchronize()
        print(f"ok: {args.launches} {args.step} CH steps N={N} M={M}")
        return
    if args.kind == "groups":
        # the multi-group mixed-precision workload at a chosen total batch: FP32
        # right-hand sides U(-1, 1), FP64 solutions, one launch for every pass
        w = synth.WORKLOADS["multigroup_fp32"]
        Ms = synth.group_split(args.total, w["ratio"], w["N"])
        facs, rhs, xs, work = [], [], [], []
        for g, (N, r, M) in enumerate(zip(w["N"], w["r"], Ms)):
            facs.append(sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", N, r)))
            rhs.append(synth.torch_uniform(w["seed"] + g, N, M, -1.0, 1.0, torch.float32, "cuda"))
            xs.append(torch.empty((N, M), dtype=torch.float64, device="cuda"))
            work.append(torch.empty((N, M), dtype=torch.float32, device="cuda"))
        for _ in range(args.launches):
            sb.sb_solve_batched_groups(facs, rhs, xs, work=work, n_refine=args.n_refine,
                                       residual_arith=args.residual)
        torch.cuda.synchronize()
        print(f"ok: {args.launches} grouped solves, {args.n_refine} refinements ({args.residual} residual), "
              f"batches {list(Ms)}")
        return
    if args.kind == "tri":
        fac = sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", args.N, 0.5))
    else:
        fac = sb.sb_factor_shared_penta(*sb.sb_build_matrix("hinged", args.N, 0.25))
    rhs = synth.torch_normal(2, args.N, args.M, dt, "cuda")
    x = torch.empty_like(rhs)
    if args.shape:
        sb.sb_shape_set(fac, tuple(int(v) for v in args.shape.split(",")), arith=args.arith,
                        rhs_dtype=sb.SB_F64 if args.dtype == "f64" else sb.SB_F32,
                        x_dtype=sb.SB_F64 if args.dtype == "f64" else sb.SB_F32)
    if args.autotune:
        shape, ms = sb.sb_autotune(fac, rhs, x, transpose=args.adjoint, arith=args.arith)
        print(f"autotuned shape {shape} ({ms:.3f} ms)")
    for _ in range(args.launches):
        sb.sb_solve_batched_ex(fac, rhs, x, transpose=args.adjoint, arith=args.arith)
    torch.cuda.synchronize()
    print(f"ok: {args.launches} launches of {args.kind} N={args.N} M={args.M} {args.dtype}"
          f"{' adjoint' if args.adjoint else ''} {args.arith}")


if __name__ == "__main__":
    main()
