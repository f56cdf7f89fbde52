"""GPU parity of the implicit time steppers (fused right-hand side + sweeps, CUDA
graph, and the unfused two-kernel pipeline) against the oracle's steps, and the
Cahn-Hilliard workload (N = 256, 2^20 simulations, 2000 steps; FP64, double-float
and FP32 sweeps with two refinement passes) on sampled systems with mass
conservation checked on every system."""
import numpy as np
import pytest

import synth
from oracle import matrices, steppers
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def oracle_run(kind, scheme, bc, N, coef, dt, C, nsteps):
    C = C.copy()
    if kind == "diffusion" and bc == "periodic":
        A = steppers.SharedTriPeriodic(*matrices.diffusion_matrix_periodic(N, coef))
        for _ in range(nsteps):
            C = A.solve(C if scheme == "be" else steppers.diffusion_cn_rhs_periodic(N, coef, C))
    elif kind == "diffusion":
        A = steppers.SharedTri(*matrices.diffusion_matrix(N, coef))
        for _ in range(nsteps):
            C = A.solve(C if scheme == "be" else steppers.diffusion_cn_rhs(N, coef, C))
    elif kind == "hyperdiffusion":
        A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, coef, bc))
        for _ in range(nsteps):
            C = A.solve(C if scheme == "be" else steppers.hyper_cn_rhs(N, coef, C, bc))
    else:
        A = steppers.SharedPenta(*matrices.ch_matrix(N, dt * coef))
        for _ in range(nsteps):
            C = steppers.ch_step(A, C, dt)
    return C


CASES = [
    ("diffusion", "be", "dirichlet", 0.5, 0.0, 1.0),
    ("diffusion", "cn", "dirichlet", 0.4, 0.0, 1.0),
    ("diffusion", "be", "periodic", 0.5, 0.0, 1.0),
    ("diffusion", "cn", "periodic", 0.4, 0.0, 1.0),
    ("hyperdiffusion", "be", "hinged", 0.25, 0.0, 1.0),
    ("hyperdiffusion", "cn", "hinged", 0.3, 0.0, 1.0),
    ("hyperdiffusion", "cn", "truncated", 0.3, 0.0, 1.0),
    ("cahn_hilliard", "be", "noflux", synth.CH_GAMMA_GRID, synth.CH_DT_GRID, 0.1),
    ("cahn_hilliard", "be", "noflux", 1.0, 0.05, 0.9),  # strongly nonlinear
]


@pytest.mark.parametrize("mode", ["graph", "direct", "unfused"])
@pytest.mark.parametrize("arith", ["native", "df32"])
@pytest.mark.parametrize("kind,scheme,bc,coef,dt,amp", CASES)
@pytest.mark.parametrize("N", [1, 2, 5, 37])
def test_stepper_matches_oracle(env, kind, scheme, bc, coef, dt, amp, N, arith, mode):
    sb, torch = env
    if bc == "periodic" and N < 3:
        pytest.skip("periodic ends need N >= 3")
    M, ld, nsteps = 300, 301, 70  # 70 steps: one 64-step graph plus direct launches
    st = sb.sb_stepper_create(kind, scheme, bc, N, coef, dt)
    C0 = synth.rhs_uniform(seed=N, N=N, M=M, ld=ld, lo=-amp, hi=amp, pad_value=3.5)
    d = to_dev(C0, torch)
    work = torch.empty_like(d) if mode == "unfused" else None
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())  # the copy to `d` ran on the default stream
    with torch.cuda.stream(stream):
        sb.sb_stepper_run(st, d, nsteps, arith=arith, mode=mode, work=work, M=M, stream=stream)
    torch.cuda.synchronize()
    out = to_host(d)
    ref = oracle_run(kind, scheme, bc, N, coef, dt, C0[:, :M], nsteps)
    # double-float values share FP32's exponent range: below ~1e-38 they flush to
    # zero (N = 1 Crank-Nicolson decays to 1e-67), so for df32 the error is taken
    # relative to max(|ref|, 1e-26), i.e. an absolute 1e-38 is tolerated there
    floor = 1e-26 if arith == "df32" else 0.0
    err = np.linalg.norm(out[:, :M] - ref, axis=0) / np.maximum(np.linalg.norm(ref, axis=0), floor)
    # FP64 holds 1e-12 over the 70 steps.  Double-float re-splits the FP64 state
    # into 47 bits every step; over many steps that error, measured against the
    # slowest surviving mode, can pass 1e-12, so multi-step df32 runs are held to
    # the refined-path bound 1e-10 (single df32 solves hold 1e-12).
    assert np.max(err) <= (1e-12 if arith == "native" else 1e-10)
    assert np.all(out[:, M:] == 3.5), "padding columns were written"


def test_stepper_rejects_bad_arguments(env):
    sb, torch = env
    with pytest.raises(sb.SbError):
        sb.sb_stepper_create("cahn_hilliard", "cn", "noflux", 16, 1.0, 0.1)
    with pytest.raises(sb.SbError):
        sb.sb_stepper_create("diffusion", "be", "noflux", 16, 1.0)
    with pytest.raises(sb.SbError):
        sb.sb_stepper_create("hyperdiffusion", "be", "dirichlet", 16, 1.0)
    st = sb.sb_stepper_create("diffusion", "cn", "dirichlet", 16, 0.3)
    d = torch.zeros((16, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(sb.SbError):  # unfused without workspace
        sb.sb_stepper_run(st, d, 3, mode="unfused")
    small = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sb.SbError):  # workspace too small
        sb.sb_stepper_run(st, d, 3, mode="unfused", work=small)


def _ch_workload(sb, torch, arith, nsteps):
    w = synth.WORKLOADS["cahn_hilliard"]
    N, M = w["N"], w["M"]
    st = sb.sb_stepper_create("cahn_hilliard", "be", "noflux", N, w["gamma"], w["dt"])
    C0 = synth.torch_uniform(w["seed"], N, M, -w["amp"], w["amp"], torch.float64, "cuda")
    mass0 = C0.sum(dim=0)
    C = C0.clone()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())  # C was produced on the default stream
    with torch.cuda.stream(stream):
        sb.sb_stepper_run(st, C, nsteps, arith=arith, mode="graph", stream=stream)
    torch.cuda.synchronize()
    # mass on every system: |sum C_T - sum C_0| / (N max|C_T|)
    drift = ((C.sum(dim=0) - mass0).abs() / (N * C.abs().max(dim=0).values)).max().item()
    cols = np.linspace(0, M - 1, 256).astype(np.int64)
    c0 = to_host(C0[:, torch.as_tensor(cols, device="cuda")])
    cT = to_host(C[:, torch.as_tensor(cols, device="cuda")])
    ref = oracle_run("cahn_hilliard", "be", "noflux", N, w["gamma"], w["dt"], c0, nsteps)
    return relerr_per_system(cT, ref), drift


def test_cahn_hilliard_workload_fp64(env):
    """N = 256, 2^20 simulations, C0 ~ U[-0.1, 0.1], 2000 fused graph steps in FP64:
    256 systems spread over the batch against the oracle, mass on all systems."""
    sb, torch = env
    err, drift = _ch_workload(sb, torch, "native", synth.WORKLOADS["cahn_hilliard"]["steps"])
    assert np.max(err) <= 1e-12, (np.max(err), np.median(err))
    assert drift <= 1e-12, drift


def test_cahn_hilliard_workload_df32(env):
    """The same workload in double-float arithmetic.  About 48 significant bits per
    operation accumulate over 2000 steps, so the bound is the refined-path target
    of 1e-10 (the FP64 path above holds 1e-12)."""
    sb, torch = env
    err, drift = _ch_workload(sb, torch, "df32", synth.WORKLOADS["cahn_hilliard"]["steps"])
    assert np.max(err) <= 1e-10, (np.max(err), np.median(err))
    assert drift <= 1e-10, drift


def test_cahn_hilliard_workload_fp32_refined(env):
    """The same workload with FP32 sweeps and two refinement passes per step (FP64
    residual, sb_stepper_run_refined, graph-captured): 256 systems spread over the
    batch within 1e-10 of the oracle's FP64 steps after 2000 steps, mass on every
    system within 1e-10."""
    sb, torch = env
    w = synth.WORKLOADS["cahn_hilliard"]
    N, M, nsteps = w["N"], w["M"], w["steps"]
    st = sb.sb_stepper_create("cahn_hilliard", "be", "noflux", N, w["gamma"], w["dt"])
    C0 = synth.torch_uniform(w["seed"], N, M, -w["amp"], w["amp"], torch.float64, "cuda")
    mass0 = C0.sum(dim=0)
    C = C0.clone()
    work = torch.empty(sb.sb_stepper_refined_workspace_bytes(st, M), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        sb.sb_stepper_run_refined(st, C, nsteps, work, n_refine=2, residual_arith="native", stream=stream)
    torch.cuda.synchronize()
    del work
    drift = ((C.sum(dim=0) - mass0).abs() / (N * C.abs().max(dim=0).values)).max().item()
    cols = torch.as_tensor(np.linspace(0, M - 1, 256).astype(np.int64), device="cuda")
    ref = oracle_run("cahn_hilliard", "be", "noflux", N, w["gamma"], w["dt"], to_host(C0[:, cols]), nsteps)
    err = relerr_per_system(to_host(C[:, cols]), ref)
    assert np.max(err) <= 1e-10, (np.max(err), np.median(err))
    assert drift <= 1e-10, drift


def test_periodic_cn_diffusion_modes_and_mean(env):
    """Section 3.2's periodic Crank-Nicolson diffusion (the paper's Table 1 scheme):
    over 100 fused, graphed steps a Fourier mode k is multiplied by
    ((1 - 4 s sin^2(pi k / N)) / (1 + 4 s sin^2(pi k / N)))^100, and each system's
    mean is conserved."""
    sb, torch = env
    N, s_coef, nsteps = 256, 0.3, 100
    modes = [0, 1, 5, 64, 127, 128]
    X = np.concatenate([synth.fourier_mode_block(N, modes, "cos"),
                        synth.fourier_mode_block(N, modes[1:-1], "sin")], axis=1)
    ks = np.asarray(modes + modes[1:-1])
    g = (1.0 - 4.0 * s_coef * np.sin(np.pi * ks / N) ** 2) / (1.0 + 4.0 * s_coef * np.sin(np.pi * ks / N) ** 2)
    st = sb.sb_stepper_create("diffusion", "cn", "periodic", N, s_coef, 0.0)
    d = to_dev(X, torch)
    sb.sb_stepper_run(st, d, nsteps)
    torch.cuda.synchronize()
    assert np.max(np.abs(to_host(d) - X * (g ** nsteps)[None, :])) <= 1e-12
    C0 = synth.rhs_uniform(seed=3, N=N, M=500)
    d = to_dev(C0, torch)
    sb.sb_stepper_run(st, d, nsteps)
    torch.cuda.synchronize()
    assert np.max(np.abs(to_host(d).mean(axis=0) - C0.mean(axis=0))) <= 1e-13


def test_periodic_stepper_rejected_by_rollout(env):
    sb, torch = env
    st = sb.sb_stepper_create("diffusion", "be", "periodic", 64, 0.5, 0.0)
    nbytes = sb.sb_rollout_workspace_bytes(st, 8, 4, 2)
    work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    with pytest.raises(sb.SbError, match="periodic"):
        sb.sb_rollout_forward(st, torch.zeros((64, 8), dtype=torch.float64, device="cuda"),
                              torch.zeros((64, 8), dtype=torch.float64, device="cuda"), 4, 2, work)
