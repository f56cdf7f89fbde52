"""GPU parity of the FP32 + refinement time steps (sb_stepper_run_refined: the
right-hand side built in FP64, FP32 sweeps, n_refine passes with an FP64 or
double-float residual) against the FP64 oracle's steps: the Cahn-Hilliard workload
(no-flux, N = 256, gamma' = 16.6, dt' = 1e-3) and backward-Euler hyperdiffusion and
diffusion, graph-captured and direct.  Two passes must reach 1e-10 relative L2 per
system; with no pass the FP32 solve alone is ~1e-7, one pass already contracts it;
and the grouped solve accepts FP64 right-hand sides with refinement."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices, steppers
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def oracle_steps(kind, bc, N, coef, dt, C, steps):
    if kind == "cahn_hilliard":
        A = steppers.SharedPenta(*matrices.ch_matrix(N, dt * coef))
        for _ in range(steps):
            C = steppers.ch_step(A, C, dt)
    elif kind == "hyperdiffusion":
        A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, coef, bc))
        for _ in range(steps):
            C = steppers.hyper_be_step(A, C)
    else:
        A = steppers.SharedTri(*matrices.diffusion_matrix(N, coef))
        for _ in range(steps):
            C = steppers.diffusion_be_step(A, C)
    return C


CASES = [
    ("cahn_hilliard", "noflux", 256, synth.CH_GAMMA_GRID, synth.CH_DT_GRID, 0.1, 100),
    ("hyperdiffusion", "hinged", 200, 0.25, 0.0, 1.0, 30),
    ("diffusion", "dirichlet", 300, 0.5, 0.0, 1.0, 30),
]


@pytest.mark.parametrize("kind,bc,N,coef,dt,amp,steps", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("res", ["native", "df32"])
@pytest.mark.parametrize("mode", ["graph", "direct"])
def test_refined_steps_match_oracle(env, kind, bc, N, coef, dt, amp, steps, res, mode):
    sb, torch = env
    M, ld = 333, 340
    st = sb.sb_stepper_create(kind, "be", bc, N, coef, dt)
    C0 = synth.rhs_uniform(seed=N + 7, N=N, M=M, lo=-amp, hi=amp)
    host = np.full((N, ld), 3.25)
    host[:, :M] = C0
    d = to_dev(host, torch)
    work = torch.empty(sb.sb_stepper_refined_workspace_bytes(st, M, ld), dtype=torch.uint8, device="cuda")
    sb.sb_stepper_run_refined(st, d, steps, work, n_refine=2, residual_arith=res, mode=mode, M=M)
    torch.cuda.synchronize()
    out = to_host(d)
    ref = oracle_steps(kind, bc, N, coef, dt, C0, steps)
    err = np.max(relerr_per_system(out[:, :M], ref))
    assert err <= 1e-10, (kind, res, mode, err)
    assert np.all(out[:, M:] == 3.25)


def test_refinement_contracts_per_pass(env):
    sb, torch = env
    N, M = 256, 512
    st = sb.sb_stepper_create("cahn_hilliard", "be", "noflux", N, synth.CH_GAMMA_GRID, synth.CH_DT_GRID)
    C0 = synth.rhs_uniform(seed=3, N=N, M=M, lo=-0.1, hi=0.1)
    ref = oracle_steps("cahn_hilliard", "noflux", N, synth.CH_GAMMA_GRID, synth.CH_DT_GRID, C0, 1)
    work = torch.empty(sb.sb_stepper_refined_workspace_bytes(st, M), dtype=torch.uint8, device="cuda")
    errs = []
    for n_refine in (0, 1, 2):
        d = to_dev(C0, torch)
        sb.sb_stepper_run_refined(st, d, 1, work, n_refine=n_refine, mode="direct")
        torch.cuda.synchronize()
        errs.append(float(np.max(relerr_per_system(to_host(d), ref))))
    assert 1e-9 < errs[0] < 1e-5, errs   # FP32 sweeps alone
    assert errs[1] < errs[0] * 1e-3, errs
    assert errs[2] <= 1e-12, errs


def test_groups_refine_fp64_rhs(env):
    sb, torch = env
    N, M = 128, 1000
    diags = matrices.diffusion_matrix(N, 2.0)
    fac = sb.sb_factor_shared_tri(*diags)
    b = synth.rhs_uniform(seed=5, N=N, M=M)
    x = torch.empty((N, M), dtype=torch.float64, device="cuda")
    work = torch.empty(N * M, dtype=torch.float32, device="cuda")
    sb.sb_solve_batched_groups([fac], [to_dev(b, torch)], [x], n_refine=2, work=[work])
    torch.cuda.synchronize()
    bh, ch = banded.tri_factor(*diags)
    assert np.max(relerr_per_system(to_host(x), banded.tri_solve(diags[0], bh, ch, b))) <= 1e-12


def test_refined_steps_reject_periodic(env):
    sb, torch = env
    st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", 64, 1.0, 0.05)
    d = torch.zeros((64, 32), dtype=torch.float64, device="cuda")
    work = torch.empty(sb.sb_stepper_refined_workspace_bytes(st, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(sb.SbError, match="periodic"):
        sb.sb_stepper_run_refined(st, d, 2, work)
