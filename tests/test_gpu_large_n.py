"""Large N: when the shared factors do not fit in one CTA's shared memory (penta
FP64 beyond ~4800 rows, periodic penta beyond ~2900, the fused CH step beyond ~2200),
FP64 solves and FP64 fused steps read the single device copy of the factors
directly instead of a staged copy.  Parity with the oracle (FP64, 1e-12 relative
L2 per system), A and A^T, ragged tiles, padding canaries, periodic and
non-periodic matrices, and the fused steppers; the policies that keep only the
staged form (double-float) report SB_ERR_UNSUPPORTED instead of running."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices, steppers
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

CANARY = -3.5


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def solve_both(sb, torch, fac, rhs, M, spt):
    sb.sb_shape_set(fac, (256, 0, spt, 0))
    d = to_dev(rhs, torch)
    outs = []
    for adjoint in (False, True):
        x = torch.full(d.shape, CANARY, dtype=torch.float64, device="cuda")
        sb.sb_solve_batched_ex(fac, d, x, transpose=adjoint, M=M)
        torch.cuda.synchronize()
        outs.append(to_host(x))
    return outs


@pytest.mark.parametrize("kind,N", [("tri", 8000), ("penta", 5000), ("tri_periodic", 6000),
                                    ("penta_periodic", 3000)])
@pytest.mark.parametrize("spt", [1, 2])
def test_large_n_solves_match_oracle(env, kind, N, spt):
    sb, torch = env
    M, ld = 77, 80
    rhs = synth.rhs_normal(seed=N, N=N, M=M, ld=ld, pad_value=CANARY)
    if kind == "tri":
        diags = synth.random_tri_diagonals(3, N)
        fac = sb.sb_factor_shared_tri(*diags)
        bh, ch = banded.tri_factor(*diags)
        ref = [banded.tri_solve(diags[0], bh, ch, rhs[:, :M]), banded.tri_solve_adjoint(diags[0], bh, ch, rhs[:, :M])]
    elif kind == "penta":
        diags = synth.random_penta_diagonals(4, N)
        fac = sb.sb_factor_shared_penta(*diags)
        f = banded.penta_factor(*diags)
        ref = [banded.penta_solve(*f, rhs[:, :M]), banded.penta_solve_adjoint(*f, rhs[:, :M])]
    elif kind == "tri_periodic":
        diags = matrices.diffusion_matrix_periodic(N, 0.7)
        fac = sb.sb_factor_shared_tri_periodic(*diags)
        f = banded.tri_periodic_factor(*diags)
        ref = [banded.tri_periodic_solve(f, rhs[:, :M]), banded.tri_periodic_solve_adjoint(f, rhs[:, :M])]
    else:
        diags = matrices.ch_matrix_periodic(N, 0.3)
        fac = sb.sb_factor_shared_penta_periodic(*diags)
        f = banded.penta_periodic_factor(*diags)
        ref = [banded.penta_periodic_solve(f, rhs[:, :M]), banded.penta_periodic_solve_adjoint(f, rhs[:, :M])]
    outs = solve_both(sb, torch, fac, rhs, M, spt)
    for out, r, name in zip(outs, ref, ("A", "A^T")):
        err = np.max(relerr_per_system(out[:, :M], r))
        assert err <= 1e-12, (kind, N, spt, name, err)
        assert np.all(out[:, M:] == CANARY)


@pytest.mark.parametrize("kind,bc,N,coef,dt,amp", [
    ("cahn_hilliard", "periodic", 2500, 1.0, 0.05, 0.9),
    ("cahn_hilliard", "noflux", 2400, 1.0, 0.05, 0.9),
    ("hyperdiffusion", "hinged", 4000, 0.25, 0.0, 1.0),
])
@pytest.mark.parametrize("mode", ["graph", "unfused"])
def test_large_n_fused_steps_match_oracle(env, kind, bc, N, coef, dt, amp, mode):
    sb, torch = env
    M, steps = 70, 12
    C0 = synth.rhs_uniform(seed=N + 1, N=N, M=M, lo=-amp, hi=amp)
    st = sb.sb_stepper_create(kind, "be", bc, N, coef, dt)
    d = to_dev(C0, torch)
    work = torch.empty(N * M, dtype=torch.float64, device="cuda") if mode == "unfused" else None
    sb.sb_stepper_run(st, d, steps, mode=mode, work=work)
    torch.cuda.synchronize()
    C = C0.copy()
    if kind == "cahn_hilliard" and bc == "periodic":
        A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, dt * coef))
        step = lambda c: steppers.ch_step_periodic(A, c, dt)
    elif kind == "cahn_hilliard":
        A = steppers.SharedPenta(*matrices.ch_matrix(N, dt * coef))
        step = lambda c: steppers.ch_step(A, c, dt)
    else:
        A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, coef, "hinged"))
        step = lambda c: steppers.hyper_be_step(A, c)
    for _ in range(steps):
        C = step(C)
    err = np.max(relerr_per_system(to_host(d), C))
    assert err <= 1e-12, (kind, bc, N, mode, err)


def test_staged_only_policies_report_unsupported(env):
    sb, torch = env
    N, M = 6000, 32
    fac = sb.sb_factor_shared_penta(*synth.random_penta_diagonals(5, N))
    d = to_dev(synth.rhs_normal(seed=1, N=N, M=M), torch)
    x = torch.empty_like(d)
    with pytest.raises(sb.SbError, match="only FP64"):
        sb.sb_solve_batched_ex(fac, d, x, arith="df32")
