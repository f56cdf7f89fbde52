"""GPU parity of the travelling-wave forced Cahn-Hilliard stepper (section 6.1:
periodic CH plus adv * W(C) + amp_m g_i on the right-hand side, W the fifth-order
Hamilton-Jacobi WENO derivative) against the oracle on the same seeded inputs:
both stencil sides (sign of adv), graph-captured and direct runs, per-system
amplitudes, ragged tiles with padding canaries, the smallest periodic N, large N
(factors read from device memory), and the paper's printed convergence study of
the forced scheme (Table 4).  FP64 tolerance 1e-12 relative L2 per system."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import matrices, steppers
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

CANARY = 7.25
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table4.json")


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def oracle_forced(N, gamma, dt, adv, amp, g, C, steps):
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, dt * gamma))
    for _ in range(steps):
        C = steppers.forced_ch_step_periodic(A, C, dt, adv, amp, g)
    return C


@pytest.mark.parametrize("N,M", [(5, 3), (7, 40), (64, 45), (300, 97)])
@pytest.mark.parametrize("adv", [0.05, -0.05, 0.0])
@pytest.mark.parametrize("mode", ["graph", "direct"])
def test_forced_stepper_matches_oracle(env, N, M, adv, mode):
    sb, torch = env
    # a strongly nonlinear regime that stays bounded (|C| < 2) over the run; adv = 0.05
    # is the paper's dt v / dx (0.1 x 0.5)
    gamma, dt, steps = 1.0, 0.02, 70
    ld = M + 3
    st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, gamma, dt)
    g = dt * np.cos(2 * math.pi * np.arange(N) / N)
    sb.sb_stepper_set_forcing(st, adv, g)
    amp = np.linspace(0.0, 1.0, M)
    C0 = synth.rhs_uniform(seed=N + 3, N=N, M=M, lo=-0.5, hi=0.5) + np.linspace(0.0, 0.3, M)[None, :]
    host = np.full((N, ld), CANARY)
    host[:, :M] = C0
    d = to_dev(host, torch)
    a = to_dev(amp, torch)
    sb.sb_stepper_run_forced(st, d, a, steps, mode=mode, M=M)
    torch.cuda.synchronize()
    out = to_host(d)
    ref = oracle_forced(N, gamma, dt, adv, amp, g, C0, steps)
    err = np.max(relerr_per_system(out[:, :M], ref))
    assert err <= 1e-12, (N, M, adv, mode, err)
    assert np.all(out[:, M:] == CANARY)


def test_forced_stepper_large_n(env):
    """N = 2400: the coefficient rows exceed shared memory and are read from device
    memory."""
    sb, torch = env
    N, M, steps, gamma, dt, adv = 2400, 64, 12, 1.0, 0.05, 0.4
    st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, gamma, dt)
    g = dt * np.cos(2 * math.pi * 3 * np.arange(N) / N)
    sb.sb_stepper_set_forcing(st, adv, g)
    amp = np.linspace(0.5, 1.5, M)
    C0 = synth.rhs_uniform(seed=12, N=N, M=M, lo=-0.9, hi=0.9)
    d = to_dev(C0, torch)
    sb.sb_stepper_run_forced(st, d, to_dev(amp, torch), steps)
    torch.cuda.synchronize()
    ref = oracle_forced(N, gamma, dt, adv, amp, g, C0, steps)
    assert np.max(relerr_per_system(to_host(d), ref)) <= 1e-12


def test_forced_stepper_rejections(env):
    sb, torch = env
    st = sb.sb_stepper_create("cahn_hilliard", "be", "noflux", 32, 1.0, 0.05)
    with pytest.raises(sb.SbError):
        sb.sb_stepper_set_forcing(st, 0.1, np.zeros(32))
    st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", 32, 1.0, 0.05)
    sb.sb_stepper_set_forcing(st, 0.1, np.zeros(32))
    d = torch.zeros((32, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(sb.SbError, match="sb_stepper_run_forced"):
        sb.sb_stepper_run(st, d, 3)
    plain = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", 32, 1.0, 0.05)
    with pytest.raises(sb.SbError, match="no forcing"):
        sb.sb_stepper_run_forced(plain, d, torch.zeros(8, dtype=torch.float64, device="cuda"), 3)


def forced_gpu_run(sb, torch, N):
    w = synth.WORKLOADS["forced_ch_convergence"]
    gamma, dt, steps, dtp, C0 = synth.forced_ch_convergence_case(N)
    dx = 2 * math.pi / N
    st = sb.sb_stepper_create("cahn_hilliard", "be", "periodic", N, gamma, dt)
    sb.sb_stepper_set_forcing(st, dtp * w["v"] / dx, dtp * w["k"] * np.cos(w["k"] * dx * np.arange(N)))
    d = to_dev(C0, torch)
    sb.sb_stepper_run_forced(st, d, torch.full((1,), w["f0"], dtype=torch.float64, device="cuda"), steps)
    torch.cuda.synchronize()
    return to_host(d)[:, 0].copy()


def test_table4_forced_convergence(env):
    """Table 4 under the Table 3 reading: E_256 = 0.0013 and E_512 = 1.8e-4 to the
    printed digits; E_1024 within 1 % of the printed 4.54e-5 and the orders within
    0.01 of the printed ones (the paper's remaining digits are not reproduced; its
    E_4096 = 2.88e-5 contradicts its own order 1.9673, which implies 2.88e-6)."""
    sb, torch = env
    rows = {int(r[0]): r for r in json.load(open(GOLDEN))["rows"]}
    runs = {N: forced_gpu_run(sb, torch, N) for N in (128, 256, 512, 1024)}
    E = {N: steppers.convergence_error(runs[N // 2], runs[N]) for N in (256, 512, 1024)}
    assert abs(E[256] - rows[256][1]) <= 0.5e-4, E
    assert abs(E[512] - rows[512][1]) <= 0.5e-5, E
    assert abs(E[1024] / rows[1024][1] - 1.0) <= 0.01, E
    for N in (256, 512):
        assert abs(math.log2(E[N] / E[2 * N]) - rows[N][2]) <= 0.01, (N, E)
