"""Pins of the Hamilton-Jacobi WENO derivative (oracle/advection.py) and of the
travelling-wave forced Cahn-Hilliard step built on it (section 6.1):

* every candidate stencil is exact for cubics, so WENO is exact for cubics whatever
  its weights; the ideal-weight combination is exact for quintics;
* on smooth periodic data the linear scheme converges at fifth order and WENO at
  fourth to fifth, approaching it; across a jump it takes no information from the other side (the weights
  of stencils that cross it are ~1e-12);
* mirroring the grid swaps the left- and right-biased derivatives and flips the sign;
* a planted mistake (swapped ideal weights) breaks the quintic exactness;
* with no advection and no forcing the forced step is the plain periodic CH step;
* the paper's printed forced convergence study (Table 4): E_256 = 0.0013 and
  E_512 = 1.8e-4 under the reading of Table 3 (`tests/golden/paper_table4.json`);
  the stencil biased the other way gives E_256 of about 6.8e-4, so this also fixes
  the side."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import advection, matrices, steppers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table4.json")


def interior(N):
    return slice(4, N - 4)  # rows whose stencils do not wrap


@pytest.mark.parametrize("side", [-1, 1])
def test_exact_for_cubics(side):
    N = 40
    i = np.arange(N, dtype=np.float64)[:, None]
    rng = np.random.default_rng([1, 2])
    c = rng.uniform(-1, 1, (4, 3))
    phi = c[0] + c[1] * i + c[2] * i ** 2 + c[3] * i ** 3
    exact = c[1] + 2 * c[2] * i + 3 * c[3] * i ** 2
    W = advection.weno5_derivative(phi, side)
    s = interior(N)
    assert np.max(np.abs(W[s] - exact[s])) <= 1e-10 * np.max(np.abs(exact[s]))


@pytest.mark.parametrize("side", [-1, 1])
def test_linear_scheme_exact_for_quintics(side):
    N = 40
    i = np.arange(N, dtype=np.float64)[:, None] / 8.0
    coef = np.array([0.3, -1.1, 0.7, 0.2, -0.05, 0.01])
    phi = sum(cf * i ** k for k, cf in enumerate(coef))
    exact = sum(k * cf * i ** (k - 1) for k, cf in enumerate(coef) if k) / 8.0  # d/d(row)
    L = advection.linear_upwind5_derivative(phi, side)
    s = interior(N)
    assert np.max(np.abs(L[s] - exact[s])) <= 1e-11 * np.max(np.abs(exact[s]))


@pytest.mark.parametrize("side", [-1, 1])
def test_high_order_on_smooth_periodic_data(side):
    """The linear scheme converges at fifth order; WENO follows it at fourth to
    fifth order (its weights depart from the ideal ones at O(h^2) near extrema,
    the known behaviour of these weights), and the two approach each other."""
    eW, eL, dWL = [], [], []
    for N in (32, 64, 128, 256):
        h = 2 * math.pi / N
        x = h * np.arange(N)[:, None]
        phi = np.sin(x) + 0.3 * np.cos(2 * x)
        exact = (np.cos(x) - 0.6 * np.sin(2 * x)) * h  # d/d(row)
        W = advection.weno5_derivative(phi, side)
        L = advection.linear_upwind5_derivative(phi, side)
        eW.append(np.max(np.abs(W - exact)) / h)
        eL.append(np.max(np.abs(L - exact)) / h)
        dWL.append(np.max(np.abs(W - L)) / h)
    order = lambda e: np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert np.all(np.abs(order(eL) - 5.0) < 0.1), order(eL)
    assert np.all(order(eW) > 4.0), order(eW)
    assert np.all(order(dWL) > 4.0), order(dWL)


@pytest.mark.parametrize("side", [-1, 1])
def test_no_information_across_a_jump(side):
    N = 64
    phi = np.where(np.arange(N) < N // 2, 1.0, -1.0)[:, None] + 0.0
    W = advection.weno5_derivative(phi, side)
    far = [i for i in range(N) if min(abs(i - N // 2), abs(i - N // 2 + 1), i, N - 1 - i) >= 4]
    assert np.max(np.abs(W[far])) <= 1e-10
    assert np.all(W[N // 2 - 3: N // 2 + 3] <= 1e-10)  # a descending step: no positive overshoot


def test_mirror_swaps_sides():
    rng = np.random.default_rng([3, 4])
    phi = rng.uniform(-1, 1, (50, 3))
    mir = phi[::-1]
    left = advection.weno5_derivative(phi, -1)
    right_of_mirror = advection.weno5_derivative(mir, +1)[::-1]
    # row i of the mirror is row N-1-i; its forward difference spans rows i, i-1
    assert np.max(np.abs(left + right_of_mirror)) <= 1e-13 * np.max(np.abs(left))


def test_planted_weight_swap_is_caught(monkeypatch):
    orig = advection._candidates_and_weights

    def swapped(*q):
        (p1, p2, p3), w = orig(*q)
        return (p3, p2, p1), w

    monkeypatch.setattr(advection, "_candidates_and_weights", swapped)
    with pytest.raises(AssertionError):
        test_linear_scheme_exact_for_quintics(-1)


def test_forced_step_without_forcing_is_the_ch_step():
    N, M = 48, 5
    C = synth.rhs_uniform(seed=7, N=N, M=M, lo=-0.8, hi=0.8)
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, 0.3))
    plain = steppers.ch_step_periodic(A, C, 0.05)
    forced = steppers.forced_ch_step_periodic(A, C, 0.05, 0.0, np.zeros(M), np.zeros(N))
    assert np.array_equal(plain, forced)
    # forcing alone adds amp_m * A^{-1} g
    g = np.cos(2 * math.pi * np.arange(N) / N)
    amp = np.linspace(0.0, 2.0, M)
    f2 = steppers.forced_ch_step_periodic(A, C, 0.05, 0.0, amp, g)
    assert np.max(np.abs(f2 - plain - A.solve(g[:, None] * amp[None, :]))) <= 1e-13


def forced_run(N):
    w = synth.WORKLOADS["forced_ch_convergence"]
    gamma, dt, steps, dtp, C = synth.forced_ch_convergence_case(N)
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, dt * gamma))
    dx = 2 * math.pi / N
    beta = dtp * w["v"] / dx
    prof = dtp * w["k"] * np.cos(w["k"] * dx * np.arange(N))
    for _ in range(steps):
        C = steppers.forced_ch_step_periodic(A, C, dt, beta, np.array([w["f0"]]), prof)
    return C[:, 0]


@pytest.fixture(scope="module")
def forced_runs():
    return {N: forced_run(N) for N in (128, 256, 512)}


def test_table4_first_rows(forced_runs):
    """E_256 = 0.0013 and E_512 = 1.8e-4 as printed (two significant digits each)."""
    rows = {int(r[0]): r for r in json.load(open(GOLDEN))["rows"]}
    E256 = steppers.convergence_error(forced_runs[128], forced_runs[256])
    E512 = steppers.convergence_error(forced_runs[256], forced_runs[512])
    assert abs(E256 - rows[256][1]) <= 0.5e-4, E256  # printed 0.0013
    assert abs(E512 - rows[512][1]) <= 0.5e-5, E512  # printed 1.8e-4
