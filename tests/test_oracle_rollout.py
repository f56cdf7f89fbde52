"""Pins for oracle/rollout.py: the discrete adjoint against central finite
differences (Richardson-extrapolated) on the oracle's own forward rollout, for the
initial condition and the scalar that builds the shared matrix."""
import numpy as np
import pytest

import synth
from oracle import rollout


def fd_directional(fun, h):
    """Richardson-extrapolated central difference of a scalar function of t at 0."""
    def central(hh):
        return (fun(hh) - fun(-hh)) / (2.0 * hh)
    return (4.0 * central(h / 2) - central(h)) / 3.0


def make_case(kind):
    if kind == "diffusion":
        N, M, T = 12, 3, 6
        prob = rollout.diffusion_problem(N, 0.5)
        x0 = synth.rhs_uniform(seed=50, N=N, M=M)
        y = synth.rhs_uniform(seed=51, N=N, M=M)
        builder = lambda p: rollout.diffusion_problem(N, p)
        p0 = 0.5
    elif kind == "hyperdiffusion":
        N, M, T = 14, 3, 6
        prob = rollout.hyperdiffusion_problem(N, 0.25)
        x0 = synth.rhs_uniform(seed=56, N=N, M=M)
        y = synth.rhs_uniform(seed=57, N=N, M=M)
        builder = lambda p: rollout.hyperdiffusion_problem(N, p)
        p0 = 0.25
    elif kind == "ch_grid":
        N, M, T = 16, 3, 6
        prob = rollout.ch_problem(N, synth.CH_GAMMA_GRID, synth.CH_DT_GRID)
        x0 = synth.rhs_uniform(seed=52, N=N, M=M, lo=-0.1, hi=0.1)
        y = synth.rhs_uniform(seed=53, N=N, M=M, lo=-0.1, hi=0.1)
        builder = lambda p: rollout.ch_problem(N, p, synth.CH_DT_GRID)
        p0 = synth.CH_GAMMA_GRID
    else:  # strongly nonlinear: large dt, O(1) amplitude, so J_F matters
        N, M, T = 16, 3, 5
        prob = rollout.ch_problem(N, 1.0, 0.05)
        x0 = synth.rhs_uniform(seed=54, N=N, M=M, lo=-0.9, hi=0.9)
        y = synth.rhs_uniform(seed=55, N=N, M=M, lo=-1.0, hi=1.0)
        builder = lambda p: rollout.ch_problem(N, p, 0.05)
        p0 = 1.0
    return prob, x0, y, T, builder, p0


@pytest.mark.parametrize("kind", ["diffusion", "hyperdiffusion", "ch_grid", "ch_nonlinear"])
def test_adjoint_initial_condition_vs_fd(kind):
    prob, x0, y, T, _, _ = make_case(kind)
    L, gx0, _ = rollout.adjoint(prob, x0, y, T)
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(x0.shape)
        fd = fd_directional(lambda t: rollout.loss(rollout.forward(prob, x0 + t * v, T)[-1], y, x0.shape[1]), 1e-3)
        ad = float(np.sum(gx0 * v))
        assert abs(ad - fd) <= 1e-8 * max(abs(fd), 1e-12) + 1e-14


@pytest.mark.parametrize("kind", ["diffusion", "hyperdiffusion", "ch_grid", "ch_nonlinear"])
def test_adjoint_parameter_vs_fd(kind):
    prob, x0, y, T, builder, p0 = make_case(kind)
    _, _, dp = rollout.adjoint(prob, x0, y, T)
    h = 1e-3 * p0
    fd = fd_directional(lambda t: rollout.loss(rollout.forward(builder(p0 + t), x0, T)[-1], y, x0.shape[1]), h)
    ad = float(np.sum(dp))
    assert abs(ad - fd) <= 1e-8 * abs(fd)


def test_adjoint_subset_of_systems_matches_full_batch():
    """Systems never interact: the per-system gradients of a column subset equal
    those columns of the full-batch gradients (with the same loss normalisation)."""
    prob, x0, y, T, _, _ = make_case("ch_grid")
    _, g_full, dp_full = rollout.adjoint(prob, x0, y, T)
    cols = [0, 2]
    _, g_sub, dp_sub = rollout.adjoint(prob, x0[:, cols], y[:, cols], T, M_total=x0.shape[1])
    assert np.array_equal(g_sub, g_full[:, cols])
    # the per-system reduction over rows may pair terms differently for other widths
    assert np.allclose(dp_sub, dp_full[cols], rtol=1e-14, atol=0)


def test_planted_wrong_sign_is_caught():
    """A sign error in the parameter term (dL/dp += instead of -=) must fail the
    finite-difference pin."""
    prob, x0, y, T, builder, p0 = make_case("diffusion")
    _, _, dp = rollout.adjoint(prob, x0, y, T)
    fd = fd_directional(lambda t: rollout.loss(rollout.forward(builder(p0 + t), x0, T)[-1], y, x0.shape[1]), 1e-3)
    assert abs(-float(np.sum(dp)) - fd) > 1e-3 * abs(fd)
