"""Pins for oracle/matrices.py and oracle/steppers.py: the paper's printed stencils,
dense matrix products, closed-form eigenmode decay factors, and the Cahn-Hilliard
invariants (constant fixed point, mass conservation, linear growth rate)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import banded, matrices, steppers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_stencils.json")


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def interior_row(diags, i):
    """Row i of a banded matrix as a list over offsets -k..k."""
    k = len(diags) // 2
    return [float(diags[j][i]) for j in range(2 * k + 1)]


# ------------------------------------------------------------ paper stencils

@pytest.mark.parametrize("sigma", [0.1, 0.37, 2.0])
def test_assembled_rows_match_paper_stencils(sigma):
    g = golden()
    N = 16
    i = N // 2

    def printed(name, s):
        e = g[name]
        return [cst + s * co for cst, co in zip(e["const"], e["coef"])]

    assert np.allclose(interior_row(matrices.diffusion_matrix(N, sigma), i),
                       printed("diffusion_cn_lhs", sigma), rtol=0, atol=1e-15)
    assert np.allclose(interior_row(matrices.hyperdiffusion_matrix(N, sigma, "hinged"), i),
                       printed("hyper_cn_lhs", sigma), rtol=0, atol=1e-14)
    assert np.allclose(interior_row(matrices.hyperdiffusion_matrix(N, sigma, "truncated"), i),
                       printed("hyper_cn_lhs", sigma), rtol=0, atol=1e-14)
    assert np.allclose(interior_row(matrices.ch_matrix(N, sigma), i),
                       printed("ch_lhs", sigma), rtol=0, atol=1e-14)
    # right-hand sides: apply to unit vectors and read the stencil of row i
    E = np.eye(N)
    rhs_d = steppers.diffusion_cn_rhs(N, sigma, E)
    assert np.allclose(rhs_d[i, i - 1:i + 2], printed("diffusion_cn_rhs", sigma), atol=1e-15)
    rhs_h = steppers.hyper_cn_rhs(N, sigma, E)
    assert np.allclose(rhs_h[i, i - 2:i + 3], printed("hyper_cn_rhs", sigma), atol=1e-14)


def test_ch_nonlinear_rhs_matches_paper_stencil():
    g = golden()["ch_rhs_nonlinear"]
    alpha = 0.3
    C = synth.rhs_uniform(seed=20, N=12, M=3, lo=-1.2, hi=1.2)
    f = steppers.ch_rhs(C, alpha)
    nl = C ** 3 - C
    for i in range(1, 11):
        stencil = sum(alpha * co * nl[i + off] for off, co in zip(g["offsets"], g["coef"]))
        assert np.allclose(f[i] - C[i], stencil, rtol=1e-13, atol=1e-15)


def test_operators_equal_dense_products():
    for N in (1, 2, 3, 4, 5, 9, 20):
        D2D = matrices.bands_to_dense(*matrices.d2_dirichlet(N))
        D2N = matrices.bands_to_dense(*matrices.d2_noflux(N))
        assert np.array_equal(matrices.bands_to_dense(*matrices.square_tridiag(*matrices.d2_dirichlet(N))), D2D @ D2D)
        assert np.array_equal(matrices.bands_to_dense(*matrices.square_tridiag(*matrices.d2_noflux(N))), D2N @ D2N)
    # the closed forms quoted for the boundary rows
    a, b, c, d, e = matrices.square_tridiag(*matrices.d2_dirichlet(8))
    assert (c[0], d[0], e[0]) == (5.0, -4.0, 1.0) and (b[1], c[1], d[1], e[1]) == (-4.0, 6.0, -4.0, 1.0)
    a, b, c, d, e = matrices.square_tridiag(*matrices.d2_noflux(8))
    assert (c[0], d[0], e[0]) == (2.0, -3.0, 1.0) and (b[1], c[1], d[1], e[1]) == (-3.0, 6.0, -4.0, 1.0)
    assert (a[7], b[7], c[7]) == (1.0, -3.0, 2.0)


def test_noflux_columns_sum_to_zero():
    for N in (2, 7, 64):
        D2N = matrices.bands_to_dense(*matrices.d2_noflux(N))
        D4N = matrices.bands_to_dense(*matrices.square_tridiag(*matrices.d2_noflux(N)))
        assert np.all(D2N.sum(axis=0) == 0.0) and np.all(D4N.sum(axis=0) == 0.0)


# ----------------------------------------------------- eigenmode decay factors

@pytest.mark.parametrize("N,r", [(16, 0.5), (63, 0.5), (256, 2.0)])
def test_diffusion_be_sine_mode_decay(N, r):
    k = np.arange(1, N + 1)
    V = synth.sine_mode_block(N, k)
    lam = 1.0 + 4.0 * r * np.sin(k * np.pi / (2 * (N + 1))) ** 2
    A = steppers.SharedTri(*matrices.diffusion_matrix(N, r))
    C1 = steppers.diffusion_be_step(A, V)
    assert np.max(np.abs(C1 - V / lam) ) <= 1e-13


@pytest.mark.parametrize("N,s", [(20, 0.3), (100, 1.7)])
def test_diffusion_cn_sine_mode_decay(N, s):
    k = np.arange(1, N + 1)
    V = synth.sine_mode_block(N, k)
    mu = 4.0 * np.sin(k * np.pi / (2 * (N + 1))) ** 2
    A = steppers.SharedTri(*matrices.diffusion_matrix(N, s))
    C1 = A.solve(steppers.diffusion_cn_rhs(N, s, V))
    assert np.max(np.abs(C1 - V * (1 - s * mu) / (1 + s * mu))) <= 1e-13


@pytest.mark.parametrize("N,r", [(32, 0.25), (200, 0.25)])
def test_hyperdiffusion_be_ten_steps_hinged(N, r):
    k = np.arange(1, N + 1)
    V = synth.sine_mode_block(N, k)
    mu = 16.0 * np.sin(k * np.pi / (2 * (N + 1))) ** 4
    A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, r, "hinged"))
    C = V
    for _ in range(10):
        C = steppers.hyper_be_step(A, C)
    assert np.max(np.abs(C - V * (1.0 + r * mu) ** -10)) <= 1e-13


def test_hyperdiffusion_cn_ten_steps_hinged():
    N, s = 48, 0.6
    k = np.arange(1, N + 1)
    V = synth.sine_mode_block(N, k)
    mu = 16.0 * np.sin(k * np.pi / (2 * (N + 1))) ** 4
    A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, s, "hinged"))
    C = V
    for _ in range(10):
        C = A.solve(steppers.hyper_cn_rhs(N, s, C, "hinged"))
    assert np.max(np.abs(C - V * ((1 - s * mu) / (1 + s * mu)) ** 10)) <= 1e-12


def test_truncated_closure_is_not_sine_diagonal_but_solves_dense():
    """The truncated stencil has corner 6, so sine modes are not its eigenvectors;
    its solve is pinned against LAPACK instead."""
    N = 24
    diags = matrices.hyperdiffusion_matrix(N, 0.25, "truncated")
    V = synth.sine_mode_block(N, [1])
    x = banded.penta_solve(*banded.penta_factor(*diags), V)
    ratio = x[:, 0] / V[:, 0]
    assert np.ptp(ratio) > 1e-3
    ref = np.linalg.solve(matrices.bands_to_dense(*diags), V)
    assert np.max(np.abs(x - ref)) <= 1e-14


# -------------------------------------------------------- Cahn-Hilliard checks

SIG = synth.CH_DT_GRID * synth.CH_GAMMA_GRID


def test_ch_constant_state_is_fixed_point():
    N = 64
    A = steppers.SharedPenta(*matrices.ch_matrix(N, SIG))
    C = np.tile(np.array([0.3, -0.7, 1.0, 0.0]), (N, 1))
    C1 = steppers.ch_step(A, C, synth.CH_DT_GRID)
    assert np.max(np.abs(C1 - C)) <= 4e-16


def test_ch_mass_conserved_2000_steps():
    N, M = 32, 4
    A = steppers.SharedPenta(*matrices.ch_matrix(N, SIG))
    C = synth.rhs_uniform(seed=4, N=N, M=M, lo=-0.1, hi=0.1)
    m0 = C.sum(axis=0)
    for _ in range(2000):
        C = steppers.ch_step(A, C, synth.CH_DT_GRID)
    drift = np.abs(C.sum(axis=0) - m0) / (N * np.max(np.abs(C), axis=0))
    assert np.max(drift) <= 1e-12


@pytest.mark.parametrize("gamma,dt", [(synth.CH_GAMMA_GRID, synth.CH_DT_GRID), (0.5, 0.2)])
def test_ch_small_amplitude_growth_factor(gamma, dt):
    """For C = eps cos(k pi (i+1/2)/N), eps = 1e-6 (the amplitude of the paper's
    convergence study), one step multiplies the mode by
    (1 + dt s_k) / (1 + dt gamma s_k^2), s_k = 4 sin^2(k pi / (2N)), up to O(eps^2)."""
    N = 64
    k = np.arange(1, N)
    eps = 1e-6
    V = synth.cosine_mode_block(N, k, amplitude=eps)
    A = steppers.SharedPenta(*matrices.ch_matrix(N, dt * gamma))
    C1 = steppers.ch_step(A, V, dt)
    s = 4.0 * np.sin(k * np.pi / (2 * N)) ** 2
    growth = (1.0 + dt * s) / (1.0 + dt * gamma * s ** 2)
    assert np.max(np.abs(C1 - V * growth)) <= 1e-10 * eps


def test_fp32_rhs_reference_promotes_exactly():
    N = 20
    A = steppers.SharedTri(*matrices.diffusion_matrix(N, 0.5))
    b32 = synth.rhs_uniform(seed=33, N=N, M=3, dtype=np.float32)
    x = steppers.solve_fp32_rhs(A, b32)
    ref = np.linalg.solve(matrices.bands_to_dense(*matrices.diffusion_matrix(N, 0.5)), b32.astype(np.float64))
    assert np.max(np.abs(x - ref)) <= 1e-14
