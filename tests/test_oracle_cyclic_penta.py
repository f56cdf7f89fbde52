"""Pins of the cyclic pentadiagonal oracle (rank-2 Sherman-Morrison-Woodbury, the
block form of section 3.3's construction) and of the periodic Cahn-Hilliard step
of section 5.1: dense LAPACK solves of the cyclic matrix and its transpose for
nonsymmetric random matrices, the exact A' + U V^T = A split with A' banded, the
circulant's exact Fourier-mode decay under periodic hyperdiffusion, the periodic
CH step's constant fixed points, exact mass conservation and the linear growth
factor of small modes, the coarsening length of known states, and a planted
mistake the pins catch."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices, steppers


def random_cyclic(seed, N):
    g = np.random.default_rng([seed, 5])
    a, b, d, e = (g.uniform(-1, 1, N) for _ in range(4))
    c = np.sign(g.uniform(-1, 1, N)) * (np.abs(a) + np.abs(b) + np.abs(d) + np.abs(e) + 0.5 + g.uniform(0, 1, N))
    return a, b, c, d, e


@pytest.mark.parametrize("N", [5, 6, 7, 16, 101, 256])
def test_cyclic_penta_matches_dense_lapack(N):
    diags = random_cyclic(N, N)
    A = banded.penta_periodic_dense(*diags)
    f = banded.penta_periodic_factor(*diags)
    rhs = synth.rhs_uniform(seed=N, N=N, M=3)
    x = banded.penta_periodic_solve(f, rhs)
    assert np.max(np.abs(x - np.linalg.solve(A, rhs))) <= 1e-13 * np.max(np.abs(x))
    y = banded.penta_periodic_solve_adjoint(f, rhs)
    assert np.max(np.abs(y - np.linalg.solve(A.T, rhs))) <= 1e-13 * np.max(np.abs(y))


def test_split_is_exact_and_banded():
    N = 11
    diags = random_cyclic(3, N)
    A = banded.penta_periodic_dense(*diags)
    f = banded.penta_periodic_factor(*diags)
    Ap = banded.penta_dense(*f["diags_prime"])
    assert np.allclose(Ap + f["U"] @ f["V"].T, A, rtol=0, atol=1e-14)
    # corners of A' vanish; only the two 2 x 2 diagonal blocks change
    D = A - Ap
    mask = np.zeros((N, N), bool)
    for r in (0, 1, N - 2, N - 1):
        for c in (0, 1, N - 2, N - 1):
            mask[r, c] = True
    assert np.all(D[~mask] == 0.0)
    assert np.allclose(Ap[0:2, 0:2], 2.0 * A[0:2, 0:2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [8, 64, 256])
def test_periodic_hyperdiffusion_fourier_decay(N):
    """I + s D4_P is circulant with eigenvalue 1 + 16 s sin^4(pi k / N) on the modes
    cos/sin(2 pi k i / N)."""
    s = 0.37
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, s))
    modes = [0, 1, 3, N // 4, N // 2 - 1, N // 2]
    lam = 1.0 + 16.0 * s * np.sin(np.pi * np.asarray(modes) / N) ** 4
    for kind in ("cos", "sin"):
        X = synth.fourier_mode_block(N, modes, kind)
        assert np.max(np.abs(A.solve(X) - X / lam[None, :])) <= 1e-13


def test_periodic_ch_fixed_points_mass_and_linear_growth():
    N, gamma, dt = 256, synth.CH_GAMMA_GRID, synth.CH_DT_GRID
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, dt * gamma))
    # constants are fixed points: D2_P and D4_P annihilate them
    for v in (0.0, 0.3, -1.0, 1.0):
        C = np.full((N, 1), v)
        assert np.max(np.abs(steppers.ch_step_periodic(A, C, dt) - C)) <= 1e-15
    # mass (the sum over the ring) is conserved to roundoff over many steps
    C = synth.rhs_uniform(seed=4, N=N, M=8, lo=-0.1, hi=0.1)
    m0 = C.sum(axis=0)
    for _ in range(200):
        C = steppers.ch_step_periodic(A, C, dt)
    assert np.max(np.abs(C.sum(axis=0) - m0)) <= 1e-12 * N
    # a small mode grows by (1 + dt s_k) / (1 + dt gamma s_k^2), s_k = 4 sin^2(pi k/N)
    k = np.array([1, 3, 5, 9])
    eps = 1e-6
    X = eps * synth.fourier_mode_block(N, k, "cos")
    sk = 4.0 * np.sin(np.pi * k / N) ** 2
    g = (1.0 + dt * sk) / (1.0 + dt * gamma * sk ** 2)
    Y = steppers.ch_step_periodic(A, X, dt)
    assert np.max(np.abs(Y - X * g[None, :])) <= 10 * eps ** 3 + 1e-18


def test_coarsening_length_of_known_states():
    N = 64
    assert steppers.coarsening_length(np.zeros((N, 5))) == 1.0
    # C = +-a alternating sign has <C^2> = a^2
    a = 0.5
    C = a * np.where(np.arange(N) % 2 == 0, 1.0, -1.0)[:, None] * np.ones((1, 3))
    assert abs(steppers.coarsening_length(C) - 1.0 / (1.0 - a * a)) <= 1e-15
    # a cosine of amplitude a: <C^2> = a^2 / 2 exactly on the periodic grid
    C = a * synth.fourier_mode_block(N, [3], "cos")
    assert abs(steppers.coarsening_length(C) - 1.0 / (1.0 - a * a / 2.0)) <= 1e-14


def test_pins_catch_a_wrong_correction():
    N = 20
    diags = random_cyclic(9, N)
    f = banded.penta_periodic_factor(*diags)
    bad = dict(f)
    bad["V"] = f["V"].copy()
    bad["V"][N - 1, 0] = -bad["V"][N - 1, 0]
    rhs = synth.rhs_uniform(seed=1, N=N, M=2)
    ref = np.linalg.solve(banded.penta_periodic_dense(*diags), rhs)
    assert np.max(np.abs(banded.penta_periodic_solve(bad, rhs) - ref)) > 1e-6


def test_small_n_rejected():
    with pytest.raises(ValueError):
        banded.penta_periodic_factor(*(np.ones(4) for _ in range(5)))
