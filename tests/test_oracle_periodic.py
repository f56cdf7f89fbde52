"""Pins of the periodic tridiagonal oracle (section 3.3, Sherman-Morrison): dense
LAPACK solves of the periodic matrix (and its transpose) for nonsymmetric random
matrices, the exact A' + u v^T = A reconstruction, the exact decay factors of the
periodic grid's Fourier modes under backward Euler and Crank-Nicolson steps (the
circulant's eigenpairs), conservation of the mean, and a planted mistake in the
rank-one term that the pins catch."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices, steppers


def random_periodic(seed, N):
    a, b, c = synth.random_tri_diagonals(seed, N)
    g = np.random.default_rng([seed, 99])
    a = a.copy()
    c = c.copy()
    a[0] = g.uniform(-1, 1)       # corner A[0, N-1]
    c[N - 1] = g.uniform(-1, 1)   # corner A[N-1, 0]
    b = np.sign(b) * (np.abs(a) + np.abs(c) + 0.5 + g.uniform(0, 1, N))  # still dominant
    return a, b, c


@pytest.mark.parametrize("N", [3, 4, 5, 17, 64, 257])
def test_periodic_matches_dense_lapack(N):
    a, b, c = random_periodic(N, N)
    A = banded.tri_periodic_dense(a, b, c)
    d = synth.rhs_uniform(seed=N, N=N, M=4)
    fac = banded.tri_periodic_factor(a, b, c)
    x = banded.tri_periodic_solve(fac, d)
    assert np.max(np.abs(x - np.linalg.solve(A, d))) <= 1e-13 * np.max(np.abs(x))
    y = banded.tri_periodic_solve_adjoint(fac, d)
    assert np.max(np.abs(y - np.linalg.solve(A.T, d))) <= 1e-13 * np.max(np.abs(y))


def test_corner_entries_and_rank_one_split_reconstruct_A():
    N = 9
    a, b, c = random_periodic(3, N)
    A = banded.tri_periodic_dense(a, b, c)
    assert A[0, N - 1] == a[0] and A[N - 1, 0] == c[N - 1]
    fac = banded.tri_periodic_factor(a, b, c)
    Ap = banded.tri_dense(fac["a"], *_bp_cp(fac, b, c))
    assert np.array_equal(np.triu(np.tril(Ap, 1), -1), Ap)  # A' has no corners
    assert np.allclose(Ap + np.outer(fac["u"], fac["v"]), A, rtol=0, atol=1e-15)
    assert fac["u"][0] == -b[0] and fac["v"][N - 1] == -a[0] / b[0]


def _bp_cp(fac, b, c):
    """b', c' of A' from its factors (b'_i = bh_i + a'_i ch_{i-1}, c'_i = ch_i bh_i)."""
    bh, ch, ap = fac["bh"], fac["ch"], fac["a"]
    bp = bh.copy()
    bp[1:] = bh[1:] + ap[1:] * ch[:-1]
    cp = ch * bh
    return bp, cp


def test_adjoint_identity_nonsymmetric():
    N = 33
    a, b, c = random_periodic(11, N)
    fac = banded.tri_periodic_factor(a, b, c)
    bvec = synth.rhs_uniform(seed=1, N=N, M=1)
    yvec = synth.rhs_uniform(seed=2, N=N, M=1)
    lhs = float(banded.tri_periodic_solve(fac, bvec)[:, 0] @ yvec[:, 0])
    rhs = float(bvec[:, 0] @ banded.tri_periodic_solve_adjoint(fac, yvec)[:, 0])
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("N", [8, 64, 1024])
def test_fourier_modes_decay_exactly(N):
    """The periodic diffusion matrix is circulant: cos/sin(2 pi k i / N) are its
    eigenvectors with eigenvalue 1 + 4 r sin^2(pi k / N).  One backward-Euler solve
    divides a mode by it; one Crank-Nicolson step multiplies it by
    (1 - 4 s sin^2) / (1 + 4 s sin^2) (sections 3.2-3.3 with sigma = s)."""
    r = 0.5
    modes = [0, 1, 2, N // 4, N // 2 - 1, N // 2]
    A = steppers.SharedTriPeriodic(*matrices.diffusion_matrix_periodic(N, r))
    for kind in ("cos", "sin"):
        X = synth.fourier_mode_block(N, modes, kind)
        lam = 1.0 + 4.0 * r * np.sin(np.pi * np.asarray(modes) / N) ** 2
        Y = A.solve(X)
        assert np.max(np.abs(Y - X / lam[None, :])) <= 1e-13
        s = r  # CN: the left-hand side I + s K and the right-hand side (I - s K) C
        Z = A.solve(steppers.diffusion_cn_rhs_periodic(N, s, X))
        g = (1.0 - 4.0 * s * np.sin(np.pi * np.asarray(modes) / N) ** 2) / lam
        assert np.max(np.abs(Z - X * g[None, :])) <= 1e-13


def test_mean_is_conserved_by_periodic_diffusion():
    N, r = 100, 3.0
    A = steppers.SharedTriPeriodic(*matrices.diffusion_matrix_periodic(N, r))
    C = synth.rhs_uniform(seed=4, N=N, M=6)
    for _ in range(20):
        C = A.solve(steppers.diffusion_cn_rhs_periodic(N, r, C))
    # every column of K sums to zero, so the mean of each system is invariant
    assert np.max(np.abs(C.mean(axis=0) - synth.rhs_uniform(seed=4, N=N, M=6).mean(axis=0))) <= 1e-14


def test_pins_catch_a_wrong_rank_one_term(monkeypatch):
    """Plant a sign error in v (v_{N-1} = +a_0/b_0) and the dense pin fails."""
    N = 16
    a, b, c = random_periodic(5, N)
    fac = banded.tri_periodic_factor(a, b, c)
    bad = dict(fac)
    bad["v"] = fac["v"].copy()
    bad["v"][N - 1] = -bad["v"][N - 1]
    d = synth.rhs_uniform(seed=6, N=N, M=2)
    ref = np.linalg.solve(banded.tri_periodic_dense(a, b, c), d)
    assert np.max(np.abs(banded.tri_periodic_solve(bad, d) - ref)) > 1e-6


def test_small_n_rejected():
    with pytest.raises(ValueError):
        banded.tri_periodic_factor([1.0, 1.0], [4.0, 4.0], [1.0, 1.0])
