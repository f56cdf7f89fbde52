"""Pins for oracle/banded.py against things other than the oracle itself:
dense LAPACK solves, exact rational elimination, the factor identity A = LU / LR,
the adjoint identity, and planted mistakes that the pins must catch."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import banded, matrices


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)))


def exact_solve(A_rows, rhs):
    """Gaussian elimination with partial pivoting in exact rational arithmetic."""
    n = len(A_rows)
    A = [[Fraction(v) for v in row] + [Fraction(r)] for row, r in zip(A_rows, rhs)]
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(A[i][k]))
        A[k], A[p] = A[p], A[k]
        for i in range(k + 1, n):
            f = A[i][k] / A[k][k]
            for j in range(k, n + 1):
                A[i][j] -= f * A[k][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = A[i][n] - sum(A[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / A[i][i]
    return x


# ---------------------------------------------------------------- tridiagonal

@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 17, 64])
def test_tri_matches_dense_lapack(N):
    a, b, c = synth.random_tri_diagonals(seed=100 + N, N=N)
    d = synth.rhs_uniform(seed=200 + N, N=N, M=7)
    bh, ch = banded.tri_factor(a, b, c)
    x = banded.tri_solve(a, bh, ch, d)
    ref = np.linalg.solve(banded.tri_dense(a, b, c), d)
    assert rel_err(x, ref) <= 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 8])
def test_tri_matches_exact_rationals(N):
    a, b, c = synth.random_tri_diagonals(seed=300 + N, N=N)
    d = synth.rhs_uniform(seed=400 + N, N=N, M=3)
    bh, ch = banded.tri_factor(a, b, c)
    x = banded.tri_solve(a, bh, ch, d)
    A = banded.tri_dense(a, b, c)
    for m in range(d.shape[1]):
        ex = np.array([float(v) for v in exact_solve(A.tolist(), d[:, m].tolist())])
        assert np.max(np.abs(x[:, m] - ex)) <= 8 * np.finfo(float).eps * np.max(np.abs(ex))


@pytest.mark.parametrize("N", [2, 5, 33])
def test_tri_factor_reconstructs_A(N):
    a, b, c = synth.random_tri_diagonals(seed=500 + N, N=N)
    bh, ch = banded.tri_factor(a, b, c)
    L = np.diag(bh) + np.diag(a[1:], -1)
    U = np.eye(N) + np.diag(ch[:-1], 1)
    assert np.max(np.abs(L @ U - banded.tri_dense(a, b, c))) <= 1e-14 * np.max(np.abs(b))


@pytest.mark.parametrize("N", [1, 2, 3, 9, 64])
def test_tri_adjoint_matches_dense_transpose(N):
    a, b, c = synth.random_tri_diagonals(seed=600 + N, N=N)
    g = synth.rhs_normal(seed=700 + N, N=N, M=5)
    bh, ch = banded.tri_factor(a, b, c)
    y = banded.tri_solve_adjoint(a, bh, ch, g)
    ref = np.linalg.solve(banded.tri_dense(a, b, c).T, g)
    assert rel_err(y, ref) <= 1e-13


def test_tri_adjoint_identity_nonsymmetric():
    N = 40
    a, b, c = synth.random_tri_diagonals(seed=801, N=N)
    assert np.max(np.abs(banded.tri_dense(a, b, c) - banded.tri_dense(a, b, c).T)) > 0.1
    bvec = synth.rhs_normal(seed=802, N=N, M=6)
    yvec = synth.rhs_normal(seed=803, N=N, M=6)
    bh, ch = banded.tri_factor(a, b, c)
    lhs = np.sum(banded.tri_solve(a, bh, ch, bvec) * yvec, axis=0)
    rhs = np.sum(bvec * banded.tri_solve_adjoint(a, bh, ch, yvec), axis=0)
    assert np.max(np.abs(lhs - rhs) / np.abs(lhs)) <= 1e-13


def test_tri_zero_pivot_raises():
    with pytest.raises(ZeroDivisionError):
        banded.tri_factor([0.0, 1.0], [0.0, 1.0], [1.0, 0.0])
    # pivot that becomes zero after elimination: [[1, 1], [1, 1]]
    with pytest.raises(ZeroDivisionError):
        banded.tri_factor([0.0, 1.0], [1.0, 1.0], [1.0, 0.0])


def test_tri_linearity():
    N = 30
    a, b, c = synth.random_tri_diagonals(seed=901, N=N)
    bh, ch = banded.tri_factor(a, b, c)
    u = synth.rhs_normal(seed=902, N=N, M=4)
    v = synth.rhs_normal(seed=903, N=N, M=4)
    lhs = banded.tri_solve(a, bh, ch, 2.0 * u - 3.0 * v)
    rhs = 2.0 * banded.tri_solve(a, bh, ch, u) - 3.0 * banded.tri_solve(a, bh, ch, v)
    assert rel_err(lhs, rhs) <= 1e-13


# -------------------------------------------------------------- pentadiagonal

@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 17, 64])
def test_penta_matches_dense_lapack(N):
    diags = synth.random_penta_diagonals(seed=1000 + N, N=N)
    f = synth.rhs_uniform(seed=1100 + N, N=N, M=7)
    fac = banded.penta_factor(*diags)
    x = banded.penta_solve(*fac, f)
    ref = np.linalg.solve(banded.penta_dense(*diags), f)
    assert rel_err(x, ref) <= 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8])
def test_penta_matches_exact_rationals(N):
    diags = synth.random_penta_diagonals(seed=1200 + N, N=N)
    f = synth.rhs_uniform(seed=1300 + N, N=N, M=3)
    x = banded.penta_solve(*banded.penta_factor(*diags), f)
    A = banded.penta_dense(*diags)
    for m in range(f.shape[1]):
        ex = np.array([float(v) for v in exact_solve(A.tolist(), f[:, m].tolist())])
        assert np.max(np.abs(x[:, m] - ex)) <= 16 * np.finfo(float).eps * np.max(np.abs(ex))


@pytest.mark.parametrize("N", [3, 6, 41])
def test_penta_factor_reconstructs_A(N):
    diags = synth.random_penta_diagonals(seed=1400 + N, N=N)
    eps, beta, alpha, gamma, delta = banded.penta_factor(*diags)
    L = np.diag(alpha) + np.diag(beta[1:], -1) + np.diag(eps[2:], -2)
    R = np.eye(N) + np.diag(gamma[:-1], 1) + np.diag(delta[:-2], 2)
    A = banded.penta_dense(*diags)
    assert np.max(np.abs(L @ R - A)) <= 1e-14 * np.max(np.abs(A))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 9, 64])
def test_penta_adjoint_matches_dense_transpose(N):
    diags = synth.random_penta_diagonals(seed=1500 + N, N=N)
    g = synth.rhs_normal(seed=1600 + N, N=N, M=5)
    y = banded.penta_solve_adjoint(*banded.penta_factor(*diags), g)
    ref = np.linalg.solve(banded.penta_dense(*diags).T, g)
    assert rel_err(y, ref) <= 1e-13


def test_penta_adjoint_identity_nonsymmetric():
    N = 50
    diags = synth.random_penta_diagonals(seed=1701, N=N)
    fac = banded.penta_factor(*diags)
    bvec = synth.rhs_normal(seed=1702, N=N, M=6)
    yvec = synth.rhs_normal(seed=1703, N=N, M=6)
    lhs = np.sum(banded.penta_solve(*fac, bvec) * yvec, axis=0)
    rhs = np.sum(bvec * banded.penta_solve_adjoint(*fac, yvec), axis=0)
    assert np.max(np.abs(lhs - rhs) / np.abs(lhs)) <= 1e-13


def test_penta_on_workload_matrices_vs_dense():
    for diags in (matrices.hyperdiffusion_matrix(48, 0.25, "hinged"),
                  matrices.hyperdiffusion_matrix(48, 0.25, "truncated"),
                  matrices.ch_matrix(48, 0.0166)):
        f = synth.rhs_normal(seed=1800, N=48, M=4)
        x = banded.penta_solve(*banded.penta_factor(*diags), f)
        ref = np.linalg.solve(matrices.bands_to_dense(*diags), f)
        assert rel_err(x, ref) <= 1e-13


def test_penta_zero_pivot_raises():
    z = np.zeros(3)
    with pytest.raises(ZeroDivisionError):
        banded.penta_factor(z, z, np.array([1.0, 0.0, 1.0]), z, z)


# ---------------------------------------------- planted mistakes must be caught

def test_pins_catch_printed_thomas_typo():
    """The back substitution printed in section 3.1 (x_i = dh_i - a_i ch_i, without
    x_{i+1}) must fail the dense pin; the oracle follows Algorithm 2 instead."""
    N = 12
    a, b, c = synth.random_tri_diagonals(seed=1900, N=N)
    d = synth.rhs_uniform(seed=1901, N=N, M=3)
    bh, ch = banded.tri_factor(a, b, c)
    dh = np.empty_like(d)
    dh[0] = d[0] / bh[0]
    for i in range(1, N):
        dh[i] = (d[i] - a[i] * dh[i - 1]) / bh[i]
    wrong = dh.copy()
    for i in range(N - 2, -1, -1):
        wrong[i] = dh[i] - a[i] * ch[i]
    ref = np.linalg.solve(banded.tri_dense(a, b, c), d)
    assert rel_err(wrong, ref) > 1e-3


def test_pins_catch_printed_penta_factor_typo():
    """Algorithm 3's alpha update as printed (a_i c_{i-2} instead of a_i delta_{i-2})
    gives factors whose product is not A."""
    N = 10
    diags = synth.random_penta_diagonals(seed=1950, N=N)
    eps, beta, alpha, gamma, delta = banded.penta_factor(*diags)
    a, b, c, d, e = diags
    # recompute alpha with the printed typo and check that L R no longer equals A
    alpha_w = alpha.copy()
    for i in range(2, N):
        alpha_w[i] = c[i] - a[i] * alpha[i - 2] - beta[i] * gamma[i - 1]
    L = np.diag(alpha_w) + np.diag(beta[1:], -1) + np.diag(eps[2:], -2)
    R = np.eye(N) + np.diag(gamma[:-1], 1) + np.diag(delta[:-2], 2)
    assert np.max(np.abs(L @ R - banded.penta_dense(*diags))) > 1e-3
