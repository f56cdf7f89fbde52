"""CPU tests of the two-ended sweep data (paper_2107_05395_gb300/csrc/two_ended.h).

The header is compiled for the host (tests/native/two_ended_harness.cpp).  Its
reference application (both forward chains, the interface system, both backward
chains) is compared in FP64 with the oracle's one-ended solves (sections 3.1 and
4.1): A^{-1} b and A^{-T} b must agree up to rounding for random diagonally
dominant matrices and for every workload matrix, at the smallest N the form takes,
odd and even N, and N = 1024.  The image is checked as well: its top rows hold the
oracle factorisation of A, its bottom rows the oracle factorisation of the reversed
matrix J A J.  The rows of the whole of J A J (reversed_rows, used by the
refinement passes that eliminate from the bottom) are checked the same way: a solve
that sweeps down and then up with them, and the rows themselves."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import banded, matrices

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-12


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("two") / "two_h.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-o", out,
                    os.path.join(HERE, "native", "two_ended_harness.cpp")], check=True)
    L = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    L.h_two_ended_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_long, dp, dp]
    L.h_two_ended_image.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
    L.h_reversed_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, dp, dp, dp]
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _diag_major(diags):
    return np.ascontiguousarray(np.concatenate([np.asarray(d, np.float64) for d in diags]))


def two_ended_solve(H, diags, b, transpose=False):
    P = (len(diags) - 1) // 2
    N, M = b.shape
    dm = _diag_major(diags)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b)
    s = H.h_two_ended_solve(P, N, _dp(dm), 1 if transpose else 0, M, _dp(b), _dp(x))
    return s, x


def oracle_solve(diags, b, transpose=False):
    if len(diags) == 3:
        a, bb, c = diags
        bh, ch = banded.tri_factor(a, bb, c)
        return (banded.tri_solve_adjoint if transpose else banded.tri_solve)(a, bh, ch, b)
    fac = banded.penta_factor(*diags)
    return (banded.penta_solve_adjoint if transpose else banded.penta_solve)(*fac, b)


def relerr(x, ref):
    return np.max(np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0))


def random_diags(kind, N, seed):
    return (synth.random_tri_diagonals if kind == "tri" else synth.random_penta_diagonals)(seed=seed, N=N)


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("N", [4, 5, 8, 9, 10, 64, 65, 333, 1024])
@pytest.mark.parametrize("kind", ["tri", "penta"])
def test_random_matrices_match_the_oracle(H, kind, N, transpose):
    P = 1 if kind == "tri" else 2
    diags = random_diags(kind, N, seed=N + 3)
    b = synth.rhs_normal(seed=N, N=N, M=7)
    s, x = two_ended_solve(H, diags, b, transpose)
    if N < 4 * P:
        assert s == -1  # below the smallest size the form takes
        return
    assert s == (N + 1) // 2
    assert relerr(x, oracle_solve(diags, b, transpose)) <= TOL


@pytest.mark.parametrize("N", [16, 255, 1024])
@pytest.mark.parametrize("name", ["diffusion", "hinged", "truncated", "cahn_hilliard"])
def test_workload_matrices_match_the_oracle(H, name, N):
    diags = {"diffusion": lambda: matrices.diffusion_matrix(N, 0.5),
             "hinged": lambda: matrices.hyperdiffusion_matrix(N, 0.25, "hinged"),
             "truncated": lambda: matrices.hyperdiffusion_matrix(N, 0.25, "truncated"),
             "cahn_hilliard": lambda: matrices.ch_matrix(N, 16.6e-3)}[name]()
    b = synth.rhs_uniform(seed=5, N=N, M=5)
    for transpose in (False, True):
        _, x = two_ended_solve(H, diags, b, transpose)
        assert relerr(x, oracle_solve(diags, b, transpose)) <= TOL


@pytest.mark.parametrize("kind", ["tri", "penta"])
def test_image_rows_are_the_two_oracle_factorisations(H, kind):
    """Top rows: {1/alpha, beta/alpha[, eps/alpha]} and {1, gamma[, delta]} of A's
    factorisation; bottom rows: the same of the reversed matrix, at the reversed
    index; then the 2P x 2P interface inverse."""
    N = 37
    P = 1 if kind == "tri" else 2
    W = P + 1
    diags = random_diags(kind, N, seed=11)
    img = np.zeros(2 * W * N + 4 * P * P)
    n = H.h_two_ended_image(P, N, _dp(_diag_major(diags)), _dp(img), img.size)
    assert n == img.size
    fw = img[:W * N].reshape(N, W)
    bw = img[W * N:2 * W * N].reshape(N, W)
    s = (N + 1) // 2

    def rows(d):
        if P == 1:
            a, b, c = d
            bh, ch = banded.tri_factor(a, b, c)
            f = np.stack([1.0 / bh, a / bh], axis=1)
            f[0, 1] = 0.0
            g = np.stack([np.ones(N), ch], axis=1)
            g[N - 1, 1] = 0.0
            return f, g
        eps, beta, alpha, gamma, delta = banded.penta_factor(*d)
        f = np.stack([1.0 / alpha, beta / alpha, eps / alpha], axis=1)
        g = np.stack([np.ones(N), gamma, delta], axis=1)
        return f, g

    ft, bt = rows(diags)
    # reversed matrix J A J: diagonal at offset o of row i is A's offset -o of row N-1-i
    rev = [np.asarray(diags[2 * P - k])[::-1].copy() for k in range(2 * P + 1)]
    fr, br = rows(rev)
    np.testing.assert_allclose(fw[:s], ft[:s], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(bw[:s], bt[:s], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(fw[s:], fr[:N - s][::-1], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(bw[s:], br[:N - s][::-1], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 64, 333])
@pytest.mark.parametrize("kind", ["tri", "penta"])
def test_reversed_rows_solve_from_the_other_end(H, kind, N):
    """reversed_rows: the factorisation of the whole of J A J at A's row indices,
    which the refinement passes that eliminate from the bottom use.  Sweeping down
    with its forward rows and up with its backward rows gives A^{-1} b (the oracle's
    one-ended solve) on nonsymmetric matrices, and the rows are the oracle's
    factorisation of the reversed matrix read backwards."""
    P = 1 if kind == "tri" else 2
    W = P + 1
    diags = random_diags(kind, N, seed=N + 40)
    b = np.ascontiguousarray(synth.rhs_normal(seed=N + 1, N=N, M=6), np.float64)
    x = np.zeros_like(b)
    rows = np.zeros(2 * W * N)
    assert H.h_reversed_solve(P, N, _dp(_diag_major(diags)), b.shape[1], _dp(b), _dp(x), _dp(rows)) == 0
    assert relerr(x, oracle_solve(diags, b)) <= TOL
    rev = [np.asarray(diags[2 * P - k])[::-1].copy() for k in range(2 * P + 1)]
    if P == 1:
        a, bb, c = rev
        bh, ch = banded.tri_factor(a, bb, c)
        f = np.stack([1.0 / bh, a / bh], axis=1)
        g = np.stack([np.ones(N), ch], axis=1)
    else:
        eps, beta, alpha, gamma, delta = banded.penta_factor(*rev)
        f = np.stack([1.0 / alpha, beta / alpha, eps / alpha], axis=1)
        g = np.stack([np.ones(N), gamma, delta], axis=1)
    f[0, 1:] = 0.0  # coefficients that reach outside the matrix are zero
    if P == 2 and N > 1:
        f[1, 2] = 0.0
    g[N - 1, 1:] = 0.0
    if P == 2 and N > 1:
        g[N - 2, 2] = 0.0
    np.testing.assert_allclose(rows[:W * N].reshape(N, W), f[::-1], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(rows[W * N:].reshape(N, W), g[::-1], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("name", ["diffusion", "hinged", "truncated", "cahn_hilliard"])
def test_reversed_rows_on_workload_matrices(H, name):
    N = 255
    diags = {"diffusion": lambda: matrices.diffusion_matrix(N, 2.0),
             "hinged": lambda: matrices.hyperdiffusion_matrix(N, 0.25, "hinged"),
             "truncated": lambda: matrices.hyperdiffusion_matrix(N, 0.25, "truncated"),
             "cahn_hilliard": lambda: matrices.ch_matrix(N, 16.6e-3)}[name]()
    P = (len(diags) - 1) // 2
    b = np.ascontiguousarray(synth.rhs_uniform(seed=9, N=N, M=4), np.float64)
    x = np.zeros_like(b)
    assert H.h_reversed_solve(P, N, _dp(_diag_major(diags)), b.shape[1], _dp(b), _dp(x), None) == 0
    assert relerr(x, oracle_solve(diags, b)) <= TOL


def test_reversed_rows_report_a_zero_pivot(H):
    """A = [[1, 1], [1, 0]] factors from the top, but J A J = [[0, 1], [1, 1]] has a
    zero first pivot."""
    diags = (np.array([0.0, 1.0]), np.array([1.0, 0.0]), np.array([1.0, 0.0]))
    b = np.ones((2, 1))
    x = np.zeros_like(b)
    assert H.h_reversed_solve(1, 2, _dp(_diag_major(diags)), 1, _dp(b), _dp(x), None) == -1

