"""CPU tests of the partitioned solve's host data (paper_2107_05395_gb300/csrc/partition.h).

The header is compiled for the host (tests/native/partition_harness.cpp) and its
reference application of the partitioned solve (chunk sweeps, spikes, cyclic
reduction of the boundary system, correction) is compared, in FP64, with the
oracle's sequential solves (sections 3.1 and 4.1): chunked solves must reproduce
A^{-1} b and A^{-T} b up to rounding with identity-padded last chunks, empty
chunks, one chunk, the shortest chunks, and every workload matrix.  The device
image is checked too: its section offsets, and that chunk 0's rows hold the
global factorisation's coefficients (chunk 0 starts where the global recurrence
starts)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import banded, matrices

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("part") / "part_h.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-o", out,
                    os.path.join(HERE, "native", "partition_harness.cpp")], check=True)
    L = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L.h_partition_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_long, dp, dp, ctypes.c_int]
    L.h_partition_image.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp,
                                    ctypes.c_int, ip]
    L.h_partition_image_paired.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp,
                                           ctypes.c_int]
    L.h_partition_image_thomas.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp,
                                           ctypes.c_int, ip]
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _diag_major(diags):
    return np.ascontiguousarray(np.concatenate([np.asarray(d, np.float64) for d in diags]))


def part_solve(H, diags, L, P, b, transpose=False, thomas=False):
    PB = (len(diags) - 1) // 2
    N, M = b.shape
    dm = _diag_major(diags)
    b = np.ascontiguousarray(b, np.float64)
    x = np.empty_like(b)
    NL = H.h_partition_solve(PB, N, _dp(dm), L, P, 1 if transpose else 0, M, _dp(b), _dp(x),
                             1 if thomas else 0)
    assert NL >= 0
    return x, NL


def oracle_solve(diags, b, transpose=False):
    if len(diags) == 3:
        a, bb, c = diags
        bh, ch = banded.tri_factor(a, bb, c)
        return (banded.tri_solve_adjoint if transpose else banded.tri_solve)(a, bh, ch, b)
    fac = banded.penta_factor(*diags)
    return (banded.penta_solve_adjoint if transpose else banded.penta_solve)(*fac, b)


def relerr(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


CASES = [
    ("penta random, padded last chunk", lambda: synth.random_penta_diagonals(3, 1000), 32, 32),
    ("penta random, one chunk", lambda: synth.random_penta_diagonals(4, 200), 256, 1),
    ("penta random, 4-row chunks", lambda: synth.random_penta_diagonals(5, 128), 4, 32),
    ("penta random, 13 empty chunks", lambda: synth.random_penta_diagonals(6, 300), 16, 32),
    ("penta random, 3 chunks", lambda: synth.random_penta_diagonals(7, 90), 32, 3),
    ("hinged hyperdiffusion r=0.25", lambda: matrices.hyperdiffusion_matrix(1024, 0.25), 32, 32),
    ("hinged hyperdiffusion r=0.25, 16-row chunks", lambda: matrices.hyperdiffusion_matrix(512, 0.25), 16, 32),
    ("truncated hyperdiffusion r=2", lambda: matrices.hyperdiffusion_matrix(511, 2.0, "truncated"), 16, 32),
    ("Cahn-Hilliard", lambda: matrices.ch_matrix(256, 0.0166), 8, 32),
    ("tri random, padded", lambda: synth.random_tri_diagonals(6, 257), 16, 17),
    ("tri diffusion r=0.5", lambda: matrices.diffusion_matrix(256, 0.5), 8, 32),
    ("tri diffusion r=50", lambda: matrices.diffusion_matrix(1000, 50.0), 32, 32),
]


@pytest.mark.parametrize("name,make,L,P", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("reduced", ["cyclic_reduction", "block_thomas"])
def test_partitioned_solve_matches_sequential_oracle(H, name, make, L, P, transpose, reduced):
    diags = make()
    N = len(diags[0])
    b = synth.rhs_uniform(seed=9, N=N, M=5)
    x, NL = part_solve(H, diags, L, P, b, transpose, thomas=reduced == "block_thomas")
    assert NL == int(np.ceil(np.log2(P - 1))) if P > 2 else NL == 0
    ref = oracle_solve(diags, b, transpose)
    # both are backward-stable solves of a well-conditioned system; rounding only
    assert relerr(x, ref) <= 1e-12, relerr(x, ref)
    # and x solves the system it claims to (residual of the oracle's own product)
    dense = matrices.bands_to_dense(*diags)
    A = dense.T if transpose else dense
    assert np.max(np.abs(A @ x - b)) <= 1e-12 * np.max(np.abs(b)) * max(1.0, np.abs(A).sum(1).max())


def test_one_chunk_is_the_sequential_recurrence(H):
    """With one chunk the partitioned solve is the sequential sweep itself."""
    diags = synth.random_penta_diagonals(7, 64)
    b = synth.rhs_uniform(seed=2, N=64, M=3)
    x, NL = part_solve(H, diags, 64, 1, b)
    assert NL == 0
    assert relerr(x, oracle_solve(diags, b)) <= 1e-14


def test_image_sections_and_chunk0_coefficients(H):
    N, L, P = 100, 32, 4  # the last chunk has 4 real rows and 28 identity rows
    diags = synth.random_penta_diagonals(8, N)
    dm = _diag_major(diags)
    out = np.zeros(40000)
    lay = (ctypes.c_int * 6)()
    n = H.h_partition_image(2, N, _dp(dm), L, P, _dp(out), out.size, lay)
    fwd, bwd, cor, T0, M, total = list(lay)
    Q, PB, NP, NL = 4, 2, P * L, 2
    assert n == total
    for off in (fwd, bwd, cor, T0, M, total):
        assert off % 4 == 0
    assert bwd >= fwd + 4 * NP and cor >= bwd + PB * NP and T0 >= cor + Q * NP
    assert M == T0 + Q * Q * P and total >= M + NL * (Q * Q + 2 * Q * PB) * P
    eps, beta, alpha, gamma, delta = banded.penta_factor(*diags)
    for i in range(L):  # chunk 0 = rows [0, L)
        F0, F1, F2, pad = out[fwd + 4 * i: fwd + 4 * i + 4]
        B1, B2 = out[bwd + 2 * i: bwd + 2 * i + 2]
        assert pad == 0.0
        assert np.isclose(F0, 1.0 / alpha[i], rtol=1e-15, atol=0)
        assert np.isclose(F1, beta[i] / alpha[i], rtol=1e-15, atol=1e-300)
        assert np.isclose(F2, eps[i] / alpha[i], rtol=1e-15, atol=1e-300)
        if i < L - 2:  # the chunk's last rows drop their coupling to chunk 1
            assert np.isclose(B1, gamma[i], rtol=1e-15, atol=1e-300)
            assert np.isclose(B2, delta[i], rtol=1e-15, atol=1e-300)
    assert out[bwd + 2 * (L - 1)] == 0.0 and out[bwd + 2 * (L - 1) + 1] == 0.0
    # first row of every chunk restarts: no coupling to the rows above
    for c in range(P):
        assert out[fwd + 4 * c * L + 1] == 0.0 and out[fwd + 4 * c * L + 2] == 0.0
    # padding rows are identity rows with no spikes
    for i in range(N, NP):
        assert list(out[fwd + 4 * i: fwd + 4 * i + 4]) == [1.0, 0.0, 0.0, 0.0]
        assert not np.any(out[bwd + 2 * i: bwd + 2 * i + 2]) and not np.any(out[cor + Q * i: cor + Q * i + Q])
    # spikes of chunk 0 couple only to the right, of the last chunk only to the left
    for i in range(L):
        assert out[cor + Q * i] == 0.0 and out[cor + Q * i + 1] == 0.0
    for i in range((P - 1) * L, NP):
        assert out[cor + Q * i + 2] == 0.0 and out[cor + Q * i + 3] == 0.0
    # boundary slots beyond K = P - 1 are zero (lanes that hold no boundary)
    for e in range(Q * Q):
        assert out[T0 + e * P + P - 1] == 0.0
    assert np.all(out[T0 + 0 * P: T0 + P - 1] != 0.0)  # the diagonal of T0_k = D_k^{-1}


def test_zero_pivot_is_reported(H):
    a, b, c, d, e = synth.random_penta_diagonals(9, 40)
    c = c.copy()
    c[0] = 0.0
    b0 = np.ones((40, 1))
    x = np.empty_like(b0)
    dm = _diag_major((a, b, c, d, e))
    assert H.h_partition_solve(2, 40, _dp(dm), 10, 4, 0, 1, _dp(b0), _dp(x), 0) == -1
    # too few chunks to cover the rows
    dm2 = _diag_major(synth.random_penta_diagonals(10, 40))
    assert H.h_partition_solve(2, 40, _dp(dm2), 8, 4, 0, 1, _dp(b0), _dp(x), 0) == -1


@pytest.mark.parametrize("PB,N,L", [(1, 256, 16), (2, 500, 32), (2, 100, 8)])
def test_fp64_image_carries_both_boundary_solvers(H, PB, N, L):
    """The FP64 small-tile image (16 chunks) holds the same chunk rows as the
    cyclic-reduction image, the block-Thomas factors, and the cyclic-reduction
    sections T0 / M copied entry for entry (the kernel uses either)."""
    P = 16
    diags = synth.random_penta_diagonals(seed=N, N=N) if PB == 2 else synth.random_tri_diagonals(seed=N, N=N)
    dm = _diag_major(diags)
    a = np.zeros(200000)
    la = (ctypes.c_int * 6)()
    na = H.h_partition_image(PB, N, _dp(dm), L, P, _dp(a), a.size, la)
    b = np.zeros(200000)
    lb = (ctypes.c_int * 9)()
    nb = H.h_partition_image_thomas(PB, N, _dp(dm), L, P, _dp(b), b.size, lb)
    assert na > 0 and nb > 0
    fwd, bwd, cor, T0, M, total = list(la)
    tf, tb, tc, E, Hs, J, tT0, tM, ttotal = list(lb)
    assert (fwd, bwd, cor) == (tf, tb, tc)
    assert E == T0 and np.array_equal(a[:T0], b[:E])                # chunk rows
    assert np.array_equal(a[T0:total], b[tT0:tT0 + (total - T0)])    # T0 and the levels
    assert tM - tT0 == M - T0 and ttotal - tT0 == total - T0
    Q = 2 * PB
    assert E >= tc and Hs - E >= (P - 1) * PB * Q and J - Hs >= (P - 1) * Q * Q and tT0 - J >= (P - 1) * Q * PB
    assert np.any(b[E:Hs] != 0) and np.any(b[Hs:J] != 0)


@pytest.mark.parametrize("PB,N,L", [(2, 1000, 64), (1, 300, 32), (2, 200, 16)])
def test_paired_image_interleaves_each_chunk_pair(H, PB, N, L):
    """The paired image (two chunks per warp) holds exactly the rows of the plain image:
    row j of chunk c at padded row (c // 2) 2L + 2j + c % 2 of the fwd, bwd and cor
    sections, and the reduction sections unchanged."""
    P = 16
    diags = synth.random_penta_diagonals(seed=N, N=N) if PB == 2 else synth.random_tri_diagonals(seed=N, N=N)
    dm = _diag_major(diags)
    a = np.zeros(100000)
    la = (ctypes.c_int * 6)()
    na = H.h_partition_image(PB, N, _dp(dm), L, P, _dp(a), a.size, la)
    b = np.zeros(100000)
    nb = H.h_partition_image_paired(PB, N, _dp(dm), L, P, _dp(b), b.size)
    assert na == nb > 0
    fwd, bwd, cor, T0, M, total = list(la)
    FW, Q = (4 if PB == 2 else 2), 2 * PB
    for c in range(P):
        for j in range(L):
            src, dst = c * L + j, (c // 2) * 2 * L + 2 * j + c % 2
            assert np.array_equal(b[fwd + dst * FW: fwd + dst * FW + FW], a[fwd + src * FW: fwd + src * FW + FW])
            assert np.array_equal(b[bwd + dst * PB: bwd + dst * PB + PB], a[bwd + src * PB: bwd + src * PB + PB])
            assert np.array_equal(b[cor + dst * Q: cor + dst * Q + Q], a[cor + src * Q: cor + src * Q + Q])
    assert np.array_equal(a[T0:total], b[T0:total])
