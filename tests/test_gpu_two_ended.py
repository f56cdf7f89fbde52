"""GPU parity of the two-ended sweeps (SB_ALGO_TWO_ENDED: every system eliminated from
both ends at once, joined by a 2P x 2P interface system) through the C ABI, element
by element against the FP64 oracle's one-ended solves on the same seeded inputs:
A and A^T, tridiagonal and pentadiagonal, the smallest N the form takes, odd and
even N, several tiles with ragged last tiles and padded ld (canaries), in place,
launch sizes from one warp to 1024 threads; and the fallback to the sequential
sweeps where the form does not apply (N below 4P, periodic factors, FP32 data).

Tolerance 1e-12 relative L2 per system, as for every FP64 path."""
import numpy as np
import pytest

import synth
from oracle import banded
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = 1e-12
CANARY = 12345.678


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def factor(sb, kind, diags):
    return (sb.sb_factor_shared_tri if kind == "tri" else sb.sb_factor_shared_penta)(*diags)


def oracle(kind, diags, rhs, adjoint):
    if kind == "tri":
        a, b, c = diags
        bh, ch = banded.tri_factor(a, b, c)
        return (banded.tri_solve_adjoint if adjoint else banded.tri_solve)(a, bh, ch, rhs)
    fac = banded.penta_factor(*diags)
    return (banded.penta_solve_adjoint if adjoint else banded.penta_solve)(*fac, rhs)


def solve(sb, torch, fac, rhs_host, M, shape, adjoint=False, inplace=False, dtype=np.float64):
    rhs = to_dev(rhs_host.astype(dtype), torch)
    x = rhs if inplace else torch.full_like(rhs, CANARY)
    code = sb.SB_F64 if dtype == np.float64 else sb.SB_F32
    sb.sb_shape_set(fac, shape, rhs_dtype=code, x_dtype=code)
    sb.sb_solve_batched_ex(fac, rhs, x, transpose=adjoint, M=M, ld=rhs.shape[1])
    torch.cuda.synchronize()
    return to_host(x)


SHAPES = [(4, 33, 40), (8, 31, 32), (9, 100, 101), (64, 200, 256), (513, 300, 301), (1024, 1000, 1000),
          (2000, 70, 70)]


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("N,M,ld", SHAPES)
@pytest.mark.parametrize("kind", ["tri", "penta"])
def test_two_ended_matches_oracle(env, kind, N, M, ld, adjoint):
    sb, torch = env
    diags = (synth.random_tri_diagonals if kind == "tri" else synth.random_penta_diagonals)(seed=N, N=N)
    fac = factor(sb, kind, diags)
    rhs = synth.rhs_normal(seed=40 + N, N=N, M=M, ld=ld, pad_value=CANARY)
    x = solve(sb, torch, fac, rhs, M, (768, 0, 1, sb.SB_ALGO_TWO_ENDED), adjoint)
    assert np.max(relerr_per_system(x[:, :M], oracle(kind, diags, rhs[:, :M], adjoint))) <= TOL
    assert np.all(x[:, M:] == CANARY), "padding columns were written"


@pytest.mark.parametrize("threads", [32, 96, 256, 1024])
def test_two_ended_launch_sizes_and_in_place(env, threads):
    """Every tile solved once at each launch size (8193 systems, a ragged last tile),
    in place (x = rhs)."""
    sb, torch = env
    N, M = 101, 8193
    diags = synth.random_penta_diagonals(seed=3, N=N)
    fac = factor(sb, "penta", diags)
    rhs = synth.rhs_normal(seed=4, N=N, M=M, ld=M, pad_value=CANARY)
    x = solve(sb, torch, fac, rhs, M, (threads, 0, 1, sb.SB_ALGO_TWO_ENDED), inplace=True)
    assert np.max(relerr_per_system(x, oracle("penta", diags, rhs, False))) <= TOL


def test_two_ended_workload_matrix(env):
    """The hinged A = I + 0.25 D4 at N = 1024 (the FP64 headline matrix), 4096 systems."""
    sb, torch = env
    N, M = 1024, 4096
    diags = sb.sb_build_matrix("hinged", N, 0.25)
    fac = factor(sb, "penta", diags)
    rhs = synth.rhs_normal(seed=2, N=N, M=M)
    x = solve(sb, torch, fac, rhs, M, (1024, 0, 1, sb.SB_ALGO_TWO_ENDED))
    assert np.max(relerr_per_system(x, oracle("penta", diags, rhs, False))) <= TOL


@pytest.mark.parametrize("case", ["small_n", "periodic", "fp32"])
def test_two_ended_falls_back_where_it_does_not_apply(env, case):
    """Below N = 4P, for a periodic factor, and for FP32 data the two-ended shape runs
    the sequential sweeps with their default shape: the same result as asking for them."""
    sb, torch = env
    M = 77
    if case == "small_n":
        N = 7
        fac = factor(sb, "penta", synth.random_penta_diagonals(seed=1, N=N))
    elif case == "periodic":
        N = 40
        a, b, c = (v.copy() for v in synth.random_tri_diagonals(seed=2, N=N))
        a[0], c[N - 1] = 0.3, -0.4
        b = np.sign(b) * (np.abs(a) + np.abs(c) + 1.0)
        fac = sb.sb_factor_shared_tri_periodic(a, b, c)
    else:
        N = 64
        fac = factor(sb, "tri", synth.random_tri_diagonals(seed=3, N=N))
    dtype = np.float32 if case == "fp32" else np.float64
    rhs = synth.rhs_normal(seed=5, N=N, M=M, ld=M, pad_value=CANARY)
    x = solve(sb, torch, fac, rhs, M, (512, 0, 1, sb.SB_ALGO_TWO_ENDED), dtype=dtype)
    xs = solve(sb, torch, fac, rhs, M, (256, 0, 1, sb.SB_ALGO_SEQUENTIAL), dtype=dtype)
    assert np.array_equal(x, xs)


def test_two_ended_shape_validation(env):
    sb, _ = env
    fac = factor(sb, "tri", synth.random_tri_diagonals(seed=1, N=16))
    for bad in [(1056, 0, 1, sb.SB_ALGO_TWO_ENDED), (100, 0, 1, sb.SB_ALGO_TWO_ENDED),
                (256, 0, 2, sb.SB_ALGO_TWO_ENDED)]:
        with pytest.raises(sb.SbError):
            sb.sb_shape_set(fac, bad)
    sb.sb_shape_set(fac, (1024, 0, 1, sb.SB_ALGO_TWO_ENDED))
