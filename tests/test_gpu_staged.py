"""GPU parity of the staged sweeps (SB_ALGO_STAGED, the sequential sweeps with their
row streams staged through shared memory) through the C ABI: element by element
against the FP64 oracle on the same seeded inputs, and against the sequential
sweeps, whose arithmetic they share (equal to the last bit), for every arithmetic
mode and dtype pair, primal and adjoint.  Sizes span several tiles with ragged last
tiles and padded ld, N below and above the ring depth (8 rows) and its batch (4),
and launch sizes from one warp to 1024 threads.

Tolerances as for the sequential sweeps: 1e-12 relative L2 per system for FP64
and double-float arithmetic, 2e-5 for FP32 arithmetic."""
import numpy as np
import pytest

import synth
from oracle import banded
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

CANARY = 12345.678
SHAPES = [(1, 1, 1), (3, 31, 32), (6, 40, 41), (7, 129, 131), (64, 200, 256), (513, 300, 301),
          (1024, 1000, 1000)]
# (arith, rhs dtype, x dtype, tolerance against the oracle)
CASES = [("native", np.float64, np.float64, 1e-12), ("native", np.float32, np.float32, 2e-5),
         ("native", np.float32, np.float64, 2e-5), ("df32", np.float64, np.float64, 1e-12),
         ("df32", np.float32, np.float64, 1e-12)]


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def code(sb, dt):
    return sb.SB_F64 if dt == np.float64 else sb.SB_F32


def oracle(kind, diags, rhs, adjoint):
    if kind == "tri":
        a, b, c = diags
        bh, ch = banded.tri_factor(a, b, c)
        return (banded.tri_solve_adjoint if adjoint else banded.tri_solve)(a, bh, ch, rhs)
    fac = banded.penta_factor(*diags)
    return (banded.penta_solve_adjoint if adjoint else banded.penta_solve)(*fac, rhs)


def solve(sb, torch, fac, rhs_host, M, arith, rt, xt, shape, adjoint):
    rhs = to_dev(rhs_host.astype(rt), torch)
    x = torch.full(rhs.shape, CANARY, dtype=torch.float64 if xt == np.float64 else torch.float32,
                   device="cuda")
    sb.sb_shape_set(fac, shape, arith=arith, rhs_dtype=code(sb, rt), x_dtype=code(sb, xt))
    sb.sb_solve_batched_ex(fac, rhs, x, transpose=adjoint, arith=arith, M=M, ld=rhs.shape[1])
    torch.cuda.synchronize()
    return to_host(x)


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("arith,rt,xt,tol", CASES)
@pytest.mark.parametrize("N,M,ld", SHAPES)
@pytest.mark.parametrize("kind", ["tri", "penta"])
def test_staged_matches_oracle_and_sequential(env, kind, N, M, ld, arith, rt, xt, tol, adjoint):
    sb, torch = env
    diags = (synth.random_tri_diagonals if kind == "tri" else synth.random_penta_diagonals)(seed=N, N=N)
    fac = (sb.sb_factor_shared_tri if kind == "tri" else sb.sb_factor_shared_penta)(*diags)
    rhs = synth.rhs_normal(seed=30 + N, N=N, M=M, ld=ld, pad_value=CANARY)
    if rt == np.float32:
        rhs = rhs.astype(np.float32).astype(np.float64)  # the oracle sees the stored FP32 values
    threads = 512 if arith == "df32" else 1024
    x = solve(sb, torch, fac, rhs, M, arith, rt, xt, (threads, 0, 1, sb.SB_ALGO_STAGED), adjoint)
    ref = oracle(kind, diags, rhs[:, :M], adjoint)
    assert np.max(relerr_per_system(x[:, :M], ref)) <= tol
    assert np.all(x[:, M:] == np.asarray(CANARY, dtype=xt)), "padding columns were written"
    xs = solve(sb, torch, fac, rhs, M, arith, rt, xt, (256, 0, 1, sb.SB_ALGO_SEQUENTIAL), adjoint)
    assert np.array_equal(x[:, :M], xs[:, :M]), "staged and sequential sweeps differ"


@pytest.mark.parametrize("threads", [32, 96, 256, 768])
def test_staged_launch_sizes(env, threads):
    """One warp to 24 warps per CTA: every tile is solved once (8193 systems, a
    ragged last tile, more tiles than warps in flight for small CTAs)."""
    sb, torch = env
    N, M = 37, 8193
    diags = synth.random_penta_diagonals(seed=5, N=N)
    fac = sb.sb_factor_shared_penta(*diags)
    rhs = synth.rhs_normal(seed=6, N=N, M=M, ld=M, pad_value=CANARY)
    x = solve(sb, torch, fac, rhs, M, "native", np.float64, np.float64, (threads, 0, 1, sb.SB_ALGO_STAGED), False)
    assert np.max(relerr_per_system(x, oracle("penta", diags, rhs, False))) <= 1e-12


def test_staged_falls_back_where_it_does_not_apply(env):
    """A periodic factor (no staged form) solved with the staged shape runs the
    sequential sweeps: same result as asking for them."""
    sb, torch = env
    N, M = 50, 100
    a, b, c = (v.copy() for v in synth.random_tri_diagonals(seed=9, N=N))
    a[0], c[N - 1] = 0.3, -0.4  # the corner entries of the periodic matrix
    b = np.sign(b) * (np.abs(a) + np.abs(c) + 1.0)
    fac = sb.sb_factor_shared_tri_periodic(a, b, c)
    rhs = synth.rhs_normal(seed=10, N=N, M=M, ld=M, pad_value=CANARY)
    x = solve(sb, torch, fac, rhs, M, "native", np.float64, np.float64, (1024, 0, 1, sb.SB_ALGO_STAGED), False)
    xs = solve(sb, torch, fac, rhs, M, "native", np.float64, np.float64, (256, 0, 1, sb.SB_ALGO_SEQUENTIAL), False)
    assert np.array_equal(x, xs)


def test_staged_shape_validation(env):
    sb, _ = env
    fac = sb.sb_factor_shared_tri(*synth.random_tri_diagonals(seed=1, N=16))
    for bad in [(1056, 0, 1, sb.SB_ALGO_STAGED), (1000, 0, 1, sb.SB_ALGO_STAGED), (256, 0, 2, sb.SB_ALGO_STAGED)]:
        with pytest.raises(sb.SbError):
            sb.sb_shape_set(fac, bad)
    with pytest.raises(sb.SbError):
        sb.sb_shape_set(fac, (1024, 0, 1, sb.SB_ALGO_STAGED), arith="df32")
    sb.sb_shape_set(fac, (1024, 0, 1, sb.SB_ALGO_STAGED))
