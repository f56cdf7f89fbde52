"""GPU parity of the partitioned solve (SB_ALGO_PARTITIONED) against the FP64
oracle on the same seeded inputs: FP32 rhs with FP32 and FP64 x, A and A^T, every
chunk length (8, 16, 32 rows), identity-padded and empty chunks, a ragged last tile
of systems, padding columns left alone, in-place solves, a sampled check at the
1024 x 65536 pentadiagonal size, the fallback to the sequential sweeps where the
partition does not apply, and no timed-out waits.

Tolerance: 2e-5 relative L2 per system, as for every FP32 path (a few hundred FP32
units of roundoff on these well-conditioned matrices; the chunked form adds a few
FP32 operations per element) and 1e-12 where the fallback runs in FP64."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
CANARY = 7.0
PART = (512, 0, 1, 1)  # threads, ctas_per_sm, systems_per_thread, SB_ALGO_PARTITIONED (16 chunks)
PART32 = (1024, 0, 1, 1)  # 32 chunks
PAIRS = (256, 0, 1, 1)  # 16 chunks, two systems per thread
VARIANTS = {"16chunks": PART, "32chunks": PART32, "pairs": PAIRS}


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def oracle(diags, rhs, adjoint):
    if len(diags) == 3:
        a, b, c = diags
        bh, ch = banded.tri_factor(a, b, c)
        return (banded.tri_solve_adjoint if adjoint else banded.tri_solve)(a, bh, ch, rhs)
    fac = banded.penta_factor(*diags)
    return (banded.penta_solve_adjoint if adjoint else banded.penta_solve)(*fac, rhs)


def factor(sb, diags):
    return (sb.sb_factor_shared_tri if len(diags) == 3 else sb.sb_factor_shared_penta)(*diags)


MATS = {
    "penta_random_N500_L16": lambda: synth.random_penta_diagonals(seed=5, N=500),
    "hinged_r0.25_N1024_L32": lambda: matrices.hyperdiffusion_matrix(1024, 0.25),
    "penta_random_N1000_padded": lambda: synth.random_penta_diagonals(seed=6, N=1000),
    "truncated_r2_N300_13_empty_chunks": lambda: matrices.hyperdiffusion_matrix(300, 2.0, "truncated"),
    "ch_N256_L8": lambda: matrices.ch_matrix(256, 0.0166),
    "penta_random_N64": lambda: synth.random_penta_diagonals(seed=7, N=64),
    "tri_diffusion_N256": lambda: matrices.diffusion_matrix(256, 0.5),
    "tri_random_N333": lambda: synth.random_tri_diagonals(seed=3, N=333),
    "tri_random_N777": lambda: synth.random_tri_diagonals(seed=4, N=777),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("xt", ["f32", "f64"])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_partitioned_matches_oracle(env, name, xt, variant):
    sb, torch = env
    diags = MATS[name]()
    N = len(diags[0])
    M, ld = 1000, 1004  # 31.25 tiles of 32 systems; 4 padding columns
    fac = factor(sb, diags)
    xcode = sb.SB_F64 if xt == "f64" else sb.SB_F32
    shape = VARIANTS[variant]
    sb.sb_shape_set(fac, shape, rhs_dtype=sb.SB_F32, x_dtype=xcode)
    assert sb.sb_shape_get(fac, rhs_dtype=sb.SB_F32, x_dtype=xcode) == shape
    rhs = synth.rhs_normal(seed=11, N=N, M=M, ld=ld, pad_value=CANARY).astype(np.float32)
    d = to_dev(rhs, torch)
    x = torch.full((N, ld), CANARY, dtype=torch.float64 if xt == "f64" else torch.float32, device="cuda")
    for adjoint in (False, True):
        sb.sb_solve_batched_ex(fac, d, x, transpose=adjoint, M=M)
        torch.cuda.synchronize()
        out = to_host(x).astype(np.float64)
        ref = oracle(diags, rhs[:, :M].astype(np.float64), adjoint)
        err = np.max(relerr_per_system(out[:, :M], ref))
        assert err <= TOL32, (name, xt, adjoint, err)
        assert np.all(out[:, M:] == CANARY), "padding columns were written"
    assert sb.sb_device_timeouts(0) == 0


@pytest.mark.parametrize("M", [1, 31, 32, 33, 4097])
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_partitioned_ragged_batches_and_in_place(env, M, variant):
    sb, torch = env
    diags = synth.random_penta_diagonals(seed=21, N=257)
    fac = factor(sb, diags)
    sb.sb_shape_set(fac, VARIANTS[variant], rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32)
    ld = (M + 3) // 4 * 4
    rhs = synth.rhs_uniform(seed=22, N=257, M=M, ld=ld, pad_value=CANARY).astype(np.float32)
    d = to_dev(rhs, torch)
    sb.sb_solve_batched(fac, d, M=M, ld=ld)  # in place
    torch.cuda.synchronize()
    out = to_host(d).astype(np.float64)
    assert np.max(relerr_per_system(out[:, :M], oracle(diags, rhs[:, :M].astype(np.float64), False))) <= TOL32
    assert np.all(out[:, M:] == CANARY)
    assert sb.sb_device_timeouts(0) == 0


@pytest.mark.parametrize("kind", ["penta", "tri"])
@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("N", [333, 512])
def test_partitioned_many_tiles_per_cta_every_system(env, kind, in_place, variant, N):
    """Several tiles per persistent CTA (3 to 4 on a 152-SM GPU) and a ragged last
    tile, every system against the oracle: each CTA's loads and stores run through
    more than one round, A and A^T, in place or not.  With N = 512 (16 chunks of 32
    rows) the two-system form keeps each tile's solution in tensor memory until the
    next tile and sends the partial last tile to its direct-store kernel; N = 333 is
    stored directly."""
    sb, torch = env
    M = 152 * 32 * 3 + 17
    ld = M + 3
    diags = (synth.random_penta_diagonals if kind == "penta" else synth.random_tri_diagonals)(seed=31, N=N)
    fac = factor(sb, diags)
    sb.sb_shape_set(fac, VARIANTS[variant], rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32)
    rhs = synth.rhs_normal(seed=32, N=N, M=M, ld=ld, pad_value=CANARY).astype(np.float32)
    for adjoint in (False, True):
        d = to_dev(rhs, torch)
        x = d if in_place else torch.full_like(d, CANARY)
        sb.sb_solve_batched_ex(fac, d, x, transpose=adjoint, M=M)
        torch.cuda.synchronize()
        out = to_host(x).astype(np.float64)
        ref = oracle(diags, rhs[:, :M].astype(np.float64), adjoint)
        assert np.max(relerr_per_system(out[:, :M], ref)) <= TOL32, adjoint
        assert np.all(out[:, M:] == CANARY)
    assert sb.sb_device_timeouts(0) == 0


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("xt", ["f32", "f64"])
def test_partitioned_with_misaligned_solution(env, variant, xt):
    """A solution array offset by one element from its allocation (so not aligned for
    the two-system stores) is still written correctly, and nothing outside it."""
    sb, torch = env
    N, M, ld = 300, 200, 204
    diags = synth.random_penta_diagonals(seed=33, N=N)
    fac = factor(sb, diags)
    xcode = sb.SB_F64 if xt == "f64" else sb.SB_F32
    sb.sb_shape_set(fac, VARIANTS[variant], rhs_dtype=sb.SB_F32, x_dtype=xcode)
    rhs = synth.rhs_normal(seed=34, N=N, M=M, ld=ld).astype(np.float32)
    d = to_dev(rhs, torch)
    base = torch.full((N * ld + 1,), CANARY, dtype=torch.float64 if xt == "f64" else torch.float32, device="cuda")
    x = base[1:].view(N, ld)
    sb.sb_solve_batched_ex(fac, d, x, M=M, ld=ld)
    torch.cuda.synchronize()
    out = to_host(x).astype(np.float64)
    assert np.max(relerr_per_system(out[:, :M], oracle(diags, rhs[:, :M].astype(np.float64), False))) <= TOL32
    assert np.all(out[:, M:] == CANARY) and float(base[0]) == CANARY
    assert sb.sb_device_timeouts(0) == 0


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_partitioned_fp32_at_full_size_sampled(env, variant):
    """The 1024 x 65536 pentadiagonal solve in FP32; 96 systems spread over the batch
    (first, last, ragged tile ends, random) against the oracle."""
    sb, torch = env
    N, M = 1024, 65536
    diags = sb.sb_build_matrix("hinged", N, 0.25)
    fac = sb.sb_factor_shared_penta(*diags)
    sb.sb_shape_set(fac, VARIANTS[variant], rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32)
    rhs = synth.torch_uniform(seed=2, N=N, M=M, lo=-1.0, hi=1.0, dtype=torch.float32, device="cuda")
    x = torch.empty_like(rhs)
    sb.sb_solve_batched(fac, rhs, x)
    torch.cuda.synchronize()
    g = np.random.default_rng(5)
    cols = np.unique(np.concatenate([[0, 31, 32, M - 33, M - 32, M - 1], g.integers(0, M, 90)]))
    idx = torch.from_numpy(cols).cuda()
    b = to_host(rhs[:, idx]).astype(np.float64)
    out = to_host(x[:, idx]).astype(np.float64)
    assert np.max(relerr_per_system(out, oracle(diags, b, False))) <= TOL32
    assert sb.sb_device_timeouts(0) == 0


@pytest.mark.parametrize("case", ["N40", "N2048", "ld_odd", "misaligned", "f64_rhs", "df32"])
def test_fallback_where_the_partition_does_not_apply(env, case):
    """A solve asked to use the partitioned algorithm where it does not apply runs
    the sequential sweeps and is still correct."""
    sb, torch = env
    N = {"N40": 40, "N2048": 2048}.get(case, 256)
    diags = synth.random_penta_diagonals(seed=9, N=N)
    fac = factor(sb, diags)
    M = 100
    ld = 101 if case == "ld_odd" else 104
    rt = sb.SB_F64 if case == "f64_rhs" else sb.SB_F32
    xt = sb.SB_F64 if case in ("f64_rhs", "df32") else sb.SB_F32
    arith = "df32" if case == "df32" else "native"
    sb.sb_shape_set(fac, PART, arith=arith, rhs_dtype=rt, x_dtype=xt)
    rhs = synth.rhs_normal(seed=3, N=N, M=M, ld=ld)
    if rt == sb.SB_F32:
        rhs = rhs.astype(np.float32)
    base = to_dev(rhs if case != "misaligned" else np.pad(rhs.ravel(), (1, 0)), torch)
    d = base[1:].view(N, ld) if case == "misaligned" else base
    x = torch.zeros((N, ld), dtype=torch.float64 if xt == sb.SB_F64 else torch.float32, device="cuda")
    sb.sb_solve_batched_ex(fac, d, x, arith=arith, M=M, ld=ld)
    torch.cuda.synchronize()
    ref = oracle(diags, rhs[:, :M].astype(np.float64), False)
    tol = TOL64 if (rt == sb.SB_F64 or case == "df32") else TOL32
    assert np.max(relerr_per_system(to_host(x)[:, :M].astype(np.float64), ref)) <= tol


def test_bad_partitioned_shapes_rejected(env):
    sb, _ = env
    fac = factor(sb, synth.random_penta_diagonals(seed=1, N=256))
    for bad in [(384, 0, 1, 1), (1024, 2, 1, 1), (512, 0, 2, 1), (1024, 0, 1, 9)]:
        with pytest.raises(sb.SbError):
            sb.sb_shape_set(fac, bad)


def test_autotune_fp32_headline_shape_is_correct(env):
    sb, torch = env
    N, M = 1024, 8192
    diags = sb.sb_build_matrix("hinged", N, 0.25)
    fac = sb.sb_factor_shared_penta(*diags)
    rhs = synth.torch_uniform(seed=3, N=N, M=M, lo=-1.0, hi=1.0, dtype=torch.float32, device="cuda")
    x = torch.empty_like(rhs)
    best, ms = sb.sb_autotune(fac, rhs, x)
    assert best[3] in (0, 1, 2, 3) and ms > 0
    assert sb.sb_shape_get(fac, rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32) == best
    sb.sb_solve_batched(fac, rhs, x)
    torch.cuda.synchronize()
    ref = oracle(diags, to_host(rhs[:, :256]).astype(np.float64), False)
    assert np.max(relerr_per_system(to_host(x[:, :256]).astype(np.float64), ref)) <= TOL32


FP64 = (128, 0, 1, 1)  # the small-tile FP64 form of SB_ALGO_PARTITIONED

MATS64 = {
    "tri_diffusion_N256_M1024": (lambda: matrices.diffusion_matrix(256, 0.5), 1024),
    "penta_random_N500": (lambda: synth.random_penta_diagonals(seed=15, N=500), 1000),
    "hinged_N512": (lambda: matrices.hyperdiffusion_matrix(512, 0.25), 777),
    "ch_N256": (lambda: matrices.ch_matrix(256, 0.0166), 333),
    "tri_random_N40_padded": (lambda: synth.random_tri_diagonals(seed=16, N=40), 65),
    "penta_random_N100_empty_chunks": (lambda: synth.random_penta_diagonals(seed=17, N=100), 9),
    # more tiles than resident CTAs: the block-Thomas form of the boundary solve (the
    # cases above have one tile per CTA and take cyclic reduction)
    "tri_diffusion_N256_M40000_thomas": (lambda: matrices.diffusion_matrix(256, 0.5), 40000),
    "hinged_N512_M30000_thomas": (lambda: matrices.hyperdiffusion_matrix(512, 0.25), 30000),
}


@pytest.mark.parametrize("name", list(MATS64))
def test_partitioned_fp64_matches_oracle(env, name):
    """The FP64 form against the FP64 oracle at the FP64 tolerance, A and A^T, ragged
    tiles of 8 systems, padding columns untouched, then in place; both boundary
    solvers (cyclic reduction for one tile per CTA, block Thomas beyond)."""
    sb, torch = env
    make, M = MATS64[name]
    diags = make()
    N = len(diags[0])
    ld = M + 3
    fac = factor(sb, diags)
    sb.sb_shape_set(fac, FP64)
    assert sb.sb_shape_get(fac) == FP64
    rhs = synth.rhs_normal(seed=19, N=N, M=M, ld=ld, pad_value=CANARY)
    d = to_dev(rhs, torch)
    x = torch.full_like(d, CANARY)
    for adjoint in (False, True):
        sb.sb_solve_batched_ex(fac, d, x, transpose=adjoint, M=M)
        torch.cuda.synchronize()
        out = to_host(x)
        err = np.max(relerr_per_system(out[:, :M], oracle(diags, rhs[:, :M], adjoint)))
        assert err <= TOL64, (name, adjoint, err)
        assert np.all(out[:, M:] == CANARY)
    sb.sb_solve_batched(fac, d, M=M, ld=ld)  # in place
    torch.cuda.synchronize()
    out = to_host(d)
    assert np.max(relerr_per_system(out[:, :M], oracle(diags, rhs[:, :M], False))) <= TOL64
    assert np.all(out[:, M:] == CANARY)


def test_partitioned_fp64_falls_back_outside_its_range(env):
    sb, torch = env
    diags = synth.random_penta_diagonals(seed=18, N=1000)  # N > 512: no FP64 partition
    fac = factor(sb, diags)
    sb.sb_shape_set(fac, FP64)
    rhs = synth.rhs_normal(seed=20, N=1000, M=50)
    d = to_dev(rhs, torch)
    x = torch.empty_like(d)
    sb.sb_solve_batched(fac, d, x)
    torch.cuda.synchronize()
    assert np.max(relerr_per_system(to_host(x), oracle(diags, rhs, False))) <= TOL64
