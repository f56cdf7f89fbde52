"""GPU parity: batched shared-LHS solves and adjoint solves through the C ABI,
element by element against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 paths 1e-12 relative L2 per system (the accuracy target of the
FP64 path); FP32 storage/arithmetic 2e-5 relative L2 per system, i.e. a few
hundred FP32 units of roundoff, which covers the error growth of the sweeps on
the diagonally dominant (condition number below ~10) matrices used here."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices, steppers
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
CANARY = 12345.678


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def run_solve(sb, torch, fac, rhs_host, M, dtype=np.float64, adjoint=False, inplace=False):
    """Copy a (N, ld) host batch to the device, solve through the ABI, copy back."""
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    rhs = to_dev(rhs_host.astype(dtype), torch)
    x = rhs if inplace else torch.full_like(rhs, CANARY)
    fn = sb.sb_solve_batched_adjoint if adjoint else sb.sb_solve_batched
    fn(fac, rhs, x, M=M, ld=rhs.shape[1])
    torch.cuda.synchronize()
    assert x.dtype == tdt
    return to_host(x)


def oracle_tri(diags, rhs, adjoint=False):
    a, b, c = diags
    bh, ch = banded.tri_factor(a, b, c)
    return (banded.tri_solve_adjoint if adjoint else banded.tri_solve)(a, bh, ch, rhs)


def oracle_penta(diags, rhs, adjoint=False):
    fac = banded.penta_factor(*diags)
    return (banded.penta_solve_adjoint if adjoint else banded.penta_solve)(*fac, rhs)


SHAPES = [(1, 1, 1), (2, 5, 8), (3, 31, 32), (7, 129, 131), (64, 200, 256), (513, 300, 301),
          (1000, 70, 70)]


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("N,M,ld", SHAPES)
def test_tri_random_fp64(env, N, M, ld, adjoint):
    sb, torch = env
    diags = synth.random_tri_diagonals(seed=N, N=N)
    fac = sb.sb_factor_shared_tri(*diags)
    rhs = synth.rhs_uniform(seed=10 + N, N=N, M=M, ld=ld, pad_value=CANARY)
    x = run_solve(sb, torch, fac, rhs, M, adjoint=adjoint)
    ref = oracle_tri(diags, rhs[:, :M], adjoint)
    assert np.max(relerr_per_system(x[:, :M], ref)) <= TOL64
    assert np.all(x[:, M:] == CANARY), "padding columns were written"


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("N,M,ld", SHAPES)
def test_penta_random_fp64(env, N, M, ld, adjoint):
    sb, torch = env
    diags = synth.random_penta_diagonals(seed=N, N=N)
    fac = sb.sb_factor_shared_penta(*diags)
    rhs = synth.rhs_normal(seed=20 + N, N=N, M=M, ld=ld, pad_value=CANARY)
    x = run_solve(sb, torch, fac, rhs, M, adjoint=adjoint)
    ref = oracle_penta(diags, rhs[:, :M], adjoint)
    assert np.max(relerr_per_system(x[:, :M], ref)) <= TOL64
    assert np.all(x[:, M:] == CANARY)


@pytest.mark.parametrize("kind", ["tri", "penta"])
@pytest.mark.parametrize("algorithm", ["default", "sequential"])
def test_fp32_storage_and_arithmetic(env, kind, algorithm):
    """FP32 storage and arithmetic; the default shape of an FP32 solve is the
    partitioned algorithm, the sequential sweeps are forced once."""
    sb, torch = env
    N, M = 300, 515
    if kind == "tri":
        diags = synth.random_tri_diagonals(seed=5, N=N)
        fac = sb.sb_factor_shared_tri(*diags)
        orc = oracle_tri
    else:
        diags = synth.random_penta_diagonals(seed=5, N=N)
        fac = sb.sb_factor_shared_penta(*diags)
        orc = oracle_penta
    if algorithm == "sequential":
        sb.sb_shape_set(fac, (256, 0, 1, 0), rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32)
    else:
        assert sb.sb_shape_get(fac, rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F32)[3] == 1
    rhs = synth.rhs_uniform(seed=6, N=N, M=M, dtype=np.float32)
    for adj in (False, True):
        x = run_solve(sb, torch, fac, rhs, M, dtype=np.float32, adjoint=adj)
        ref = orc(diags, rhs.astype(np.float64), adj)
        assert np.max(relerr_per_system(x, ref)) <= TOL32


@pytest.mark.parametrize("kind", ["tri", "penta"])
def test_in_place(env, kind):
    sb, torch = env
    N, M = 100, 77
    diags = (synth.random_tri_diagonals if kind == "tri" else synth.random_penta_diagonals)(seed=9, N=N)
    fac = (sb.sb_factor_shared_tri if kind == "tri" else sb.sb_factor_shared_penta)(*diags)
    rhs = synth.rhs_uniform(seed=11, N=N, M=M)
    x = run_solve(sb, torch, fac, rhs, M, inplace=True)
    ref = (oracle_tri if kind == "tri" else oracle_penta)(diags, rhs)
    assert np.max(relerr_per_system(x, ref)) <= TOL64


def test_workload_tri_dirichlet_all_systems(env):
    """Tridiagonal backward-Euler diffusion: r = 0.5, N = 256, 1024 RHS ~ U[-1, 1]."""
    sb, torch = env
    w = synth.WORKLOADS["tri_dirichlet"]
    N, M = w["N"], w["M"]
    fac = sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", N, w["r"]))
    rhs = synth.rhs_uniform(seed=w["seed"], N=N, M=M)
    x = run_solve(sb, torch, fac, rhs, M)
    A = steppers.SharedTri(*matrices.diffusion_matrix(N, w["r"]))
    assert np.max(relerr_per_system(x, A.solve(rhs))) <= TOL64


@pytest.mark.parametrize("closure", ["hinged", "truncated"])
def test_workload_penta_hyper_full_size_all_systems(env, closure):
    """Pentadiagonal hyperdiffusion A = I + 0.25 D4, N = 1024, 65536 RHS ~ N(0, 1):
    every system against the oracle, at full size."""
    sb, torch = env
    w = synth.WORKLOADS["penta_hyper"]
    N, M = w["N"], w["M"]
    fac = sb.sb_factor_shared_penta(*sb.sb_build_matrix(closure, N, w["r"]))
    rhs = synth.rhs_normal(seed=w["seed"], N=N, M=M)
    x = run_solve(sb, torch, fac, rhs, M)
    A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, w["r"], closure))
    err = relerr_per_system(x, A.solve(rhs))
    assert np.max(err) <= TOL64, (np.max(err), np.median(err))


def test_workload_penta_sine_mode_decay_ten_steps(env):
    """Systems 0..N-1 hold the pure sine modes k = 1..N; ten implicit steps with the
    hinged matrix must multiply mode k by (1 + r 16 sin^4(k pi / (2(N+1))))^-10."""
    sb, torch = env
    w = synth.WORKLOADS["penta_hyper"]
    N, r = w["N"], w["r"]
    M = 4096
    rhs = synth.rhs_normal(seed=w["seed"], N=N, M=M)
    k = np.arange(1, N + 1)
    rhs[:, :N] = synth.sine_mode_block(N, k)
    fac = sb.sb_factor_shared_penta(*sb.sb_build_matrix("hinged", N, r))
    t = to_dev(rhs, torch)
    for _ in range(w["decay_steps"]):
        sb.sb_solve_batched(fac, t)
    torch.cuda.synchronize()
    x = to_host(t)
    lam = 1.0 + r * 16.0 * np.sin(k * np.pi / (2 * (N + 1))) ** 4
    expect = synth.sine_mode_block(N, k) * lam ** -w["decay_steps"]
    assert np.max(np.abs(x[:, :N] - expect)) <= 1e-13


# ------------------------------------------------------------- error paths

def test_rejects_host_pointer_and_bad_sizes(env):
    sb, torch = env
    N = 16
    fac = sb.sb_factor_shared_tri(*synth.random_tri_diagonals(seed=1, N=N))
    host = np.zeros((N, 8))
    dev = torch.zeros((N, 8), dtype=torch.float64, device="cuda")
    L = sb.lib()
    rc = L.sb_solve_batched(fac.handle, host.ctypes.data, dev.data_ptr(), 8, 8, 0, None)
    assert rc == sb.SB_ERR_INVALID_ARG and "host" in sb.sb_last_error()
    # ld < M
    assert L.sb_solve_batched(fac.handle, dev.data_ptr(), dev.data_ptr(), 8, 4, 0, None) == sb.SB_ERR_INVALID_ARG
    # misaligned pointer
    assert L.sb_solve_batched(fac.handle, dev.data_ptr() + 4, dev.data_ptr(), 4, 4, 0, None) == sb.SB_ERR_INVALID_ARG
    # partial overlap of rhs and x
    assert L.sb_solve_batched(fac.handle, dev.data_ptr(), dev.data_ptr() + 8, 4, 7, 0, None) == sb.SB_ERR_INVALID_ARG
    assert "overlap" in sb.sb_last_error()
    # range past the end of the allocation (ld too large for the buffer)
    small = torch.zeros(N * 8, dtype=torch.float64, device="cuda")
    big_ld = 1 << 22
    rc = L.sb_solve_batched(fac.handle, small.data_ptr(), small.data_ptr(), 8, big_ld, 0, None)
    assert rc == sb.SB_ERR_INVALID_ARG
    # M = 0 is a no-op
    assert L.sb_solve_batched(fac.handle, dev.data_ptr(), dev.data_ptr(), 0, 8, 0, None) == sb.SB_OK
    # unknown dtype
    assert L.sb_solve_batched(fac.handle, dev.data_ptr(), dev.data_ptr(), 8, 8, 7, None) == sb.SB_ERR_INVALID_ARG


# ------------------------------------------------ sb_solve_batched_ex / df32

def run_ex(sb, torch, fac, rhs_host, M, rhs_dtype, x_dtype, arith, adjoint=False):
    tin = torch.float64 if rhs_dtype == np.float64 else torch.float32
    tout = torch.float64 if x_dtype == np.float64 else torch.float32
    rhs = to_dev(rhs_host.astype(rhs_dtype), torch)
    x = torch.full(rhs.shape, CANARY, dtype=tout, device="cuda")
    sb.sb_solve_batched_ex(fac, rhs, x, transpose=adjoint, arith=arith, M=M, ld=rhs.shape[1])
    torch.cuda.synchronize()
    return to_host(x)


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("kind", ["tri", "penta"])
@pytest.mark.parametrize("N,M,ld", [(1, 3, 3), (2, 33, 40), (5, 100, 100), (130, 257, 260), (1024, 300, 301)])
def test_df32_fp64_io_matches_oracle(env, kind, N, M, ld, adjoint):
    sb, torch = env
    if kind == "tri":
        diags = synth.random_tri_diagonals(seed=40 + N, N=N)
        fac = sb.sb_factor_shared_tri(*diags)
        orc = oracle_tri
    else:
        diags = synth.random_penta_diagonals(seed=40 + N, N=N)
        fac = sb.sb_factor_shared_penta(*diags)
        orc = oracle_penta
    rhs = synth.rhs_normal(seed=50 + N, N=N, M=M, ld=ld, pad_value=CANARY)
    x = run_ex(sb, torch, fac, rhs, M, np.float64, np.float64, "df32", adjoint)
    ref = orc(diags, rhs[:, :M], adjoint)
    assert np.max(relerr_per_system(x[:, :M], ref)) <= TOL64
    assert np.all(x[:, M:] == CANARY)


@pytest.mark.parametrize("kind", ["tri", "penta"])
@pytest.mark.parametrize("algorithm", ["default", "sequential"])
def test_fp32_rhs_fp64_solution(env, kind, algorithm):
    """FP32-stored right-hand side solved into an FP64 solution: with df32
    arithmetic to FP64 accuracy of the promoted input, with native FP32 to FP32
    accuracy."""
    sb, torch = env
    N, M = 512, 1000
    if kind == "tri":
        diags = tuple(sb.sb_build_matrix("diffusion", N, 2.0))
        fac = sb.sb_factor_shared_tri(*diags)
        A = steppers.SharedTri(*matrices.diffusion_matrix(N, 2.0))
    else:
        diags = tuple(sb.sb_build_matrix("hinged", N, 0.25))
        fac = sb.sb_factor_shared_penta(*diags)
        A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, 0.25, "hinged"))
    if algorithm == "sequential":
        sb.sb_shape_set(fac, (256, 0, 1, 0), rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F64)
    b32 = synth.rhs_uniform(seed=3, N=N, M=M, dtype=np.float32)
    ref = steppers.solve_fp32_rhs(A, b32)
    x = run_ex(sb, torch, fac, b32, M, np.float32, np.float64, "df32")
    assert np.max(relerr_per_system(x, ref)) <= TOL64
    x = run_ex(sb, torch, fac, b32, M, np.float32, np.float64, "native")
    assert np.max(relerr_per_system(x, ref)) <= TOL32


def test_workload_penta_df32_full_size_all_systems(env):
    sb, torch = env
    w = synth.WORKLOADS["penta_hyper"]
    N, M = w["N"], w["M"]
    fac = sb.sb_factor_shared_penta(*sb.sb_build_matrix("hinged", N, w["r"]))
    rhs = synth.rhs_normal(seed=w["seed"], N=N, M=M)
    x = run_ex(sb, torch, fac, rhs, M, np.float64, np.float64, "df32")
    A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, w["r"], "hinged"))
    err = relerr_per_system(x, A.solve(rhs))
    assert np.max(err) <= TOL64, (np.max(err), np.median(err))


def test_ex_rejects_unsupported_and_bad_alias(env):
    sb, torch = env
    N = 16
    fac = sb.sb_factor_shared_tri(*synth.random_tri_diagonals(seed=1, N=N))
    d64 = torch.zeros((N, 8), dtype=torch.float64, device="cuda")
    d32 = torch.zeros((N, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(sb.SbError) as ei:   # FP64 rhs into FP32 x is not offered
        sb.sb_solve_batched_ex(fac, d64, d32, arith="native")
    assert ei.value.code == sb.SB_ERR_UNSUPPORTED
    with pytest.raises(sb.SbError) as ei:   # df32 with FP32 output is not offered
        sb.sb_solve_batched_ex(fac, d32, d32, arith="df32")
    assert ei.value.code == sb.SB_ERR_UNSUPPORTED
    L = sb.lib()
    rc = L.sb_solve_batched_ex(fac.handle, 0, d32.data_ptr(), 1, d32.data_ptr(), 0, 8, 8, 0, None)
    assert rc == sb.SB_ERR_INVALID_ARG and "alias" in sb.sb_last_error()
    assert L.sb_solve_batched_ex(fac.handle, 2, d64.data_ptr(), 0, d64.data_ptr(), 0, 8, 8, 0, None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_solve_batched_ex(fac.handle, 0, d64.data_ptr(), 0, d64.data_ptr(), 0, 8, 8, 9, None) == sb.SB_ERR_INVALID_ARG
