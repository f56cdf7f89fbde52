"""GPU parity of the host-memory solve (chunked, copy/solve overlapped on internal
streams): pinned and pageable host arrays, chunks that do not divide the batch,
ld > M, in-place host arrays, both arithmetic modes and the transposed solve."""
import numpy as np
import pytest

import synth
from oracle import banded
from tests.gpu_util import lib_or_skip, relerr_per_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("arith,transpose", [("native", False), ("df32", False), ("native", True)])
@pytest.mark.parametrize("chunk", [0, 100, 1000])
def test_host_solve_matches_oracle(env, pinned, arith, transpose, chunk):
    sb, torch = env
    N, M, ld = 200, 1000, 1003
    diags = synth.random_penta_diagonals(seed=3, N=N)
    fac = sb.sb_factor_shared_penta(*diags)
    host = synth.rhs_normal(seed=4, N=N, M=M, ld=ld, pad_value=2.5)
    rhs = torch.from_numpy(host.copy())
    x = torch.full_like(rhs, 2.5)
    if pinned:
        rhs, x = rhs.pin_memory(), x.pin_memory()
    work = torch.empty(sb.sb_host_workspace_bytes(fac, M, chunk), dtype=torch.uint8, device="cuda")
    sb.sb_solve_batched_host(fac, rhs, x, work, transpose=transpose, arith=arith, chunk_systems=chunk, M=M)
    torch.cuda.synchronize()
    out = x.numpy()
    fo = banded.penta_factor(*diags)
    ref = (banded.penta_solve_adjoint if transpose else banded.penta_solve)(*fo, host[:, :M])
    assert np.max(relerr_per_system(out[:, :M], ref)) <= 1e-12
    assert np.all(out[:, M:] == 2.5)


def test_host_solve_in_place_and_errors(env):
    sb, torch = env
    N, M = 64, 500
    diags = synth.random_tri_diagonals(seed=5, N=N)
    fac = sb.sb_factor_shared_tri(*diags)
    host = synth.rhs_uniform(seed=6, N=N, M=M)
    t = torch.from_numpy(host.copy()).pin_memory()
    work = torch.empty(sb.sb_host_workspace_bytes(fac, M, 128), dtype=torch.uint8, device="cuda")
    sb.sb_solve_batched_host(fac, t, t, work, chunk_systems=128)
    torch.cuda.synchronize()
    a, b, c = diags
    bh, ch = banded.tri_factor(a, b, c)
    assert np.max(relerr_per_system(t.numpy(), banded.tri_solve(a, bh, ch, host))) <= 1e-12
    with pytest.raises(sb.SbError):  # workspace too small
        sb.sb_solve_batched_host(fac, t, t, work[:16], chunk_systems=128)
    dev = torch.zeros((N, M), dtype=torch.float64, device="cuda")
    with pytest.raises(sb.SbError):  # device memory where host memory is expected
        sb.sb_solve_batched_host(fac, dev, t, work, chunk_systems=128)


@pytest.mark.parametrize("kind", ["penta", "tri_periodic", "penta_periodic"])
def test_chunking_does_not_change_the_bits(env, kind):
    """The chunk size only changes which copies overlap which solves: the default
    chunking and 128-system chunks give the same bits (each system's arithmetic is
    the same), in place too, for A and A^T, periodic and not."""
    sb, torch = env
    N, M, ld = 300, 777, 800
    if kind == "penta":
        fac = sb.sb_factor_shared_penta(*synth.random_penta_diagonals(seed=8, N=N))
    elif kind == "tri_periodic":
        fac = sb.sb_factor_shared_tri_periodic(*sb.sb_build_matrix("diffusion_periodic", N, 0.6))
    else:
        fac = sb.sb_factor_shared_penta_periodic(*sb.sb_build_matrix("ch_periodic", N, 0.4))
    host = synth.rhs_normal(seed=9, N=N, M=M, ld=ld, pad_value=-1.5)
    for transpose in (False, True):
        rhs = torch.from_numpy(host.copy()).pin_memory()
        outs = []
        for chunk in (0, 128):
            x = torch.full_like(rhs, -1.5).pin_memory()
            work = torch.empty(sb.sb_host_workspace_bytes(fac, M, chunk), dtype=torch.uint8, device="cuda")
            sb.sb_solve_batched_host(fac, rhs, x, work, transpose=transpose, chunk_systems=chunk, M=M)
            torch.cuda.synchronize()
            outs.append(x.numpy().copy())
        assert np.array_equal(outs[0], outs[1])
        assert np.all(outs[0][:, M:] == -1.5)
        work = torch.empty(sb.sb_host_workspace_bytes(fac, M), dtype=torch.uint8, device="cuda")
        sb.sb_solve_batched_host(fac, rhs, rhs, work, transpose=transpose, M=M)  # in place, direct
        torch.cuda.synchronize()
        assert np.array_equal(rhs.numpy()[:, :M], outs[0][:, :M])


@pytest.mark.parametrize("N,chunk", [(5, 3), (201, 7), (77, 0)])
def test_fp32_rhs_fp64_solution_with_odd_slot_sizes(env, N, chunk):
    """FP32 right-hand sides with FP64 solutions: with an odd N * chunk the FP64 part
    of each workspace slot follows an odd number of FP32 values, so this case checks
    the slot layout's alignment on the device (chunk 0 picks M itself when M is small)."""
    sb, torch = env
    M, ld = 29, 31
    diags = synth.random_penta_diagonals(seed=12, N=N)
    fac = sb.sb_factor_shared_penta(*diags)
    host = synth.rhs_uniform(seed=13, N=N, M=M, ld=ld, dtype=np.float32, pad_value=0.5)
    rhs = torch.from_numpy(host.copy()).pin_memory()
    x = torch.full((N, ld), 0.5, dtype=torch.float64).pin_memory()
    work = torch.empty(sb.sb_host_workspace_bytes(fac, M, chunk, rhs_dtype=sb.SB_F32, x_dtype=sb.SB_F64),
                       dtype=torch.uint8, device="cuda")
    sb.sb_solve_batched_host(fac, rhs, x, work, chunk_systems=chunk, M=M)
    torch.cuda.synchronize()
    fo = banded.penta_factor(*diags)
    ref = banded.penta_solve(*fo, host[:, :M].astype(np.float64))
    # FP32 sweeps of an exactly widened FP32 right-hand side
    assert np.max(relerr_per_system(x.numpy()[:, :M], ref)) <= 2e-5
    assert np.all(x.numpy()[:, M:] == 0.5)
