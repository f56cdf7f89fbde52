"""The allocation-free refined solve (sb_solve_batched_refined_noalloc).

Callers that cannot allocate device memory at solve time use this entry point: it
takes no workspace and draws its FP32 scratch from an array compiled into the
library.  Here it is called through the C ABI twice in a row (the second call
reuses the scratch left by the first, on different inputs) and each result must
match the ordinary workspace entry point within the FP64 tolerance of the other
tests.  This file is collected last so that a failure here leaves every other
test already run."""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


@pytest.mark.parametrize("kind,residual", [("tri", "native"), ("penta", "df32")])
def test_noalloc_matches_workspace_entry_point_twice(env, kind, residual):
    sb, torch = env
    N, M, ld = 512, 3000, 3001
    if kind == "tri":
        fac = sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", N, 2.0))
    else:
        fac = sb.sb_factor_shared_penta(*sb.sb_build_matrix("hinged", N, 0.25))
    L = sb.lib()
    res = sb.SB_ARITH_DF32 if residual == "df32" else sb.SB_ARITH_NATIVE
    for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs
        b = to_dev(synth.rhs_uniform(seed=seed, N=N, M=M, ld=ld, dtype=np.float32, pad_value=0.0), torch)
        x_ref = torch.zeros((N, ld), dtype=torch.float64, device="cuda")
        work = torch.empty((N, ld), dtype=torch.float32, device="cuda")
        sb.sb_solve_batched_refined(fac, b, x_ref, n_refine=2, residual_arith=residual, work=work, M=M)
        x = torch.full((N, ld), 5.0, dtype=torch.float64, device="cuda")
        rc = L.sb_solve_batched_refined_noalloc(fac.handle, b.data_ptr(), x.data_ptr(), M, ld, 2, res,
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == sb.SB_OK, sb.sb_last_error()
        torch.cuda.synchronize()
        got, want = to_host(x), to_host(x_ref)
        assert np.max(relerr_per_system(got[:, :M], want[:, :M])) <= TOL64, call
        assert np.all(got[:, M:] == 5.0), "padding columns were written"


def test_noalloc_rejects_batches_beyond_its_scratch(env):
    sb, torch = env
    N = 1024
    fac = sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", N, 0.5))
    M = (4 << 20) // N + 64  # (N-1)*M + M > 4 Mi elements
    b = torch.zeros((N, M), dtype=torch.float32, device="cuda")
    x = torch.zeros((N, M), dtype=torch.float64, device="cuda")
    rc = sb.lib().sb_solve_batched_refined_noalloc(fac.handle, b.data_ptr(), x.data_ptr(), M, M, 2,
                                                   sb.SB_ARITH_NATIVE, None)
    assert rc == sb.SB_ERR_INVALID_ARG
    assert "exceeds the allocation-free scratch" in sb.sb_last_error()
