"""GPU checks of the launch-shape table and the autotuner: every candidate shape
gives the same (oracle-exact) result, the autotuner stores a valid shape, and bad
shapes are rejected."""
import numpy as np
import pytest

import synth
from oracle import banded
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


@pytest.mark.parametrize("arith", ["native", "df32"])
@pytest.mark.parametrize("shape", [(32, 1, 1), (64, 2, 2), (128, 0, 1), (256, 1, 2), (512, 0, 2)])
def test_every_shape_matches_oracle(env, arith, shape):
    sb, torch = env
    N, M = 77, 1000  # M not a multiple of 64: ragged last tile for two systems per thread
    diags = synth.random_penta_diagonals(seed=7, N=N)
    fac = sb.sb_factor_shared_penta(*diags)
    sb.sb_shape_set(fac, shape, arith=arith)
    assert sb.sb_shape_get(fac, arith=arith) == shape + (0,)
    rhs = synth.rhs_normal(seed=8, N=N, M=M, ld=M + 3, pad_value=7.0)
    d = to_dev(rhs, torch)
    x = torch.full_like(d, 7.0)
    for transpose in (False, True):
        sb.sb_solve_batched_ex(fac, d, x, transpose=transpose, arith=arith, M=M)
        torch.cuda.synchronize()
        out = to_host(x)
        fac_o = banded.penta_factor(*diags)
        ref = (banded.penta_solve_adjoint if transpose else banded.penta_solve)(*fac_o, rhs[:, :M])
        assert np.max(relerr_per_system(out[:, :M], ref)) <= 1e-12
        assert np.all(out[:, M:] == 7.0)


def test_autotune_stores_a_valid_shape(env):
    sb, torch = env
    N, M = 256, 8192
    diags = sb.sb_build_matrix("diffusion", N, 0.5)
    fac = sb.sb_factor_shared_tri(*diags)
    rhs = to_dev(synth.rhs_uniform(seed=1, N=N, M=M), torch)
    x = torch.empty_like(rhs)
    best, ms = sb.sb_autotune(fac, rhs, x, arith="df32")
    assert best[0] % 32 == 0 and 32 <= best[0] <= 512 and best[2] in (1, 2) and ms > 0
    assert sb.sb_shape_get(fac, arith="df32") == best
    sb.sb_solve_batched_ex(fac, rhs, x, arith="df32")
    torch.cuda.synchronize()
    a, b, c = diags
    bh, ch = banded.tri_factor(a, b, c)
    ref = banded.tri_solve(a, bh, ch, to_host(rhs))
    assert np.max(relerr_per_system(to_host(x), ref)) <= 1e-12


def test_bad_shapes_rejected(env):
    sb, _ = env
    fac = sb.sb_factor_shared_tri(*synth.random_tri_diagonals(seed=1, N=8))
    for bad in [(48, 0, 1), (1024, 0, 1), (64, -1, 1), (64, 0, 3), (64, 0, 1, 1), (256, 0, 2, 1),
                (256, 0, 1, 7)]:
        with pytest.raises(sb.SbError):
            sb.sb_shape_set(fac, bad)


def test_measured_rates_are_plausible(env):
    """The arithmetic-rate probe: every rate positive, FP32 FMA well above FP64 FMA
    (GB300's FP64 pipe is a small fraction of its FP32 pipe), and the FP64 FMA rate
    below 2 per clock per SM at the highest SM clock (the pipe's issue limit)."""
    sb, torch = env
    r = sb.sb_measure_rates(0)
    assert r["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert r["fp64_fma_per_s"] > 0 and r["fp32_fma_per_s"] > 0 and r["f64_f32_conversions_per_s"] > 0
    assert r["fp32_fma_per_s"] > 10 * r["fp64_fma_per_s"]
    assert r["fp64_fma_per_s"] <= 2.0 * r["sm_count"] * 2.2e9 * 1.05
