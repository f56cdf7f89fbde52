"""GPU parity of the periodic tridiagonal solve (section 3.3) against the oracle's
Sherman-Morrison solve on the same seeded inputs: A and A^T, native FP64, FP32,
FP32 -> FP64 and double-float arithmetic, both systems-per-thread shapes, ragged
tiles and padding canaries, in place, the host-memory call, the periodic diffusion
matrix with its exact Fourier-mode decay, and the rejections (N < 3, refinement).

Tolerances: 1e-12 relative L2 per system (FP64 and double-float), 2e-5 (FP32)."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
CANARY = 5.5


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def random_periodic(seed, N):
    a, b, c = synth.random_tri_diagonals(seed, N)
    g = np.random.default_rng([seed, 99])
    a = a.copy()
    c = c.copy()
    a[0] = g.uniform(-1, 1)
    c[N - 1] = g.uniform(-1, 1)
    b = np.sign(b) * (np.abs(a) + np.abs(c) + 0.5 + g.uniform(0, 1, N))
    return a, b, c


def oracle(diags, rhs, adjoint):
    fac = banded.tri_periodic_factor(*diags)
    return (banded.tri_periodic_solve_adjoint if adjoint else banded.tri_periodic_solve)(fac, rhs)


CASES = [(3, 7), (4, 33), (17, 64), (256, 1000), (1000, 515), (1024, 65)]


@pytest.mark.parametrize("N,M", CASES)
@pytest.mark.parametrize("mode", ["native64", "native32", "f32_to_f64", "df32"])
@pytest.mark.parametrize("spt", [1, 2])
def test_periodic_matches_oracle(env, N, M, mode, spt):
    sb, torch = env
    diags = random_periodic(N, N)
    fac = sb.sb_factor_shared_tri_periodic(*diags)
    ld = M + 3
    rt, xt, arith = {"native64": (np.float64, np.float64, "native"),
                     "native32": (np.float32, np.float32, "native"),
                     "f32_to_f64": (np.float32, np.float64, "native"),
                     "df32": (np.float64, np.float64, "df32")}[mode]
    codes = {np.float64: sb.SB_F64, np.float32: sb.SB_F32}
    sb.sb_shape_set(fac, (128, 0, spt, 0), arith=arith, rhs_dtype=codes[rt], x_dtype=codes[xt])
    rhs = synth.rhs_normal(seed=N + 1, N=N, M=M, ld=ld, pad_value=CANARY).astype(rt)
    d = to_dev(rhs, torch)
    x = torch.full((N, ld), CANARY, dtype=torch.float64 if xt == np.float64 else torch.float32,
                   device="cuda")
    tol = TOL32 if mode in ("native32", "f32_to_f64") else TOL64
    for adjoint in (False, True):
        sb.sb_solve_batched_ex(fac, d, x, transpose=adjoint, arith=arith, M=M)
        torch.cuda.synchronize()
        out = to_host(x).astype(np.float64)
        ref = oracle(diags, rhs[:, :M].astype(np.float64), adjoint)
        err = np.max(relerr_per_system(out[:, :M], ref))
        assert err <= tol, (N, M, mode, spt, adjoint, err)
        assert np.all(out[:, M:] == CANARY)


def test_periodic_in_place_and_default_shape(env):
    sb, torch = env
    N, M = 300, 777
    diags = random_periodic(7, N)
    fac = sb.sb_factor_shared_tri_periodic(*diags)
    rhs = synth.rhs_uniform(seed=8, N=N, M=M)
    d = to_dev(rhs, torch)
    sb.sb_solve_batched(fac, d)
    torch.cuda.synchronize()
    assert np.max(relerr_per_system(to_host(d), oracle(diags, rhs, False))) <= TOL64
    # FP32 rhs: the partitioned default falls back to the sweeps for a periodic handle
    r32 = synth.rhs_uniform(seed=9, N=N, M=M, dtype=np.float32)
    d32 = to_dev(r32, torch)
    x32 = torch.empty_like(d32)
    sb.sb_solve_batched(fac, d32, x32)
    torch.cuda.synchronize()
    assert np.max(relerr_per_system(to_host(x32), oracle(diags, r32.astype(np.float64), False))) <= TOL32


def test_periodic_diffusion_fourier_modes_and_host_call(env):
    """The periodic diffusion matrix from the library's builder: one solve divides
    cos/sin(2 pi k i / N) by 1 + 4 r sin^2(pi k / N), through the host-memory call."""
    sb, torch = env
    N, r = 1024, 0.5
    fac = sb.sb_factor_shared_tri_periodic(*sb.sb_build_matrix("diffusion_periodic", N, r))
    modes = list(range(0, N // 2 + 1, 7))
    X = np.concatenate([synth.fourier_mode_block(N, modes, "cos"),
                        synth.fourier_mode_block(N, modes, "sin")], axis=1)
    lam = 1.0 + 4.0 * r * np.sin(np.pi * np.asarray(modes + modes) / N) ** 2
    h_rhs = torch.from_numpy(np.ascontiguousarray(X)).pin_memory()
    h_x = torch.empty_like(h_rhs).pin_memory()
    M = X.shape[1]
    work = torch.empty(sb.sb_host_workspace_bytes(fac, M), dtype=torch.uint8, device="cuda")
    sb.sb_solve_batched_host(fac, h_rhs, h_x, work)
    torch.cuda.synchronize()
    assert np.max(np.abs(h_x.numpy() - X / lam[None, :])) <= 1e-13


def test_periodic_full_size_sampled(env):
    """Tridiagonal periodic N = 1024, M = 65536 (FP64) on sampled systems."""
    sb, torch = env
    N, M = 1024, 65536
    diags = sb.sb_build_matrix("diffusion_periodic", N, 0.5)
    fac = sb.sb_factor_shared_tri_periodic(*diags)
    rhs = synth.torch_uniform(seed=12, N=N, M=M, lo=-1.0, hi=1.0, dtype=torch.float64, device="cuda")
    x = torch.empty_like(rhs)
    sb.sb_solve_batched(fac, rhs, x)
    torch.cuda.synchronize()
    cols = np.unique(np.concatenate([[0, 31, 32, M - 1], np.random.default_rng(1).integers(0, M, 60)]))
    idx = torch.from_numpy(cols).cuda()
    ref = oracle(diags, to_host(rhs[:, idx]), False)
    assert np.max(relerr_per_system(to_host(x[:, idx]), ref)) <= TOL64


def test_periodic_rejections(env):
    sb, torch = env
    with pytest.raises(sb.SbError):
        sb.sb_factor_shared_tri_periodic([1.0, 1.0], [4.0, 4.0], [1.0, 1.0])
    with pytest.raises(sb.SbError):
        sb.sb_factor_shared_tri_periodic([1.0, 1.0, 1.0], [0.0, 4.0, 4.0], [1.0, 1.0, 1.0])
    fac = sb.sb_factor_shared_tri_periodic(*random_periodic(3, 64))
    b32 = torch.zeros((64, 8), dtype=torch.float32, device="cuda")
    x64 = torch.zeros((64, 8), dtype=torch.float64, device="cuda")
    work = torch.empty((64, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(sb.SbError):
        sb.sb_solve_batched_refined(fac, b32, x64, n_refine=1, work=work)
