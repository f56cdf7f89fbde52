"""GPU parity of the mixed-precision refinement and the multi-group launch.

Reference: the FP64 oracle applied to the FP32 right-hand side promoted exactly to
FP64.  Bounds: a plain FP32 solve is FP32-accurate (2e-5); each refinement pass
must shrink the error; after two passes the error is below 1e-10 (the refined-path
target).  The multi-group workload (N = 128 / 512 / 2048, r = 0.1 / 0.5 / 2.0,
2^21 right-hand sides split 4:2:1, two refinements, one call) is checked per
group on systems sampled across each batch."""
import numpy as np
import pytest

import synth
from oracle import banded, matrices, steppers
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


def make(sb, kind, N, seed):
    if kind == "tri":
        d = synth.random_tri_diagonals(seed=seed, N=N)
        a, b, c = d
        bh, ch = banded.tri_factor(a, b, c)
        return sb.sb_factor_shared_tri(*d), (lambda r: banded.tri_solve(a, bh, ch, r))
    d = synth.random_penta_diagonals(seed=seed, N=N)
    fac = banded.penta_factor(*d)
    return sb.sb_factor_shared_penta(*d), (lambda r: banded.penta_solve(*fac, r))


@pytest.mark.parametrize("residual", ["native", "df32"])
@pytest.mark.parametrize("kind", ["tri", "penta"])
@pytest.mark.parametrize("N,M,ld", [(1, 5, 5), (2, 40, 41), (9, 100, 128), (300, 333, 333)])
def test_refinement_contracts_to_fp64_accuracy(env, kind, N, M, ld, residual):
    sb, torch = env
    fac, ref_fn = make(sb, kind, N, seed=N + 3)
    b32 = synth.rhs_uniform(seed=N, N=N, M=M, ld=ld, dtype=np.float32, pad_value=9.0)
    ref = ref_fn(b32[:, :M].astype(np.float64))
    d_b = to_dev(b32, torch)
    work = torch.full((N, ld), -1.0, dtype=torch.float32, device="cuda")
    errs = []
    for n in (0, 1, 2):
        x = torch.full((N, ld), 7.0, dtype=torch.float64, device="cuda")
        sb.sb_solve_batched_refined(fac, d_b, x, n_refine=n, residual_arith=residual, work=work, M=M)
        torch.cuda.synchronize()
        out = to_host(x)
        assert np.all(out[:, M:] == 7.0)
        errs.append(np.max(relerr_per_system(out[:, :M], ref)))
    assert errs[0] <= 2e-5
    assert errs[2] <= 1e-10, errs
    assert errs[1] <= max(errs[0] * 1e-2, 1e-13) and errs[2] <= max(errs[1], 1e-13), errs


@pytest.mark.parametrize("residual", ["native", "df32"])
@pytest.mark.parametrize("kind,N,M", [("tri", 37, 70), ("penta", 37, 70), ("tri", 3, 33), ("penta", 6, 33),
                                      ("tri", 2048, 100), ("penta", 1400, 65), ("penta", 2000, 65),
                                      ("penta", 2400, 40)])
def test_refinement_passes_alternate_direction(env, kind, N, M, residual):
    """FP32 right-hand sides take the fused passes: pass k eliminates from the top
    (A = LU) for even k and from the bottom (the rows of J A J) for odd k, each
    correction pass merged into the backward sweep before it.  One to four passes
    cover both directions of the merged and of the last pass (n = 2 with the FP64
    residual runs the paired-tile form, always with an 8-row ring).  Shared memory
    holds the coefficients and a ring per thread: 16 rows (512 threads) for N <= 37,
    8 rows for tri N = 2048 and penta N = 1400 (512 threads) and penta N = 2000
    (416 threads); penta N = 2400 leaves no room and runs the separate passes.
    The random matrices are nonsymmetric, so a wrong reversal of J A J's diagonals
    stops the contraction."""
    sb, torch = env
    fac, ref_fn = make(sb, kind, N, seed=N + 11)
    ld = M + 3
    b32 = synth.rhs_uniform(seed=N + 1, N=N, M=M, ld=ld, dtype=np.float32, pad_value=9.0)
    ref = ref_fn(b32[:, :M].astype(np.float64))
    d_b = to_dev(b32, torch)
    work = torch.full((N, ld), -1.0, dtype=torch.float32, device="cuda")
    errs = []
    for n in (0, 1, 2, 3, 4):
        x = torch.full((N, ld), 7.0, dtype=torch.float64, device="cuda")
        sb.sb_solve_batched_refined(fac, d_b, x, n_refine=n, residual_arith=residual, work=work, M=M)
        torch.cuda.synchronize()
        out = to_host(x)
        assert np.all(out[:, M:] == 7.0)
        errs.append(np.max(relerr_per_system(out[:, :M], ref)))
    assert errs[0] <= 2e-5, errs
    assert errs[1] <= max(errs[0] * 1e-2, 1e-13), errs
    assert max(errs[2:]) <= 1e-10, errs


@pytest.mark.parametrize("residual", ["native", "df32"])
@pytest.mark.parametrize("kind,N", [("tri", 7), ("penta", 9)])
def test_two_refinements_many_tiles_per_warp(env, kind, N, residual):
    """With two refinements and the FP64 residual each warp carries two tiles two
    sweeps apart (the double-float residual runs one tile at a time).  200003
    systems are 6251 tiles, several per warp on every SM, the last one ragged, so the
    steps with one tile, with two, and the odd and even tile counts per warp all run;
    every system is checked."""
    sb, torch = env
    M = 200003
    fac, ref_fn = make(sb, kind, N, seed=N + 21)
    b32 = synth.rhs_uniform(seed=N + 2, N=N, M=M, ld=M, dtype=np.float32, pad_value=0.0)
    ref = ref_fn(b32.astype(np.float64))
    work = torch.empty((N, M), dtype=torch.float32, device="cuda")
    x = torch.empty((N, M), dtype=torch.float64, device="cuda")
    sb.sb_solve_batched_refined(fac, to_dev(b32, torch), x, n_refine=2, residual_arith=residual, work=work)
    torch.cuda.synchronize()
    assert np.max(relerr_per_system(to_host(x), ref)) <= 1e-10


def test_refinement_without_reversed_rows(env):
    """A = [[1, 1], [1, 0]] factors from the top, but J A J = [[0, 1], [1, 1]] has a
    zero first pivot: the solve then runs the passes without alternating."""
    sb, torch = env
    a, b, c = np.array([0.0, 1.0]), np.array([1.0, 0.0]), np.array([1.0, 0.0])
    fac = sb.sb_factor_shared_tri(a, b, c)
    M = 40
    b32 = synth.rhs_uniform(seed=5, N=2, M=M, ld=M, dtype=np.float32, pad_value=0.0)
    ref = np.linalg.solve(np.array([[1.0, 1.0], [1.0, 0.0]]), b32.astype(np.float64))
    work = torch.zeros((2, M), dtype=torch.float32, device="cuda")
    for n in (1, 2, 3):
        x = torch.zeros((2, M), dtype=torch.float64, device="cuda")
        sb.sb_solve_batched_refined(fac, to_dev(b32, torch), x, n_refine=n, work=work)
        torch.cuda.synchronize()
        assert np.max(relerr_per_system(to_host(x), ref)) <= 1e-12, n


@pytest.mark.parametrize("arith,rt,xt,tol", [("native", "f64", "f64", 1e-12), ("df32", "f64", "f64", 1e-12),
                                             ("df32", "f32", "f64", 1e-12), ("native", "f32", "f32", 2e-5)])
def test_groups_without_refinement(env, arith, rt, xt, tol):
    sb, torch = env
    tdt = {"f64": torch.float64, "f32": torch.float32}
    Ns, Ms = (5, 64, 300), (1000, 77, 300)
    facs, refs, rhs, xs, hosts = [], [], [], [], []
    for g, (N, M) in enumerate(zip(Ns, Ms)):
        fac, ref_fn = make(sb, "penta", N, seed=100 + g)
        h = synth.rhs_normal(seed=g, N=N, M=M).astype(np.float32 if rt == "f32" else np.float64)
        facs.append(fac)
        refs.append(ref_fn(h.astype(np.float64)))
        rhs.append(to_dev(h, torch))
        xs.append(torch.zeros((N, M), dtype=tdt[xt], device="cuda"))
    sb.sb_solve_batched_groups(facs, rhs, xs, arith=arith)
    torch.cuda.synchronize()
    for g in range(3):
        assert np.max(relerr_per_system(to_host(xs[g]), refs[g])) <= tol, g


@pytest.mark.parametrize("kind", ["tri", "penta"])
@pytest.mark.parametrize("n_refine,residual", [(1, "native"), (2, "native"), (2, "df32"), (3, "native")])
def test_refined_groups_of_different_n(env, kind, n_refine, residual):
    """Refined solves of three groups of different N in one launch, in every pass
    form the launch can pick: two FP64-residual passes take the paired tiles, the
    other counts and the double-float residual the single-tile merged passes.
    Every system of every group is checked against the oracle."""
    sb, torch = env
    Ns, Ms = (5, 64, 300), (1000, 77, 3001)
    facs, refs, rhs, xs, work = [], [], [], [], []
    for g, (N, M) in enumerate(zip(Ns, Ms)):
        fac, ref_fn = make(sb, kind, N, seed=200 + g)
        h = synth.rhs_uniform(seed=g + 7, N=N, M=M, ld=M, dtype=np.float32, pad_value=0.0)
        facs.append(fac)
        refs.append(ref_fn(h.astype(np.float64)))
        rhs.append(to_dev(h, torch))
        xs.append(torch.zeros((N, M), dtype=torch.float64, device="cuda"))
        work.append(torch.empty((N, M), dtype=torch.float32, device="cuda"))
    sb.sb_solve_batched_groups(facs, rhs, xs, n_refine=n_refine, residual_arith=residual, work=work)
    torch.cuda.synchronize()
    for g in range(3):
        err = np.max(relerr_per_system(to_host(xs[g]), refs[g]))
        assert err <= (1e-10 if n_refine >= 2 else 1e-9), (g, err)


def test_groups_reject_mixed_bandwidth(env):
    sb, torch = env
    f1, _ = make(sb, "tri", 8, 1)
    f2, _ = make(sb, "penta", 8, 2)
    r = [torch.zeros((8, 4), dtype=torch.float64, device="cuda") for _ in range(2)]
    x = [torch.zeros((8, 4), dtype=torch.float64, device="cuda") for _ in range(2)]
    with pytest.raises(sb.SbError) as ei:
        sb.sb_solve_batched_groups([f1, f2], r, x)
    assert ei.value.code == sb.SB_ERR_UNSUPPORTED


def test_refinement_rejects_missing_workspace(env):
    sb, torch = env
    fac, _ = make(sb, "tri", 16, 1)
    b = torch.zeros((16, 8), dtype=torch.float32, device="cuda")
    x = torch.zeros((16, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(sb.SbError):
        sb.sb_solve_batched_refined(fac, b, x, n_refine=1, work=None)
    small = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(sb.SbError):
        sb.sb_solve_batched_refined(fac, b, x, n_refine=1, work=small)


def test_multigroup_workload_two_refinements(env):
    """Three tridiagonal groups, 2^21 FP32 right-hand sides split 4:2:1, two
    refinement passes with the FP64 residual, all groups in one call."""
    sb, torch = env
    w = synth.WORKLOADS["multigroup_fp32"]
    Ms = synth.group_split(w["total"], w["ratio"], w["N"])
    facs, rhs, xs, work = [], [], [], []
    for g, (N, r, M) in enumerate(zip(w["N"], w["r"], Ms)):
        facs.append(sb.sb_factor_shared_tri(*sb.sb_build_matrix("diffusion", N, r)))
        rhs.append(synth.torch_uniform(w["seed"] + g, N, M, -1.0, 1.0, torch.float32, "cuda"))
        xs.append(torch.empty((N, M), dtype=torch.float64, device="cuda"))
        work.append(torch.empty((N, M), dtype=torch.float32, device="cuda"))
    sb.sb_solve_batched_groups(facs, rhs, xs, n_refine=w["n_refine"], work=work)
    torch.cuda.synchronize()
    for g, (N, r, M) in enumerate(zip(w["N"], w["r"], Ms)):
        cols = torch.as_tensor(np.linspace(0, M - 1, 256).astype(np.int64), device="cuda")
        b = to_host(rhs[g][:, cols]).astype(np.float64)
        A = steppers.SharedTri(*matrices.diffusion_matrix(N, r))
        err = relerr_per_system(to_host(xs[g][:, cols]), A.solve(b))
        assert np.max(err) <= 1e-10, (g, np.max(err))
