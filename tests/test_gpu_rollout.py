"""GPU parity of the checkpointed rollout adjoint (A^T solves with the shared
factors, per-system and batch-summed parameter gradients) against the oracle's
discrete adjoint, bitwise checkpoint invariance, central finite differences run
on the GPU forward rollout, the torch.autograd.Function, and the rollout workload
(N = 512, 2^16 systems, 200 steps, checkpoints every 20) on sampled systems.

Bounds: GPU adjoint vs oracle adjoint 1e-10 relative; GPU adjoint vs finite
differences 1e-6 relative."""
import numpy as np
import pytest

import synth
from oracle import rollout
from tests.gpu_util import lib_or_skip, relerr_per_system, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_or_skip()


CASES = {
    "diffusion": dict(kind="diffusion", N=24, p=0.5, dt=0.0, amp=1.0),
    "hyperdiffusion": dict(kind="hyperdiffusion", N=20, p=0.25, dt=0.0, amp=1.0),
    "ch_grid": dict(kind="cahn_hilliard", N=32, p=synth.CH_GAMMA_GRID, dt=synth.CH_DT_GRID, amp=0.1),
    "ch_nonlinear": dict(kind="cahn_hilliard", N=16, p=1.0, dt=0.05, amp=0.9),
}


def oracle_problem(c, p=None):
    p = c["p"] if p is None else p
    if c["kind"] == "diffusion":
        return rollout.diffusion_problem(c["N"], p)
    if c["kind"] == "hyperdiffusion":
        return rollout.hyperdiffusion_problem(c["N"], p)
    return rollout.ch_problem(c["N"], p, c["dt"])


def gpu_grads(sb, torch, c, x0, y, T, k, M_total=None, p=None):
    """(loss, grad_C0, per-system dp, scalar dp) through the C ABI."""
    N = c["N"]
    p = c["p"] if p is None else p
    bc = {"diffusion": "dirichlet", "hyperdiffusion": "hinged", "cahn_hilliard": "noflux"}[c["kind"]]
    st = sb.sb_stepper_create(c["kind"], "be", bc, N, p, c["dt"])
    M = x0.shape[1]
    M_total = M if M_total is None else M_total
    d0 = to_dev(x0, torch) if isinstance(x0, np.ndarray) else x0
    dy = to_dev(y, torch) if isinstance(y, np.ndarray) else y
    work = torch.empty(sb.sb_rollout_workspace_bytes(st, M, T, k) // 8, dtype=torch.float64, device="cuda")
    CT = torch.empty_like(d0)
    sb.sb_rollout_forward(st, d0, CT, T, k, work)
    gCT = 2.0 * (CT - dy) / (N * M_total)
    gC0 = torch.empty_like(d0)
    dp_sys = torch.empty(M, dtype=torch.float64, device="cuda")
    dp = torch.zeros((), dtype=torch.float64, device="cuda")
    sb.sb_rollout_backward(st, gCT, gC0, T, k, work, grad_param=dp, grad_param_per_system=dp_sys)
    torch.cuda.synchronize()
    loss = float(((CT - dy) ** 2).sum().item()) / (N * M_total)
    return loss, gC0, dp_sys, dp


def gpu_loss(sb, torch, c, d0, dy, T, p=None):
    N = c["N"]
    p = c["p"] if p is None else p
    bc = {"diffusion": "dirichlet", "hyperdiffusion": "hinged", "cahn_hilliard": "noflux"}[c["kind"]]
    st = sb.sb_stepper_create(c["kind"], "be", bc, N, p, c["dt"])
    C = d0.clone()
    sb.sb_stepper_run(st, C, T, mode="direct")
    torch.cuda.synchronize()
    return float(((C - dy) ** 2).sum().item()) / (N * d0.shape[1])


@pytest.mark.parametrize("case", list(CASES))
def test_rollout_adjoint_matches_oracle(env, case):
    sb, torch = env
    c = CASES[case]
    N, M, T, k = c["N"], 40, 13, 5
    x0 = synth.rhs_uniform(seed=1, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    y = synth.rhs_uniform(seed=2, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    L, gC0, dp_sys, dp = gpu_grads(sb, torch, c, x0, y, T, k)
    Lo, g_ref, dp_ref = rollout.adjoint(oracle_problem(c), x0, y, T)
    assert abs(L - Lo) <= 1e-12 * abs(Lo)
    assert np.max(relerr_per_system(to_host(gC0), g_ref)) <= 1e-10
    assert np.max(np.abs(to_host(dp_sys) - dp_ref)) <= 1e-10 * np.max(np.abs(dp_ref))
    assert abs(dp.item() - dp_ref.sum()) <= 1e-10 * abs(dp_ref.sum())


@pytest.mark.parametrize("case", ["diffusion", "ch_nonlinear"])
def test_checkpointing_is_bitwise_invariant(env, case):
    sb, torch = env
    c = CASES[case]
    N, M, T = c["N"], 64, 13
    x0 = synth.rhs_uniform(seed=3, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    y = synth.rhs_uniform(seed=4, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    results = [gpu_grads(sb, torch, c, x0, y, T, k) for k in (1, 4, 13, 20)]
    _, g1, s1, d1 = results[0]
    for _, g, s, d in results[1:]:
        assert torch.equal(g, g1) and torch.equal(s, s1) and torch.equal(d, d1)


@pytest.mark.parametrize("case", list(CASES))
def test_rollout_adjoint_matches_gpu_finite_differences(env, case):
    sb, torch = env
    c = CASES[case]
    N, M, T, k = c["N"], 16, 9, 4
    x0 = synth.rhs_uniform(seed=5, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    y = synth.rhs_uniform(seed=6, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    _, gC0, _, dp = gpu_grads(sb, torch, c, x0, y, T, k)
    d0, dy = to_dev(x0, torch), to_dev(y, torch)
    v = to_dev(np.random.default_rng(7).standard_normal(x0.shape), torch)

    def rich(fun, h):
        cen = lambda hh: (fun(hh) - fun(-hh)) / (2 * hh)
        return (4 * cen(h / 2) - cen(h)) / 3

    fd = rich(lambda t: gpu_loss(sb, torch, c, d0 + t * v, dy, T), 1e-3)
    ad = float((gC0 * v).sum().item())
    assert abs(ad - fd) <= 1e-6 * abs(fd)
    h = 1e-3 * c["p"]
    fdp = rich(lambda t: gpu_loss(sb, torch, c, d0, dy, T, p=c["p"] + t), h)
    assert abs(dp.item() - fdp) <= 1e-6 * abs(fdp)


def test_autograd_function_matches_abi(env):
    sb, torch = env
    c = CASES["ch_nonlinear"]
    N, M, T, k = c["N"], 32, 11, 4
    x0 = synth.rhs_uniform(seed=8, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    y = synth.rhs_uniform(seed=9, N=N, M=M, lo=-c["amp"], hi=c["amp"])
    C0 = to_dev(x0, torch).requires_grad_(True)
    p = torch.tensor(c["p"], dtype=torch.float64, device="cuda", requires_grad=True)
    CT = sb.SharedLHSRollout.apply(C0, p, c["kind"], N, c["dt"], T, k)
    loss = ((CT - to_dev(y, torch)) ** 2).sum() / (N * M)
    gC0, gp = torch.autograd.grad(loss, (C0, p))
    _, g_ref, _, dp_ref = gpu_grads(sb, torch, c, x0, y, T, k)
    # torch forms dL/dC_T itself (its own rounding of 2 (C_T - y) / (N M)), so the
    # comparison is to rounding level rather than bitwise
    assert np.max(relerr_per_system(to_host(gC0), to_host(g_ref))) <= 1e-13
    assert abs(gp.item() - dp_ref.item()) <= 1e-13 * abs(dp_ref.item())


@pytest.mark.parametrize("kind", ["diffusion", "cahn_hilliard"])
def test_rollout_workload_sampled_systems(env, kind):
    """N = 512, 2^16 systems, 200 steps, checkpoints every 20 (CH: the 4 pi domain
    with dx = 2 pi / 256, gamma' and dt' as the coarsening workload)."""
    sb, torch = env
    w = synth.WORKLOADS["adjoint_rollout"]
    N, M, T, k = w["N"], w["M"], w["steps"], w["ckpt_every"]
    if kind == "diffusion":
        c = dict(kind="diffusion", N=N, p=w["r"], dt=0.0, amp=1.0)
    else:
        c = dict(kind="cahn_hilliard", N=N, p=w["gamma"], dt=w["dt"], amp=0.1)
    x0 = synth.torch_uniform(w["seed"], N, M, -c["amp"], c["amp"], torch.float64, "cuda")
    y = synth.torch_uniform(w["seed"] + 1, N, M, -c["amp"], c["amp"], torch.float64, "cuda")
    _, gC0, dp_sys, dp = gpu_grads(sb, torch, c, x0, y, T, k)
    cols = torch.as_tensor(np.linspace(0, M - 1, 128).astype(np.int64), device="cuda")
    x0s, ys = to_host(x0[:, cols]), to_host(y[:, cols])
    _, g_ref, dp_ref = rollout.adjoint(oracle_problem(c), x0s, ys, T, M_total=M)
    assert np.max(relerr_per_system(to_host(gC0[:, cols]), g_ref)) <= 1e-10
    assert np.max(np.abs(to_host(dp_sys[cols]) - dp_ref)) <= 1e-10 * np.max(np.abs(dp_ref))
    total = float(np.sum(to_host(dp_sys)))
    assert abs(dp.item() - total) <= 1e-12 * abs(total)
