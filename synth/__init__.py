"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds random-number draws and workload sizes only. It contains none of
the solver's arithmetic (no matrix assembly, no factorisation, no sweep): the
oracle (``oracle/``) and the CUDA library (``paper_2107_05395_gb300``) each build
their own matrices from the scalar coefficients listed here.

Layout convention used everywhere: element ``(i, m)`` of a batch of ``M`` systems
of ``N`` unknowns lives at ``i * ld + m`` (system index fastest, the interleaved
layout of the paper's Fig. 2); host arrays are therefore shaped ``(N, ld)``.

Workload recipes (the paper's own workloads are synthetic; no dataset exists):

* ``tri_dirichlet``    -- N=256 unknowns, M=1024 right-hand sides, U[-1, 1], seed 1.
* ``penta_hyper``      -- N=1024, M=65536, N(0, 1), seed 2 (+ pure sine modes).
* ``multigroup_fp32``  -- three groups, N=(128, 512, 2048), 2^21 RHS split 4:2:1
                          as M=(1198592, 599040, 299520), U[-1, 1] stored FP32, seed 3.
* ``cahn_hilliard``    -- N=256, M=2^20 simulations, C0 ~ U[-0.1, 0.1], seed 4.
* ``adjoint_rollout``  -- N=512, M=2^16, 200 steps, targets U[-1,1] / U[-0.1,0.1], seed 5.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "WORKLOADS",
    "group_split",
    "rhs_uniform",
    "rhs_normal",
    "random_tri_diagonals",
    "random_penta_diagonals",
    "sine_mode_block",
    "cosine_mode_block",
    "fourier_mode_block",
    "ch_convergence_case",
    "forced_ch_convergence_case",
    "torch_uniform",
    "torch_normal",
]

# Scalar parameters of each workload.  ``r`` / ``sigma`` / ``gamma`` / ``dt`` are
# the coefficients that build the shared matrix; the builders live on each side.
CH_GAMMA_GRID = 0.01 / (2.0 * math.pi / 256.0) ** 2   # gamma' = gamma / dx^2, dx = 2*pi/256
CH_DT_GRID = 1.0e-3

WORKLOADS = {
    "tri_dirichlet": dict(N=256, M=1024, r=0.5, seed=1, dist="uniform"),
    "penta_hyper": dict(N=1024, M=65536, r=0.25, seed=2, dist="normal", decay_steps=10),
    "multigroup_fp32": dict(N=(128, 512, 2048), r=(0.1, 0.5, 2.0), total=1 << 21,
                            ratio=(4, 2, 1), seed=3, n_refine=2),
    "cahn_hilliard": dict(N=256, M=1 << 20, gamma=CH_GAMMA_GRID, dt=CH_DT_GRID,
                          steps=2000, seed=4, amp=0.1),
    "adjoint_rollout": dict(N=512, M=1 << 16, steps=200, ckpt_every=20, r=0.5,
                            gamma=CH_GAMMA_GRID, dt=CH_DT_GRID, seed=5),
    # convergence study of the periodic CH scheme (section 5.2): L = 2 pi, gamma = 0.01,
    # dt = 0.1 dx, C(x, 0) = eps cos(5 x); the final time is not printed (T = 20 read)
    "ch_convergence": dict(N=(64, 128, 256, 512, 1024, 2048, 4096, 8192), gamma=0.01,
                           eps=1e-6, k=5, dt_over_dx=0.1, T=20.0),
    # the same study for the travelling-wave forced CH scheme (section 6.1): forcing
    # f0 k cos(k eta) with k = 1, f0 = 1, wave speed v = 0.5
    "forced_ch_convergence": dict(N=(128, 256, 512, 1024, 2048, 4096), gamma=0.01, eps=1e-6,
                                  k_init=5, dt_over_dx=0.1, T=20.0, k=1.0, f0=1.0, v=0.5),
    # the flow-pattern batch of section 6.3: N = 512 on L = 2 pi, a 768 x 768 grid of
    # (f0 in [0, 2], <C> in [0, 1.5]) = 589 824 simulations, C0 = <C> + U[-0.1, 0.1]
    "forced_ch_map": dict(N=512, side=768, f0=(0.0, 2.0), mean=(0.0, 1.5), k=1.0, v=0.5,
                          gamma=0.01, dt_over_dx=0.1, T=50.0, seed=6, amp=0.1),
}


def forced_ch_convergence_case(N: int):
    """As ch_convergence_case, for the forced study's parameters (gamma' = gamma/dx^2,
    dt' = dt/dx^2, steps = ceil(T/dt), physical dt, C0 = eps cos(5 x_i))."""
    w = WORKLOADS["forced_ch_convergence"]
    dx = 2.0 * math.pi / N
    dt = w["dt_over_dx"] * dx
    steps = int(math.ceil(w["T"] / dt))
    C0 = w["eps"] * fourier_mode_block(N, [w["k_init"]], "cos")
    return w["gamma"] / dx ** 2, dt / dx ** 2, steps, dt, C0


def ch_convergence_case(N: int):
    """Grid-unit parameters of the convergence study at N points on [0, 2 pi):
    (gamma' = gamma / dx^2, dt' = dt / dx^2, steps = ceil(T / dt), physical dt, C0 of
    shape (N, 1) = eps cos(5 x_i) with x_i = i dx)."""
    w = WORKLOADS["ch_convergence"]
    dx = 2.0 * math.pi / N
    dt = w["dt_over_dx"] * dx
    steps = int(math.ceil(w["T"] / dt))
    C0 = w["eps"] * fourier_mode_block(N, [w["k"]], "cos")
    return w["gamma"] / dx ** 2, dt / dx ** 2, steps, dt, C0


def group_split(total: int, ratio, N) -> tuple:
    """Split ``total`` right-hand sides over groups in ``ratio`` (4:2:1 for the
    multi-group workload).  2^21 is not divisible by 7, so the unit is the largest
    multiple of 128 not above total/7/128*128 and the remainder goes to group 0.
    Returns the per-group batch sizes."""
    unit = (total // sum(ratio) // 128) * 128
    sizes = [unit * w for w in ratio]
    sizes[0] += total - sum(sizes)
    return tuple(int(s) for s in sizes)


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def rhs_uniform(seed: int, N: int, M: int, lo: float = -1.0, hi: float = 1.0,
                ld: int | None = None, dtype=np.float64, stream: int = 0,
                pad_value: float = np.nan) -> np.ndarray:
    """Interleaved batch ``(N, ld)`` with columns ``m < M`` i.i.d. U[lo, hi].
    Columns ``M <= m < ld`` are padding set to ``pad_value`` (a canary)."""
    ld = M if ld is None else ld
    out = np.full((N, ld), pad_value, dtype=dtype)
    out[:, :M] = _rng(seed, stream).uniform(lo, hi, size=(N, M)).astype(dtype)
    return out


def rhs_normal(seed: int, N: int, M: int, ld: int | None = None, dtype=np.float64,
               stream: int = 0, pad_value: float = np.nan) -> np.ndarray:
    """Interleaved batch ``(N, ld)`` with columns ``m < M`` i.i.d. N(0, 1)."""
    ld = M if ld is None else ld
    out = np.full((N, ld), pad_value, dtype=dtype)
    out[:, :M] = _rng(seed, stream).standard_normal(size=(N, M)).astype(dtype)
    return out


def random_tri_diagonals(seed: int, N: int, margin: float = 0.5, stream: int = 7):
    """Random nonsymmetric, row-diagonally-dominant tridiagonal matrix as diagonals
    ``(a, b, c)`` (sub, main, super; a[0] and c[N-1] are outside the matrix and set
    to 0).  |b_i| >= |a_i| + |c_i| + margin, signs of b random."""
    g = _rng(seed, stream)
    a = g.uniform(-1.0, 1.0, N)
    c = g.uniform(-1.0, 1.0, N)
    a[0] = 0.0
    c[-1] = 0.0
    sign = np.where(g.uniform(size=N) < 0.5, -1.0, 1.0)
    b = sign * (np.abs(a) + np.abs(c) + margin + g.uniform(0.0, 1.0, N))
    return a, b, c


def random_penta_diagonals(seed: int, N: int, margin: float = 0.5, stream: int = 11):
    """Random nonsymmetric, row-diagonally-dominant pentadiagonal matrix as the
    five diagonals ``(a, b, c, d, e)`` (offsets -2, -1, 0, +1, +2, the naming of
    section 4.1).  Entries outside the matrix are set to 0."""
    g = _rng(seed, stream)
    a, b, d, e = (g.uniform(-1.0, 1.0, N) for _ in range(4))
    a[:2] = 0.0
    b[:1] = 0.0
    d[-1:] = 0.0
    e[-2:] = 0.0
    sign = np.where(g.uniform(size=N) < 0.5, -1.0, 1.0)
    c = sign * (np.abs(a) + np.abs(b) + np.abs(d) + np.abs(e) + margin + g.uniform(0.0, 1.0, N))
    return a, b, c, d, e


def sine_mode_block(N: int, modes) -> np.ndarray:
    """Columns are the discrete Dirichlet sine modes sin((i+1) k pi / (N+1)),
    i = 0..N-1, one column per k in ``modes``.  Shape ``(N, len(modes))``."""
    # the integer phase (i+1)k is reduced modulo 2(N+1) exactly before scaling, so
    # the argument stays in [0, 2 pi) and each sample is accurate to about an ulp
    i = np.arange(1, N + 1, dtype=np.int64)[:, None]
    k = np.asarray(modes, dtype=np.int64)[None, :]
    phase = (i * k) % (2 * (N + 1))
    return np.sin(phase.astype(np.float64) * np.pi / (N + 1))


def cosine_mode_block(N: int, modes, amplitude: float = 1.0) -> np.ndarray:
    """Columns are amplitude * cos(k pi (i + 1/2) / N), the cell-centred Neumann
    modes, one per k in ``modes``.  Shape ``(N, len(modes))``."""
    # cos(k pi (2i+1) / (2N)): the integer phase k(2i+1) is reduced modulo 4N first
    i = np.arange(N, dtype=np.int64)[:, None]
    k = np.asarray(modes, dtype=np.int64)[None, :]
    phase = (k * (2 * i + 1)) % (4 * N)
    return amplitude * np.cos(phase.astype(np.float64) * np.pi / (2 * N))


def fourier_mode_block(N: int, modes, kind: str = "cos") -> np.ndarray:
    """Columns are the periodic grid modes cos(2 pi k i / N) (or sin), i = 0..N-1,
    one column per k in ``modes``.  Shape ``(N, len(modes))``."""
    # the integer phase k i is reduced modulo N exactly before scaling
    i = np.arange(N, dtype=np.int64)[:, None]
    k = np.asarray(modes, dtype=np.int64)[None, :]
    phase = ((i * k) % N).astype(np.float64) * (2.0 * np.pi / N)
    return np.cos(phase) if kind == "cos" else np.sin(phase)


# --- device-side generators for the full-size workloads (torch Philox stream) ---

def torch_uniform(seed: int, N: int, M: int, lo: float, hi: float, dtype, device, ld=None):
    """Full-size interleaved U[lo, hi] batch drawn on ``device`` from torch's
    generator seeded with ``seed``.  Returns a tensor of shape ``(N, ld)``; padding
    columns (``m >= M``) are NaN.  The host copy of any sampled columns gives the
    oracle identical bits."""
    import torch
    ld = M if ld is None else ld
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.full((N, ld), float("nan"), dtype=dtype, device=device)
    out[:, :M].uniform_(lo, hi, generator=gen)
    return out


def torch_normal(seed: int, N: int, M: int, dtype, device, ld=None):
    """Full-size interleaved N(0, 1) batch drawn on ``device`` (see torch_uniform)."""
    import torch
    ld = M if ld is None else ld
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.full((N, ld), float("nan"), dtype=dtype, device=device)
    out[:, :M].normal_(0.0, 1.0, generator=gen)
    return out
