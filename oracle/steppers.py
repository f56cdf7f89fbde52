"""Oracle: implicit time steps of the diffusion, hyperdiffusion and Cahn-Hilliard
workloads, and the FP64 reference for FP32-stored right-hand sides.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

State arrays are interleaved ``(N, M)`` (column m = simulation m).  Every step
builds its right-hand side from the previous state and solves with the shared
matrix through :mod:`oracle.banded`.
"""
from __future__ import annotations

import numpy as np

from . import advection, banded, matrices

__all__ = [
    "SharedTri", "SharedPenta",
    "SharedTriPeriodic", "diffusion_be_step", "diffusion_cn_rhs", "diffusion_cn_rhs_periodic",
    "hyper_be_step", "hyper_cn_rhs",
    "ch_rhs", "ch_step", "solve_fp32_rhs",
    "SharedPentaPeriodic", "ch_rhs_periodic", "ch_step_periodic", "coarsening_length",
    "convergence_error", "forced_ch_rhs_periodic", "forced_ch_step_periodic",
]


class SharedTri:
    """A shared tridiagonal matrix, factorised once (section 3.1, Algorithm 1)."""

    def __init__(self, a, b, c):
        self.a, self.b, self.c = (np.asarray(v, dtype=np.float64) for v in (a, b, c))
        self.bh, self.ch = banded.tri_factor(self.a, self.b, self.c)

    def solve(self, d):
        return banded.tri_solve(self.a, self.bh, self.ch, d)

    def solve_adjoint(self, g):
        return banded.tri_solve_adjoint(self.a, self.bh, self.ch, g)

    def apply(self, x):
        return matrices.apply_tri(self.a, self.b, self.c, x)


class SharedTriPeriodic:
    """A shared periodic tridiagonal matrix (section 3.3): A' factorised once and
    z = A'^{-1} u solved once; every solve is a tridiagonal solve plus the
    Sherman-Morrison correction."""

    def __init__(self, a, b, c):
        self.a, self.b, self.c = (np.asarray(v, dtype=np.float64) for v in (a, b, c))
        self.fac = banded.tri_periodic_factor(self.a, self.b, self.c)

    def solve(self, d):
        return banded.tri_periodic_solve(self.fac, d)

    def solve_adjoint(self, g):
        return banded.tri_periodic_solve_adjoint(self.fac, g)

    def apply(self, x):
        return matrices.apply_tri_periodic(self.a, self.b, self.c, x)


class SharedPenta:
    """A shared pentadiagonal matrix, factorised once (section 4.1, Algorithm 3)."""

    def __init__(self, a, b, c, d, e):
        self.diags = tuple(np.asarray(v, dtype=np.float64) for v in (a, b, c, d, e))
        self.factors = banded.penta_factor(*self.diags)

    def solve(self, f):
        return banded.penta_solve(*self.factors, f)

    def solve_adjoint(self, g):
        return banded.penta_solve_adjoint(*self.factors, g)

    def apply(self, x):
        return matrices.apply_penta(*self.diags, x)


def diffusion_be_step(A: SharedTri, C):
    """Backward Euler: (I + r K) C^{n+1} = C^n."""
    return A.solve(C)


def diffusion_cn_rhs(N, sigma, C):
    """Crank-Nicolson right-hand side of section 3.2's scheme, with Dirichlet rows:
    sigma C_{i-1} + (1 - 2 sigma) C_i + sigma C_{i+1} = (I - sigma K) C."""
    sub, dia, sup = matrices.d2_dirichlet(N)
    return np.asarray(C, dtype=np.float64) + sigma * matrices.apply_tri(sub, dia, sup, C)


def diffusion_cn_rhs_periodic(N, sigma, C):
    """Crank-Nicolson right-hand side of section 3.2's periodic scheme:
    sigma C_{i-1} + (1 - 2 sigma) C_i + sigma C_{i+1} with the indices wrapping."""
    sub, dia, sup = matrices.d2_periodic(N)
    return np.asarray(C, dtype=np.float64) + sigma * matrices.apply_tri_periodic(sub, dia, sup, C)


def hyper_be_step(A: SharedPenta, C):
    """Backward Euler for hyperdiffusion: (I + r D4) C^{n+1} = C^n."""
    return A.solve(C)


def hyper_cn_rhs(N, sigma, C, closure="hinged"):
    """Crank-Nicolson right-hand side of section 4.2's scheme:
    -sigma C_{i-2} + 4 sigma C_{i-1} + (1 - 6 sigma) C_i + 4 sigma C_{i+1} - sigma C_{i+2}
    = (I - sigma D4) C, with the same D4 closure as the left-hand side."""
    if closure == "hinged":
        D4 = matrices.square_tridiag(*matrices.d2_dirichlet(N))
    else:
        D4 = matrices.d4_truncated(N)
    return np.asarray(C, dtype=np.float64) - sigma * matrices.apply_penta(*D4, C)


def ch_rhs(C, alpha):
    """Right-hand side of the semi-implicit Cahn-Hilliard scheme (section 5.1):
    f = C^n + alpha * D2_N (C^3 - C)^n, alpha = dt / dx^2 (dx = 1 in grid units),
    with the no-flux closure of D2_N.  (Section 5.1 prints f_i without the C^n
    term; the scheme it discretises has C^n on the right-hand side.)"""
    C = np.asarray(C, dtype=np.float64)
    N = C.shape[0]
    nl = C * C * C - C
    sub, dia, sup = matrices.d2_noflux(N)
    return C + alpha * matrices.apply_tri(sub, dia, sup, nl)


def ch_step(A: SharedPenta, C, alpha):
    """One semi-implicit Cahn-Hilliard step: (I + sigma D4_N) C^{n+1} = ch_rhs(C^n)."""
    return A.solve(ch_rhs(C, alpha))


class SharedPentaPeriodic:
    """A shared cyclic pentadiagonal matrix: A' factored once and the rank-2
    correction formed once (banded.penta_periodic_factor)."""

    def __init__(self, a, b, c, d, e):
        self.diags = tuple(np.asarray(v, dtype=np.float64) for v in (a, b, c, d, e))
        self.fac = banded.penta_periodic_factor(*self.diags)

    def solve(self, f):
        return banded.penta_periodic_solve(self.fac, f)

    def solve_adjoint(self, g):
        return banded.penta_periodic_solve_adjoint(self.fac, g)

    def apply(self, x):
        return matrices.apply_penta_periodic(*self.diags, x)


def ch_rhs_periodic(C, alpha):
    """Section 5.1's right-hand side with the paper's periodic ends:
    f = C^n + alpha * D2_P (C^3 - C)^n."""
    C = np.asarray(C, dtype=np.float64)
    N = C.shape[0]
    nl = C * C * C - C
    return C + alpha * matrices.apply_tri_periodic(*matrices.d2_periodic(N), nl)


def ch_step_periodic(A: SharedPentaPeriodic, C, alpha):
    """One semi-implicit Cahn-Hilliard step with periodic ends:
    (I + sigma D4_P) C^{n+1} = ch_rhs_periodic(C^n)."""
    return A.solve(ch_rhs_periodic(C, alpha))


def coarsening_length(C):
    """Section 5.3's typical domain size: ell = 1 / (1 - <C^2>) per simulation, with
    <C^2> = (1/L) int_0^L C^2 dx taken on the periodic grid as the mean of C_i^2
    (the rectangle rule, exact for the grid's trigonometric interpolant), then
    averaged over the simulations (the columns)."""
    C = np.asarray(C, dtype=np.float64)
    return float(np.mean(1.0 / (1.0 - np.mean(C * C, axis=0))))


def forced_ch_rhs_periodic(C, alpha, beta, amp, profile):
    """Right-hand side of the travelling-wave forced Cahn-Hilliard scheme (section
    6.1) in grid units, periodic ends:
        f = C^n + alpha D2_P (C^3 - C)^n + beta W(C^n) + amp_m g_i,
    with W the fifth-order Hamilton-Jacobi WENO derivative, left-biased for
    beta > 0 and right-biased for beta < 0 (the forcing wave's direction of travel),
    beta = dt v / dx, g_i the forcing profile (the paper: dt k cos(k eta_i)) and
    amp_m the amplitude of system m (the paper: f_0, one value per simulation)."""
    C = np.asarray(C, dtype=np.float64)
    f = ch_rhs_periodic(C, alpha)
    if beta != 0.0:
        f = f + beta * advection.weno5_derivative(C, -1 if beta > 0 else +1)
    g = np.asarray(profile, dtype=np.float64)[:, None]
    a = np.asarray(amp, dtype=np.float64)[None, :]
    return f + a * g


def forced_ch_step_periodic(A: SharedPentaPeriodic, C, alpha, beta, amp, profile):
    """One semi-implicit forced CH step: (I + sigma D4_P) C^{n+1} =
    forced_ch_rhs_periodic(C^n)."""
    return A.solve(forced_ch_rhs_periodic(C, alpha, beta, amp, profile))


def convergence_error(C_half, C_full):
    """E_N of the convergence study (section 5.2, Table 3) between the solution on N/2
    points and the one on N points of the same periodic grid family x_i = i L / N:
    the mean over the N/2 shared points of |C^(N/2)_i - C^(N)_(2i)|.  The paper does
    not define E_N; this reading reproduces its printed values."""
    C_half = np.asarray(C_half, dtype=np.float64)
    C_full = np.asarray(C_full, dtype=np.float64)
    assert C_full.shape[0] == 2 * C_half.shape[0]
    return float(np.mean(np.abs(C_half - C_full[::2])))


def solve_fp32_rhs(A, b32):
    """FP64 reference for a right-hand side stored in FP32: the FP32 values are
    promoted exactly to FP64 and solved with the FP64 oracle."""
    return A.solve(np.asarray(b32, dtype=np.float32).astype(np.float64))
