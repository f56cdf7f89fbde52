"""Oracle: discrete adjoint of an implicit rollout with a shared matrix.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no counterpart for this part (it only runs rollouts forward).  The
rollout is x_{n+1} = A(p)^{-1} F(x_n), n = 0 .. T-1, with

* diffusion:       A = I + r K (Dirichlet), F = identity, parameter p = r;
* hyperdiffusion:  A = I + r D4 (hinged closure), F = identity, parameter p = r;
* Cahn-Hilliard:   A = I + dt gamma D4_N, F(x) = x + dt D2_N (x^3 - x),
                   parameter p = gamma (in grid units, dt fixed).

Loss L = sum((x_T - y)^2) / (N * M_total) over all systems.  The oracle stores
every state (no checkpointing) and runs the textbook reverse sweep:

    gbar_T = 2 (x_T - y) / (N M_total)
    for n = T-1 .. 0:
        mu      = A^{-T} gbar_{n+1}
        dL/dp  -= mu . (dA/dp) x_{n+1}
        gbar_n  = J_F(x_n)^T mu
    dL/dx_0 = gbar_0

with dA/dr = K (diffusion) or D4 (hyperdiffusion), dA/dgamma = dt D4_N, and J_F(x)^T mu = mu + dt (3 x^2 - 1) * (D2_N^T mu).
Systems never interact, so any subset of columns can be run on its own; the
parameter gradient is then the sum of the per-system contributions returned here.
"""
from __future__ import annotations

import numpy as np

from . import matrices, steppers

__all__ = ["Problem", "diffusion_problem", "hyperdiffusion_problem", "ch_problem", "forward", "loss", "adjoint"]


class Problem:
    """A rollout problem: shared matrix builder, explicit map F and its adjoint."""

    def __init__(self, kind, N, param, dt=None):
        self.kind, self.N, self.param, self.dt = kind, N, float(param), dt
        if kind == "diffusion":
            self.A = steppers.SharedTri(*matrices.diffusion_matrix(N, self.param))
            sub, dia, sup = matrices.d2_dirichlet(N)
            self.dA = (-sub, -dia, -sup)                     # K = -D2_D
        elif kind == "hyperdiffusion":
            self.A = steppers.SharedPenta(*matrices.hyperdiffusion_matrix(N, self.param, "hinged"))
            self.dA = matrices.square_tridiag(*matrices.d2_dirichlet(N))   # D4 (hinged)
        elif kind == "cahn_hilliard":
            self.A = steppers.SharedPenta(*matrices.ch_matrix(N, dt * self.param))
            self.dA = tuple(dt * v for v in matrices.square_tridiag(*matrices.d2_noflux(N)))
            self.d2n = matrices.d2_noflux(N)
        else:
            raise ValueError(kind)

    def F(self, x):
        if self.kind in ("diffusion", "hyperdiffusion"):
            return np.asarray(x, dtype=np.float64).copy()
        return steppers.ch_rhs(x, self.dt)

    def F_adjoint(self, x, mu):
        """J_F(x)^T mu."""
        if self.kind in ("diffusion", "hyperdiffusion"):
            return mu.copy()
        sub, dia, sup = self.d2n
        # transpose of a tridiagonal matrix: sub-diagonal of T^T is super of T shifted
        N = self.N
        tsub = np.zeros(N)
        tsup = np.zeros(N)
        tsub[1:] = sup[:-1]
        tsup[:-1] = sub[1:]
        return mu + self.dt * (3.0 * x * x - 1.0) * matrices.apply_tri(tsub, dia, tsup, mu)

    def apply_dA(self, x):
        if self.kind == "diffusion":
            return matrices.apply_tri(*self.dA, x)
        if self.kind == "hyperdiffusion":
            return matrices.apply_penta(*self.dA, x)
        return matrices.apply_penta(*self.dA, x)


def diffusion_problem(N, r):
    return Problem("diffusion", N, r)


def hyperdiffusion_problem(N, r):
    return Problem("hyperdiffusion", N, r)


def ch_problem(N, gamma, dt):
    return Problem("cahn_hilliard", N, gamma, dt)


def forward(prob: Problem, x0, steps):
    """All states x_0 .. x_T of the rollout (list of (N, M) arrays)."""
    xs = [np.asarray(x0, dtype=np.float64)]
    for _ in range(steps):
        xs.append(prob.A.solve(prob.F(xs[-1])))
    return xs


def loss(xT, y, M_total):
    """L = sum((x_T - y)^2) / (N * M_total)."""
    N = xT.shape[0]
    return float(np.sum((xT - y) ** 2) / (N * M_total))


def adjoint(prob: Problem, x0, y, steps, M_total=None):
    """Reverse sweep.  Returns (L, dL/dx0 of shape (N, M), per-system dL/dp of
    shape (M,)).  ``M_total`` is the batch size used in the loss normalisation
    (defaults to the number of columns given)."""
    x0 = np.asarray(x0, dtype=np.float64)
    M_total = x0.shape[1] if M_total is None else M_total
    xs = forward(prob, x0, steps)
    N = x0.shape[0]
    gbar = 2.0 * (xs[-1] - y) / (N * M_total)
    dp = np.zeros(x0.shape[1])
    for n in range(steps - 1, -1, -1):
        mu = prob.A.solve_adjoint(gbar)
        dp -= np.sum(mu * prob.apply_dA(xs[n + 1]), axis=0)
        gbar = prob.F_adjoint(xs[n], mu)
    return loss(xs[-1], y, M_total), gbar, dp
