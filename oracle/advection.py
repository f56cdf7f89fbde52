"""Oracle: the Hamilton-Jacobi WENO derivative used for the advection term of the
travelling-wave forced Cahn-Hilliard scheme (section 6.1, the scheme with the
v dC/d(eta) term on the right-hand side; the paper takes the derivative from the
Hamilton-Jacobi WENO scheme of Osher and Fedkiw's book, i.e. the fifth-order
scheme of Jiang and Peng).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Arrays are interleaved ``(N, M)`` on a periodic grid with unit spacing (grid units:
divide by the physical spacing for d/dx).  Written from the published algorithm:

* one-sided differences D_j = phi_{j+1} - phi_j;
* for the left-biased derivative at row i the five differences
  q1..q5 = D_{i-3}, D_{i-2}, D_{i-1}, D_i, D_{i+1} (the right-biased one takes
  D_{i+2}, D_{i+1}, D_i, D_{i-1}, D_{i-2}, the same formulas mirrored);
* three third-order candidates
  p1 = q1/3 - 7 q2/6 + 11 q3/6,  p2 = -q2/6 + 5 q3/6 + q4/3,  p3 = q3/3 + 5 q4/6 - q5/6;
* smoothness indicators
  S1 = 13/12 (q1 - 2 q2 + q3)^2 + 1/4 (q1 - 4 q2 + 3 q3)^2,
  S2 = 13/12 (q2 - 2 q3 + q4)^2 + 1/4 (q2 - q4)^2,
  S3 = 13/12 (q3 - 2 q4 + q5)^2 + 1/4 (3 q3 - 4 q4 + q5)^2;
* eps = 1e-6 max(q_k^2) + 1e-99, a_k = (0.1, 0.6, 0.3)_k / (S_k + eps)^2,
  weights w_k = a_k / (a1 + a2 + a3), derivative = w1 p1 + w2 p2 + w3 p3.
"""
from __future__ import annotations

import numpy as np

__all__ = ["weno5_derivative", "linear_upwind5_derivative"]


def _candidates_and_weights(q1, q2, q3, q4, q5):
    p1 = q1 / 3.0 - 7.0 * q2 / 6.0 + 11.0 * q3 / 6.0
    p2 = -q2 / 6.0 + 5.0 * q3 / 6.0 + q4 / 3.0
    p3 = q3 / 3.0 + 5.0 * q4 / 6.0 - q5 / 6.0
    s1 = 13.0 / 12.0 * (q1 - 2.0 * q2 + q3) ** 2 + 0.25 * (q1 - 4.0 * q2 + 3.0 * q3) ** 2
    s2 = 13.0 / 12.0 * (q2 - 2.0 * q3 + q4) ** 2 + 0.25 * (q2 - q4) ** 2
    s3 = 13.0 / 12.0 * (q3 - 2.0 * q4 + q5) ** 2 + 0.25 * (3.0 * q3 - 4.0 * q4 + q5) ** 2
    eps = 1e-6 * np.maximum.reduce([q1 * q1, q2 * q2, q3 * q3, q4 * q4, q5 * q5]) + 1e-99
    a1 = 0.1 / (s1 + eps) ** 2
    a2 = 0.6 / (s2 + eps) ** 2
    a3 = 0.3 / (s3 + eps) ** 2
    return (p1, p2, p3), (a1, a2, a3)


def _differences(phi, side):
    """(q1, ..., q5) at every row for the left- (side = -1) or right-biased (+1)
    derivative, periodic in the row index."""
    phi = np.asarray(phi, dtype=np.float64)
    D = np.roll(phi, -1, axis=0) - phi              # D_j = phi_{j+1} - phi_j
    sh = lambda k: np.roll(D, -k, axis=0)            # row i holds D_{i+k}
    if side < 0:
        return sh(-3), sh(-2), sh(-1), sh(0), sh(1)
    return sh(2), sh(1), sh(0), sh(-1), sh(-2)


def weno5_derivative(phi, side):
    """Fifth-order Hamilton-Jacobi WENO approximation of d(phi)/di on a periodic
    grid of unit spacing, left-biased (side = -1, the stencil reaches rows i-3..i+2)
    or right-biased (side = +1, rows i-2..i+3)."""
    (p1, p2, p3), (a1, a2, a3) = _candidates_and_weights(*_differences(phi, side))
    s = a1 + a2 + a3
    return (a1 / s) * p1 + (a2 / s) * p2 + (a3 / s) * p3


def linear_upwind5_derivative(phi, side):
    """The same candidates combined with the ideal weights (0.1, 0.6, 0.3): the
    linear fifth-order upwind-biased difference that WENO reduces to where the data
    is smooth."""
    (p1, p2, p3), _ = _candidates_and_weights(*_differences(phi, side))
    return 0.1 * p1 + 0.6 * p2 + 0.3 * p3
