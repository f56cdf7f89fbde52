"""Oracle: the finite-difference operators and shared matrices of the workloads.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each operator is built the plain way: the second-difference matrix D2 is written
down row by row from its stencil, and every fourth-difference matrix is the
product D2 @ D2 of two such matrices, formed entry by entry over the three
non-zero terms of each row.  Shared matrices are ``I + coefficient * operator``.
Results are returned as diagonals (offsets -2..+2 for pentadiagonal, -1..+1 for
tridiagonal) in the naming of sections 3.1 and 4.1.

Boundary readings (the paper's own benchmarks are periodic; the workloads here
use the non-periodic closures below):

* ``dirichlet``  -- unknowns are the N interior points of a grid whose two end
  values are held at 0; the stencil is truncated at the first and last rows.
  D2_D = tridiag(1, -2, 1).
* ``hinged``     -- D4 = D2_D @ D2_D (odd reflection of the ghost points, i.e.
  C = C'' = 0 at both ends); corner entries 5, next rows (-4, 6, -4, 1).
* ``truncated``  -- D4 is the plain Toeplitz (1, -4, 6, -4, 1) cut at the edges
  (corner entries 6).
* ``periodic``   -- the paper's own closure (sections 3.2 and 3.3): row 0's left
  neighbour is row N-1 and row N-1's right neighbour is row 0; the two wrapped
  coefficients sit in sub[0] and sup[N-1] (the corners of section 3.3).
* ``noflux``     -- cell-centred Neumann closure: D2_N has rows (-1, 1),
  (1, -2, 1), ..., (1, -1) (even reflection of the ghost cell), and
  D4_N = D2_N @ D2_N.  Every column of D2_N sums to zero, so sum(C) is
  conserved by both operators.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "d2_dirichlet", "d2_noflux", "d2_periodic", "d4_periodic", "square_tridiag", "d4_truncated",
    "diffusion_matrix", "diffusion_matrix_periodic", "hyperdiffusion_matrix", "ch_matrix",
    "ch_matrix_periodic", "apply_tri", "apply_tri_periodic", "apply_penta",
    "apply_penta_periodic", "bands_to_dense",
]


def d2_dirichlet(N):
    """Second difference with zero Dirichlet ghosts: rows (1, -2, 1) truncated.
    Returns (sub, diag, super)."""
    sub = np.ones(N)
    sup = np.ones(N)
    dia = -2.0 * np.ones(N)
    sub[0] = 0.0
    sup[N - 1] = 0.0
    return sub, dia, sup


def d2_noflux(N):
    """Cell-centred Neumann second difference D2_N: rows (-1, 1), (1, -2, 1), ...,
    (1, -1).  For N = 1 the operator is the 1x1 zero matrix."""
    sub = np.ones(N)
    sup = np.ones(N)
    dia = -2.0 * np.ones(N)
    sub[0] = 0.0
    sup[N - 1] = 0.0
    dia[0] += 1.0       # ghost C_{-1} = C_0
    dia[N - 1] += 1.0   # ghost C_N = C_{N-1}
    return sub, dia, sup


def square_tridiag(sub, dia, sup):
    """Product T @ T of a tridiagonal matrix with itself, as five diagonals
    (a, b, c, d, e) with offsets (-2, -1, 0, +1, +2).

    (T T)[i, j] = sum over k in {i-1, i, i+1} of T[i, k] T[k, j].
    """
    N = len(dia)

    def T(i, k):
        if k < 0 or k >= N or i < 0 or i >= N:
            return 0.0
        if k == i:
            return dia[i]
        if k == i - 1:
            return sub[i]
        if k == i + 1:
            return sup[i]
        return 0.0

    out = {off: np.zeros(N) for off in (-2, -1, 0, 1, 2)}
    for i in range(N):
        for off in (-2, -1, 0, 1, 2):
            j = i + off
            if j < 0 or j >= N:
                continue
            out[off][i] = sum(T(i, k) * T(k, j) for k in (i - 1, i, i + 1))
    return out[-2], out[-1], out[0], out[1], out[2]


def d4_truncated(N):
    """Toeplitz fourth difference (1, -4, 6, -4, 1) truncated at the edges."""
    a = np.ones(N)
    b = -4.0 * np.ones(N)
    c = 6.0 * np.ones(N)
    d = -4.0 * np.ones(N)
    e = np.ones(N)
    a[:2] = 0.0
    b[:1] = 0.0
    d[N - 1:] = 0.0
    e[N - 2:] = 0.0
    return a, b, c, d, e


def d2_periodic(N):
    """Periodic second difference: rows (1, -2, 1) everywhere, wrapping around;
    sub[0] and sup[N-1] are the corner entries (section 3.3's matrix).  N >= 3."""
    if N < 3:
        raise ValueError("the periodic operator needs N >= 3")
    return np.ones(N), -2.0 * np.ones(N), np.ones(N)


def diffusion_matrix_periodic(N, r):
    """A = I + r K with K = -D2_P: section 3.2's left-hand side with a = c = -r,
    b = 1 + 2r on every row, the corners included.  Returns (a, b, c)."""
    sub, dia, sup = d2_periodic(N)
    return -r * sub, 1.0 - r * dia, -r * sup


def diffusion_matrix(N, r):
    """A = I + r K with K = -D2_D = tridiag(-1, 2, -1): the backward-Euler matrix of
    the diffusion equation (section 3.2's coefficients a = c = -sigma,
    b = 1 + 2 sigma with sigma -> r), Dirichlet rows truncated.
    Returns (a, b, c)."""
    sub, dia, sup = d2_dirichlet(N)
    return -r * sub, 1.0 - r * dia, -r * sup


def hyperdiffusion_matrix(N, r, closure="hinged"):
    """A = I + r D4 (section 4.2's left-hand side, interior row
    (r, -4r, 1 + 6r, -4r, r)), with D4 = D2_D @ D2_D (``hinged``) or the truncated
    Toeplitz stencil (``truncated``).  Returns (a, b, c, d, e)."""
    if closure == "hinged":
        a, b, c, d, e = square_tridiag(*d2_dirichlet(N))
    elif closure == "truncated":
        a, b, c, d, e = d4_truncated(N)
    else:
        raise ValueError(closure)
    return r * a, r * b, 1.0 + r * c, r * d, r * e


def ch_matrix(N, sigma):
    """A = I + sigma D4_N, the implicit matrix of the Cahn-Hilliard scheme of
    section 5.1 (C^{n+1} + dt gamma D4 C^{n+1} = ...), with sigma = dt * gamma in
    grid units and the no-flux closure D4_N = D2_N @ D2_N.  Returns (a, b, c, d, e)."""
    a, b, c, d, e = square_tridiag(*d2_noflux(N))
    return sigma * a, sigma * b, 1.0 + sigma * c, sigma * d, sigma * e


def d4_periodic(N):
    """Periodic fourth difference D2_P @ D2_P: rows (1, -4, 6, -4, 1) everywhere,
    wrapping around (the operator of section 5.1 with periodic ends).  N >= 5.
    Formed as the product of two periodic second differences, entry by entry."""
    if N < 5:
        raise ValueError("the periodic fourth difference needs N >= 5")
    D2 = np.zeros((N, N))
    for i in range(N):
        D2[i, (i - 1) % N] += 1.0
        D2[i, i] += -2.0
        D2[i, (i + 1) % N] += 1.0
    D4 = D2 @ D2
    return tuple(np.array([D4[i, (i + off) % N] for i in range(N)]) for off in (-2, -1, 0, 1, 2))


def ch_matrix_periodic(N, sigma):
    """A = I + sigma D4_P: section 5.1's implicit matrix with periodic ends (the
    paper's own choice, a = e = sigma, b = d = -4 sigma, c = 1 + 6 sigma on every
    row; the wrapped entries sit in a[0], a[1], b[0], d[N-1], e[N-2], e[N-1])."""
    a, b, c, d, e = d4_periodic(N)
    return sigma * a, sigma * b, 1.0 + sigma * c, sigma * d, sigma * e


def apply_tri(sub, dia, sup, x):
    """y = T x for a tridiagonal T given by diagonals, x of shape (N, M)."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    y = dia[:, None] * x
    if N > 1:
        y[1:] += sub[1:, None] * x[:-1]
        y[:-1] += sup[:-1, None] * x[1:]
    return y


def apply_tri_periodic(sub, dia, sup, x):
    """y = T x for a periodic tridiagonal T (corners sub[0] at (0, N-1) and
    sup[N-1] at (N-1, 0)), x of shape (N, M)."""
    x = np.asarray(x, dtype=np.float64)
    y = apply_tri(sub, dia, sup, x)
    N = x.shape[0]
    y[0] += sub[0] * x[N - 1]
    y[N - 1] += sup[N - 1] * x[0]
    return y


def apply_penta(a, b, c, d, e, x):
    """y = P x for a pentadiagonal P given by diagonals, x of shape (N, M)."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    y = c[:, None] * x
    if N > 1:
        y[1:] += b[1:, None] * x[:-1]
        y[:-1] += d[:-1, None] * x[1:]
    if N > 2:
        y[2:] += a[2:, None] * x[:-2]
        y[:-2] += e[:-2, None] * x[2:]
    return y


def apply_penta_periodic(a, b, c, d, e, x):
    """y = P x for a cyclic pentadiagonal P (indices modulo N), x of shape (N, M)."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    y = np.zeros_like(x)
    for off, v in ((-2, a), (-1, b), (0, c), (1, d), (2, e)):
        y += np.asarray(v)[:, None] * np.roll(x, -off, axis=0)
    return y


def bands_to_dense(*diags):
    """Dense matrix from 3 (offsets -1..1) or 5 (offsets -2..2) diagonals."""
    N = len(diags[len(diags) // 2])
    offs = range(-(len(diags) // 2), len(diags) // 2 + 1)
    A = np.zeros((N, N))
    for off, v in zip(offs, diags):
        for i in range(N):
            j = i + off
            if 0 <= j < N:
                A[i, j] = v[i]
    return A
