"""Oracle: shared-LHS tridiagonal and pentadiagonal factor / solve / adjoint solve.

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 NumPy.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may use it; the
product library never imports it.

Every function works on a batch of right-hand sides stored interleaved, i.e. as a
NumPy array of shape ``(N, M)`` whose column ``m`` is system ``m`` (element
``(i, m)`` at ``i*M + m`` in memory, the layout of the paper's Fig. 2).  Rows are
processed one at a time in the order the recurrences state; each row operation is
applied to all systems at once, which changes nothing in the per-system arithmetic
(the systems never interact).

Indices are 0-based here; the paper's are 1-based (paper row i = our row i-1).
The oracle divides by pivots, as the equations are printed; it never stores
reciprocals.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "tri_factor", "tri_solve", "tri_solve_adjoint",
    "tri_periodic_factor", "tri_periodic_solve", "tri_periodic_solve_adjoint", "tri_periodic_dense",
    "penta_factor", "penta_solve", "penta_solve_adjoint",
    "penta_periodic_factor", "penta_periodic_solve", "penta_periodic_solve_adjoint", "penta_periodic_dense",
    "tri_dense", "penta_dense",
]


# ----------------------------------------------------------------------------
# Tridiagonal (section 3.1, "Tridiagonal Inversion Algorithm"; Algorithms 1-2)
# ----------------------------------------------------------------------------

def tri_factor(a, b, c):
    """Pre-factorisation of section 3.1 (Algorithm 1), done once for the shared A.

    A has sub-diagonal ``a`` (a[0] unused), diagonal ``b`` and super-diagonal ``c``
    (c[N-1] unused).  Returns ``(bh, ch)``:
        ch_0 = c_0 / b_0,   bh_0 = b_0
        bh_i = b_i - a_i * ch_{i-1},   ch_i = c_i / bh_i      (i = 1 .. N-1)
    ch[N-1] is not part of the factorisation and is returned as 0.
    Raises ZeroDivisionError on a zero pivot (no pivoting, as in the paper).
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    N = b.shape[0]
    bh = np.zeros(N)
    ch = np.zeros(N)
    for i in range(N):
        bh[i] = b[i] if i == 0 else b[i] - a[i] * ch[i - 1]
        if bh[i] == 0.0 or not np.isfinite(bh[i]):
            raise ZeroDivisionError(f"zero or non-finite pivot at row {i}")
        if i < N - 1:
            ch[i] = c[i] / bh[i]
    return bh, ch


def tri_solve(a, bh, ch, d):
    """Forward and backward sweeps of section 3.1 (Algorithm 2) for every column
    of ``d`` (shape (N, M)), with the shared factors from :func:`tri_factor`.

        forward:  dh_0 = d_0 / bh_0,  dh_i = (d_i - a_i dh_{i-1}) / bh_i
        backward: x_{N-1} = dh_{N-1}, x_i = dh_i - ch_i x_{i+1}

    The backward recurrence is the one of Algorithm 2 (the printed equation
    "x_i = dh_i - a_i ch_i" in section 3.1 drops x_{i+1}; Algorithm 2 and the
    standard Thomas algorithm multiply ch_i by x_{i+1}).
    """
    d = np.asarray(d, dtype=np.float64)
    N = d.shape[0]
    dh = np.empty_like(d)
    dh[0] = d[0] / bh[0]
    for i in range(1, N):
        dh[i] = (d[i] - a[i] * dh[i - 1]) / bh[i]
    x = np.empty_like(d)
    x[N - 1] = dh[N - 1]
    for i in range(N - 2, -1, -1):
        x[i] = dh[i] - ch[i] * x[i + 1]
    return x


def tri_solve_adjoint(a, bh, ch, g):
    """Solve A^T y = g with the same shared factors (no counterpart in the paper;
    it is the transpose of the factorisation A = L U of section 3.1).

    L is lower bidiagonal (diagonal bh, sub-diagonal a), U is unit upper
    bidiagonal (super-diagonal ch), so A^T = U^T L^T:
        U^T w = g:  w_0 = g_0,  w_i = g_i - ch_{i-1} w_{i-1}
        L^T y = w:  y_{N-1} = w_{N-1} / bh_{N-1},  y_i = (w_i - a_{i+1} y_{i+1}) / bh_i
    """
    g = np.asarray(g, dtype=np.float64)
    N = g.shape[0]
    w = np.empty_like(g)
    w[0] = g[0]
    for i in range(1, N):
        w[i] = g[i] - ch[i - 1] * w[i - 1]
    y = np.empty_like(g)
    y[N - 1] = w[N - 1] / bh[N - 1]
    for i in range(N - 2, -1, -1):
        y[i] = (w[i] - a[i + 1] * y[i + 1]) / bh[i]
    return y


def tri_dense(a, b, c):
    """Dense N x N matrix with the given three diagonals (for checks only)."""
    N = len(b)
    A = np.diag(np.asarray(b, dtype=np.float64))
    for i in range(1, N):
        A[i, i - 1] = a[i]
        A[i - 1, i] = c[i - 1]
    return A



# ----------------------------------------------------------------------------
# Periodic tridiagonal (section 3.3, "Periodic Tridiagonal Matrix")
# ----------------------------------------------------------------------------

def tri_periodic_dense(a, b, c):
    """Dense periodic tridiagonal matrix: the three diagonals of :func:`tri_dense`
    plus the two corner entries of section 3.3, A[0, N-1] = a_0 (row 0's
    sub-diagonal coefficient wraps around) and A[N-1, 0] = c_{N-1} (row N-1's
    super-diagonal coefficient wraps around).  N >= 3."""
    N = len(b)
    if N < 3:
        raise ValueError("a periodic tridiagonal matrix needs N >= 3")
    A = tri_dense(a, b, c)
    A[0, N - 1] = a[0]
    A[N - 1, 0] = c[N - 1]
    return A


def tri_periodic_factor(a, b, c):
    """Section 3.3: write A = A' + u v^T with

        u = (-b_0, 0, ..., 0, c_{N-1})^T,   v = (1, 0, ..., 0, -a_0 / b_0)^T,

    so that A' is the plain tridiagonal matrix with b'_0 = 2 b_0 and
    b'_{N-1} = b_{N-1} + a_0 c_{N-1} / b_0 and no corner entries (the section's
    constant-coefficient u, v and A' with the coefficients taken per row).  A' is
    factored by section 3.1 once, and z = A'^{-1} u is solved once, as the section
    says ("need only be performed once").  Returns a dict with the factors of A',
    u, v and z."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    N = b.shape[0]
    if N < 3:
        raise ValueError("a periodic tridiagonal matrix needs N >= 3")
    u = np.zeros(N)
    v = np.zeros(N)
    u[0], u[N - 1] = -b[0], c[N - 1]
    v[0], v[N - 1] = 1.0, -a[0] / b[0]
    ap, bp, cp = a.copy(), b.copy(), c.copy()
    ap[0] = 0.0
    cp[N - 1] = 0.0
    bp[0] = b[0] - u[0] * v[0]
    bp[N - 1] = b[N - 1] - u[N - 1] * v[N - 1]
    bh, ch = tri_factor(ap, bp, cp)
    z = tri_solve(ap, bh, ch, u[:, None])[:, 0]
    return {"a": ap, "bh": bh, "ch": ch, "u": u, "v": v, "z": z}


def tri_periodic_solve(fac, d):
    """Solve A x = d for every column of ``d`` (section 3.3):
        A' y = d,   x = y - ((v . y) / (1 + v . z)) z."""
    y = tri_solve(fac["a"], fac["bh"], fac["ch"], d)
    vy = fac["v"] @ y
    return y - np.outer(fac["z"], vy / (1.0 + fac["v"] @ fac["z"]))


def tri_periodic_solve_adjoint(fac, g):
    """Solve A^T y = g (no counterpart in the paper): A^T = A'^T + v u^T, so with
    the same factors of A', w = A'^{-T} g, z' = A'^{-T} v and
        y = w - ((u . w) / (1 + u . z')) z'."""
    w = tri_solve_adjoint(fac["a"], fac["bh"], fac["ch"], g)
    zt = tri_solve_adjoint(fac["a"], fac["bh"], fac["ch"], fac["v"][:, None])[:, 0]
    uw = fac["u"] @ w
    return w - np.outer(zt, uw / (1.0 + fac["u"] @ zt))

# ----------------------------------------------------------------------------
# Pentadiagonal (section 4.1, "Pentadiagonal Inversion Algorithm"; Algorithms 3-4)
# ----------------------------------------------------------------------------

def penta_factor(a, b, c, d, e):
    """Factorisation A = L R of section 4.1 (Algorithm 3), once for the shared A.

    A has diagonals ``a`` (offset -2), ``b`` (-1), ``c`` (0), ``d`` (+1), ``e`` (+2);
    entries outside the matrix are ignored.  L is lower triangular with diagonal
    alpha, first sub-diagonal beta and second sub-diagonal eps; R is unit upper
    triangular with super-diagonals gamma and delta.  Section 4.1 lists the
    recurrences with the first two and last two rows written out separately; they
    are the single recurrence below with every out-of-range coefficient equal to 0:

        beta_i  = b_i - a_i gamma_{i-2}
        alpha_i = c_i - a_i delta_{i-2} - beta_i gamma_{i-1}
        gamma_i = (d_i - beta_i delta_{i-1}) / alpha_i
        delta_i = e_i / alpha_i
        eps_i   = a_i

    (Algorithm 3 as printed subtracts a_i c_{i-2} in the alpha update, misses a
    parenthesis in the gamma update and uses d_N in the last beta; the section 4.1
    equations, followed here, are a_i delta_{i-2}, (d_i - beta_i delta_{i-1})/alpha_i
    and a_N gamma_{N-2}.)  Returns ``(eps, beta, alpha, gamma, delta)``.
    """
    a, b, c, d, e = (np.asarray(v, dtype=np.float64) for v in (a, b, c, d, e))
    N = c.shape[0]
    alpha = np.zeros(N)
    beta = np.zeros(N)
    gamma = np.zeros(N)
    delta = np.zeros(N)
    eps = np.zeros(N)

    def at(v, j):          # coefficient j of a factor vector; 0 outside the matrix
        return v[j] if 0 <= j < N else 0.0

    def coef(v, i, lo, hi):  # matrix entry of diagonal v on row i, present only if lo <= i <= hi
        return v[i] if lo <= i <= hi else 0.0

    for i in range(N):
        ai = coef(a, i, 2, N - 1)
        bi = coef(b, i, 1, N - 1)
        di = coef(d, i, 0, N - 2)
        ei = coef(e, i, 0, N - 3)
        beta[i] = bi - ai * at(gamma, i - 2)
        alpha[i] = c[i] - ai * at(delta, i - 2) - beta[i] * at(gamma, i - 1)
        if alpha[i] == 0.0 or not np.isfinite(alpha[i]):
            raise ZeroDivisionError(f"zero or non-finite pivot at row {i}")
        gamma[i] = (di - beta[i] * at(delta, i - 1)) / alpha[i]
        delta[i] = ei / alpha[i]
        eps[i] = ai
    return eps, beta, alpha, gamma, delta


def penta_solve(eps, beta, alpha, gamma, delta, f):
    """Solve A x = f with the factors of :func:`penta_factor` (section 4.1,
    Algorithm 4), every column of ``f`` (shape (N, M)) independently.

        L g = f:  g_i = (f_i - eps_i g_{i-2} - beta_i g_{i-1}) / alpha_i
        R x = g:  x_i = g_i - gamma_i x_{i+1} - delta_i x_{i+2}
    with terms whose index falls outside 0..N-1 omitted.  (Algorithm 4 prints
    "d_i d_{rowID+M}" in the backward loop; section 4.1 has gamma_i x_{i+1}.)
    """
    f = np.asarray(f, dtype=np.float64)
    N = f.shape[0]
    g = np.empty_like(f)
    for i in range(N):
        s = f[i].copy()
        if i >= 2:
            s -= eps[i] * g[i - 2]
        if i >= 1:
            s -= beta[i] * g[i - 1]
        g[i] = s / alpha[i]
    x = np.empty_like(f)
    for i in range(N - 1, -1, -1):
        s = g[i].copy()
        if i + 1 < N:
            s -= gamma[i] * x[i + 1]
        if i + 2 < N:
            s -= delta[i] * x[i + 2]
        x[i] = s
    return x


def penta_solve_adjoint(eps, beta, alpha, gamma, delta, g):
    """Solve A^T y = g with the same factors (no counterpart in the paper; it is the
    transpose of A = L R from section 4.1).  A^T = R^T L^T:

        R^T w = g:  w_i = g_i - gamma_{i-1} w_{i-1} - delta_{i-2} w_{i-2}
        L^T y = w:  y_i = (w_i - beta_{i+1} y_{i+1} - eps_{i+2} y_{i+2}) / alpha_i
    """
    g = np.asarray(g, dtype=np.float64)
    N = g.shape[0]
    w = np.empty_like(g)
    for i in range(N):
        s = g[i].copy()
        if i >= 1:
            s -= gamma[i - 1] * w[i - 1]
        if i >= 2:
            s -= delta[i - 2] * w[i - 2]
        w[i] = s
    y = np.empty_like(g)
    for i in range(N - 1, -1, -1):
        s = w[i].copy()
        if i + 1 < N:
            s -= beta[i + 1] * y[i + 1]
        if i + 2 < N:
            s -= eps[i + 2] * y[i + 2]
        y[i] = s / alpha[i]
    return y


def penta_dense(a, b, c, d, e):
    """Dense N x N matrix with the given five diagonals (for checks only)."""
    N = len(c)
    A = np.diag(np.asarray(c, dtype=np.float64))
    for i in range(N):
        if i >= 2:
            A[i, i - 2] = a[i]
        if i >= 1:
            A[i, i - 1] = b[i]
        if i + 1 < N:
            A[i, i + 1] = d[i]
        if i + 2 < N:
            A[i, i + 2] = e[i]
    return A


# ----------------------------------------------------------------------------
# Cyclic pentadiagonal (the periodic matrix of section 5.1's scheme; the paper
# refers to the literature for its solution)
# ----------------------------------------------------------------------------

def penta_periodic_dense(a, b, c, d, e):
    """Dense cyclic pentadiagonal matrix: row i is a_i x_{i-2} + b_i x_{i-1} + c_i x_i
    + d_i x_{i+1} + e_i x_{i+2} with the indices taken modulo N (N >= 5), so the
    corner entries are A[0, N-2] = a_0, A[0, N-1] = b_0, A[1, N-1] = a_1,
    A[N-2, 0] = e_{N-2}, A[N-1, 0] = d_{N-1}, A[N-1, 1] = e_{N-1}."""
    a, b, c, d, e = (np.asarray(v, dtype=np.float64) for v in (a, b, c, d, e))
    N = c.shape[0]
    if N < 5:
        raise ValueError("a cyclic pentadiagonal matrix needs N >= 5")
    A = np.zeros((N, N))
    for i in range(N):
        for off, v in ((-2, a), (-1, b), (0, c), (1, d), (2, e)):
            A[i, (i + off) % N] += v[i]
    return A


def penta_periodic_factor(a, b, c, d, e):
    """Split A = A' + U V^T with a rank-2 correction, the 2 x 2 block form of
    section 3.3's construction (which is its 1 x 1 case).  With TR the top-right
    2 x 2 corner block (rows 0,1; columns N-2,N-1), BL the bottom-left one (rows
    N-2,N-1; columns 0,1) and X = -(the top-left 2 x 2 block of A):

        U = [X; 0; BL]  (rows 0,1 | middle | N-2,N-1),   V = [I; 0; (X^{-1} TR)^T],

    so U V^T puts X X^0 = X in the top-left block, TR and BL in the corners and
    BL X^{-1} TR in the bottom-right block.  A' = A - U V^T is pentadiagonal (no
    corners; top-left block 2 A_tl, bottom-right block A_br - BL X^{-1} TR), factored
    by section 4.1; Z = A'^{-1} U and the 2 x 2 matrix S = I + V^T Z are formed once.
    Returns a dict with the factors of A' and U, V, Z, S."""
    a, b, c, d, e = (np.asarray(v, dtype=np.float64).copy() for v in (a, b, c, d, e))
    N = c.shape[0]
    if N < 5:
        raise ValueError("a cyclic pentadiagonal matrix needs N >= 5")
    A = penta_periodic_dense(a, b, c, d, e)
    TL = A[0:2, 0:2]
    TR = A[0:2, N - 2:N]
    BL = A[N - 2:N, 0:2]
    X = -TL
    W = np.linalg.solve(X, TR)  # X^{-1} TR
    U = np.zeros((N, 2))
    V = np.zeros((N, 2))
    U[0:2, :] = X
    U[N - 2:N, :] = BL
    V[0:2, :] = np.eye(2)
    V[N - 2:N, :] = W.T
    Ap = A - U @ V.T
    # A' is banded: read its five diagonals back (the corners cancel exactly)
    ap, bp, cp, dp, ep = (np.zeros(N) for _ in range(5))
    for i in range(N):
        if i >= 2:
            ap[i] = Ap[i, i - 2]
        if i >= 1:
            bp[i] = Ap[i, i - 1]
        cp[i] = Ap[i, i]
        if i + 1 < N:
            dp[i] = Ap[i, i + 1]
        if i + 2 < N:
            ep[i] = Ap[i, i + 2]
    fac = penta_factor(ap, bp, cp, dp, ep)
    Z = penta_solve(*fac, U)
    S = np.eye(2) + V.T @ Z
    return {"factors": fac, "U": U, "V": V, "Z": Z, "S": S,
            "diags_prime": (ap, bp, cp, dp, ep)}


def penta_periodic_solve(f, rhs):
    """Solve A x = rhs (Sherman-Morrison-Woodbury): A' y = rhs,
    x = y - Z S^{-1} (V^T y)."""
    y = penta_solve(*f["factors"], rhs)
    return y - f["Z"] @ np.linalg.solve(f["S"], f["V"].T @ y)


def penta_periodic_solve_adjoint(f, g):
    """Solve A^T y = g (no counterpart in the paper): A^T = A'^T + V U^T, so with
    w = A'^{-T} g, Z' = A'^{-T} V and S' = I + U^T Z':  y = w - Z' S'^{-1} (U^T w)."""
    w = penta_solve_adjoint(*f["factors"], g)
    Zt = penta_solve_adjoint(*f["factors"], f["V"])
    St = np.eye(2) + f["U"].T @ Zt
    return w - Zt @ np.linalg.solve(St, f["U"].T @ w)
