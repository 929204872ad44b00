"""B-spline and quadrature primitives of the oracle (test infrastructure only).

* Open uniform knot vector on [0, 1] (Sec. 3.1): xi_1..xi_{p+1} = 0,
  xi_{m+1}..xi_{m+p+1} = 1, uniform spacing 1/(m-p) = h in between.
* Univariate B-splines by the Cox-de Boor recursion (de Boor, "A Practical Guide
  to Splines", Ch. IX), values and first derivatives, as dense collocation
  matrices (slow, obviously correct).
* Gauss-Legendre rule by the Golub-Welsch eigenvalue method (Golub & Welsch 1969).
* Greville abscissae gamma_k = (xi_{k+1} + ... + xi_{k+p}) / p.

Indices are 0-based in code; the paper's 1-based index k is code index k-1.
"""
import numpy as np


def open_uniform_knots(n_el, p):
    """Open uniform knot vector with n_el elements and degree p (Sec. 3.1)."""
    inner = np.arange(1, n_el, dtype=np.float64) / n_el
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def _last_nonempty_span(knots):
    """Index j of the last knot interval [knots[j], knots[j+1]) with positive length."""
    for j in range(len(knots) - 2, -1, -1):
        if knots[j] < knots[j + 1]:
            return j
    raise ValueError("degenerate knot vector")


def collocation(knots, deg, x, deriv=0):
    """Dense matrix B[r, k] = (d/dx)^deriv B_{k,deg}(x_r) for all basis functions.

    Cox-de Boor recursion carried out on the full knot vector; 0/0 terms are 0.
    The right end point of the knot vector belongs to the last non-empty span so
    that the basis is a partition of unity on the closed interval.
    deriv is 0 or 1.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = np.asarray(knots, dtype=np.float64)
    nk = len(t)
    last = _last_nonempty_span(t)
    # degree 0: indicator functions of the knot spans
    B = np.zeros((len(x), nk - 1))
    for j in range(nk - 1):
        inside = (t[j] <= x) & (x < t[j + 1])
        if j == last:
            inside |= x == t[j + 1]
        B[:, j] = inside.astype(np.float64)

    def raise_degree(B, r):
        # B holds the degree r-1 functions; returns the degree r functions
        nb = nk - 1 - r
        out = np.zeros((len(x), nb))
        for k in range(nb):
            d1 = t[k + r] - t[k]
            d2 = t[k + r + 1] - t[k + 1]
            if d1 > 0:
                out[:, k] += (x - t[k]) / d1 * B[:, k]
            if d2 > 0:
                out[:, k] += (t[k + r + 1] - x) / d2 * B[:, k + 1]
        return out

    if deriv == 0:
        for r in range(1, deg + 1):
            B = raise_degree(B, r)
        return B
    if deriv != 1:
        raise ValueError("deriv must be 0 or 1")
    if deg == 0:
        return np.zeros((len(x), nk - 1))
    for r in range(1, deg):
        B = raise_degree(B, r)
    # B'_{k,deg} = deg/(t_{k+deg}-t_k) B_{k,deg-1} - deg/(t_{k+deg+1}-t_{k+1}) B_{k+1,deg-1}
    nb = nk - 1 - deg
    D = np.zeros((len(x), nb))
    for k in range(nb):
        d1 = t[k + deg] - t[k]
        d2 = t[k + deg + 1] - t[k + 1]
        if d1 > 0:
            D[:, k] += deg / d1 * B[:, k]
        if d2 > 0:
            D[:, k] -= deg / d2 * B[:, k + 1]
    return D


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1] by Golub-Welsch.

    The Jacobi matrix of the Legendre three-term recurrence has zero diagonal and
    off-diagonal entries k / sqrt(4k^2 - 1); its eigenvalues are the nodes on
    [-1, 1] and the squared first components of the normalised eigenvectors,
    times the measure 2, are the weights.
    """
    k = np.arange(1, n, dtype=np.float64)
    off = k / np.sqrt(4.0 * k * k - 1.0)
    J = np.diag(off, 1) + np.diag(off, -1)
    nodes, vecs = np.linalg.eigh(J)
    weights = 2.0 * vecs[0, :] ** 2
    return 0.5 * (nodes + 1.0), 0.5 * weights


def greville(knots, p):
    """Greville abscissae gamma_k = mean(xi_{k+1}..xi_{k+p}) for every basis function."""
    t = np.asarray(knots)
    m = len(t) - p - 1
    if p == 0:
        return 0.5 * (t[:m] + t[1:m + 1])
    return np.array([t[k + 1:k + p + 1].mean() for k in range(m)])
