"""Pins of oracle parts whose only earlier check was indirect.

* interp_knots (Sec. 3.3: quasi-uniform knots taken from the samples; Sec. 5.1:
  MATLAB spapi, whose default knot vector is order q+1 with (q+1)-fold end knots and
  de Boor averages of q consecutive abscissae inside): expected vectors written out
  by hand from that definition, not recomputed by a formula.
* CubeSinePerturbed (the 3-D map of the cube workloads): the Jacobian itself, through
  stiffness and mass entries computed by an independent quadrature with a sympy
  Jacobian and scipy B-splines.
* SinCosCoef and the Ricker wavelet: values at points where the formulas are known
  in closed form.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.assembly import Space, true_rows
from oracle.bspline import collocation, open_uniform_knots
from oracle.geometry import ConstCoef, CubeSinePerturbed, SinCosCoef
from oracle.surrogate import cardinal_point, interp_knots, sample_indices
from oracle.wave import ricker

# de Boor averages of q consecutive samples on the abscissae 0, 1, ..., 6:
# odd q gives sample points, even q midpoints (hand values)
UNIFORM7 = {
    1: [0, 0, 1, 2, 3, 4, 5, 6, 6],
    2: [0, 0, 0, 1.5, 2.5, 3.5, 4.5, 6, 6, 6],
    3: [0, 0, 0, 0, 2, 3, 4, 6, 6, 6, 6],
}


@pytest.mark.parametrize("q", [1, 2, 3])
def test_interp_knots_uniform_samples_hand_values(q):
    xs = np.arange(7, dtype=float)
    assert np.array_equal(interp_knots(xs, q), np.array(UNIFORM7[q], dtype=float))


def test_interp_knots_uniform_samples_scale_and_shift():
    # the knot rule commutes with affine maps of the abscissae
    xs = 0.25 + 0.5 * np.arange(7, dtype=float)
    assert np.allclose(interp_knots(xs, 2), 0.25 + 0.5 * np.array(UNIFORM7[2]), rtol=0, atol=1e-15)


def test_interp_knots_config1_sample_set():
    """annulus64_p2 (p = 2, n_el = 64, M = 4): the sampled interior offsets are
    0, 4, 8, 11, 15, 19, 23, 27, 30, 34, 38, 42, 46, 49, 53, 57 (Sec. 5.1 rule, pinned
    elsewhere); q = 2 averages consecutive pairs after the first sample.  The
    abscissae are the cardinal points x~ = (k - 3/2) h of the 1-based indices
    k = offset + 5, i.e. (offset + 3.5) / 64."""
    off = np.array([0, 4, 8, 11, 15, 19, 23, 27, 30, 34, 38, 42, 46, 49, 53, 57])
    samp = sample_indices(66, 2, 4)
    assert np.array_equal(samp - 4, off)
    hand = [0, 0, 0, 6, 9.5, 13, 17, 21, 25, 28.5, 32, 36, 40, 44, 47.5, 51, 57, 57, 57]
    knots = interp_knots(cardinal_point(samp, 2, 1.0 / 64), 2)
    assert np.allclose(knots, (np.array(hand) + 3.5) / 64, rtol=0, atol=1e-15)


@pytest.mark.parametrize("m,p,M,q", [(66, 2, 4, 2), (515, 3, 8, 3), (98, 2, 6, 2), (40, 3, 5, 1), (70, 2, 3, 3)])
def test_interp_knots_schoenberg_whitney(m, p, M, q):
    """t_j < x_j < t_{j+q+1} for every interior abscissa (the first / last abscissa sit
    on the (q+1)-fold end knots): B_j(x_j) > 0 and the collocation matrix is
    invertible (Schoenberg-Whitney)."""
    xs = cardinal_point(sample_indices(m, p, M), p, 1.0 / (m - p))
    t = interp_knots(xs, q)
    n = len(xs)
    assert len(t) == n + q + 1
    for j in range(1, n - 1):
        assert t[j] < xs[j] < t[j + q + 1]
    assert t[0] == xs[0] == t[q] and t[n] == xs[-1] == t[n + q]
    A = collocation(t, q, xs)
    assert np.all(np.diag(A) > 0)
    assert np.linalg.cond(A) < 1e3


def _gauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def test_perturbed_cube_entries_vs_independent_quadrature():
    """K and M entries of the sine-perturbed cube (eps 0.1) on a tiny mesh against a
    tensor Gauss rule written here (12 points per element and direction) with the
    Jacobian of x_a = s_a + eps sin(pi s) sin(pi t) sin(pi u) taken by sympy and the
    basis from scipy.  A transposed or wrongly differentiated J keeps det J (so |Omega|)
    but changes G = det J J^-1 J^-T and fails here."""
    import sympy as sy
    p, n_el, eps = 2, 10, 0.1
    sp = Space(3, p, n_el, CubeSinePerturbed(eps), ConstCoef(), quad_pts=8)
    s = sy.symbols("s0 s1 s2")
    g = sy.sin(sy.pi * s[0]) * sy.sin(sy.pi * s[1]) * sy.sin(sy.pi * s[2])
    F = sy.Matrix([s[a] + eps * g for a in range(3)])
    J = F.jacobian(list(s))
    detJ = J.det()
    Ji = J.inv()
    G = detJ * (Ji * Ji.T)
    fdet = sy.lambdify(s, detJ, "numpy")
    fG = [[sy.lambdify(s, G[a, b], "numpy") for b in range(3)] for a in range(3)]
    knots = open_uniform_knots(n_el, p)

    def basis(k, d):
        c = np.zeros(sp.m)
        c[k] = 1.0
        b = BSpline(knots, c, p)
        return b.derivative() if d else b

    gx, gw = _gauss(12)
    pairs = [((0, 0, 0), (1, 2, 0)), ((5, 4, 6), (6, 5, 7)), ((3, 7, 2), (2, 6, 4)), ((6, 6, 6), (6, 6, 6)),
             ((11, 0, 5), (10, 1, 5))]
    rows = np.array([a for a, _ in pairs])
    TK, TM = true_rows(sp, rows)
    deltas = sp.deltas()
    for r, (i, j) in enumerate(pairs):
        lo = [max(0, max(i[k], j[k]) - p) for k in range(3)]
        hi = [min(n_el, min(i[k], j[k]) + 1) for k in range(3)]
        pts, wts = [], []
        for k in range(3):
            e = np.arange(lo[k], hi[k])
            pts.append(((e[:, None] + gx[None, :]) / n_el).ravel())
            wts.append(np.tile(gw / n_el, len(e)))
        S0, S1, S2 = np.meshgrid(*pts, indexing="ij")
        W = np.einsum("a,b,c->abc", *wts)
        bi = [basis(i[k], 0)(pts[k]) for k in range(3)]
        bj = [basis(j[k], 0)(pts[k]) for k in range(3)]
        di = [basis(i[k], 1)(pts[k]) for k in range(3)]
        dj = [basis(j[k], 1)(pts[k]) for k in range(3)]
        Bi = np.einsum("a,b,c->abc", *bi)
        Bj = np.einsum("a,b,c->abc", *bj)
        gi = [np.einsum("a,b,c->abc", *[di[k] if k == a else bi[k] for k in range(3)]) for a in range(3)]
        gj = [np.einsum("a,b,c->abc", *[dj[k] if k == a else bj[k] for k in range(3)]) for a in range(3)]
        dt = fdet(S0, S1, S2)
        m_ref = np.sum(W * Bi * Bj * dt)
        k_ref = 0.0
        for a in range(3):
            for b in range(3):
                k_ref += np.sum(W * gi[a] * np.broadcast_to(fG[a][b](S0, S1, S2), S0.shape) * gj[b])
        dl = np.array(j) - np.array(i)
        t = int(np.flatnonzero((deltas == dl).all(axis=1))[0])
        assert abs(TM[r, t] - m_ref) <= 1e-11 * abs(m_ref) + 1e-16
        assert abs(TK[r, t] - k_ref) <= 1e-10 * max(abs(k_ref), 1e-3 * np.abs(TK[r]).max())


def test_sincos_coefficient_closed_form():
    # c(x) = 1 + a sin(2 pi x) cos(2 pi y): (1/4, 0) -> 1 + a, (3/4, 0) -> 1 - a,
    # (1/4, 1/2) -> 1 - a, (0, y) -> 1
    co = SinCosCoef(0.5)
    x = np.array([[0.25, 0.0], [0.75, 0.0], [0.25, 0.5], [0.0, 0.3]])
    assert np.allclose(co.c2(x, x), [2.25, 0.25, 0.25, 1.0], rtol=0, atol=1e-15)


def test_ricker_closed_form():
    # r(t0) = 1; zero crossings where (pi f0 (t - t0))^2 = 1/2; r(t0 + 1/(pi f0)) = -exp(-1)
    f0, t0 = 10.0, 0.1
    dz = 1.0 / (np.sqrt(2.0) * np.pi * f0)
    assert ricker(t0, f0, t0) == 1.0
    assert abs(ricker(t0 + dz, f0, t0)) < 1e-15 and abs(ricker(t0 - dz, f0, t0)) < 1e-15
    assert abs(ricker(t0 + 1.0 / (np.pi * f0), f0, t0) + np.exp(-1.0)) < 1e-15
