"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own code path: library routines
(numpy / scipy / sympy), closed forms, invariants stated in the paper, textbook
values, or brute force.  No GPU is needed.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy.interpolate import BSpline, make_interp_spline

import inputs
from oracle.assembly import Space, stencil_to_csr, true_rows
from oracle.bspline import collocation, gauss_legendre, greville, open_uniform_knots
from oracle.geometry import (AnnulusQuarter, BsplineThetaCoef, ConstCoef, CubeSinePerturbed,
                             IdentityMap, SinCosCoef)
from oracle.surrogate import Surrogate, interp_knots, sample_indices
from oracle.wave import Leapfrog, gaussian_pulse, pcg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- primitives
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9])
def test_gauss_legendre_matches_numpy_and_is_exact(n):
    x, w = gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(np.sort(x), 0.5 * (xr + 1), atol=1e-14)
    np.testing.assert_allclose(w[np.argsort(x)], 0.5 * wr, atol=1e-14)
    for k in range(2 * n):          # exact for degree <= 2n-1 on [0, 1]
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("p,n_el", [(1, 5), (2, 7), (3, 9), (5, 11)])
def test_bspline_collocation_matches_scipy(p, n_el):
    t = open_uniform_knots(n_el, p)
    x = np.linspace(0.0, 1.0, 41)
    B = collocation(t, p, x)
    np.testing.assert_allclose(B, BSpline.design_matrix(x, t, p).toarray(), atol=1e-14)
    D = collocation(t, p, x, 1)
    for k in range(B.shape[1]):
        c = np.zeros(B.shape[1])
        c[k] = 1.0
        np.testing.assert_allclose(D[:, k], BSpline(t, c, p).derivative()(x), atol=1e-12)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-14)        # partition of unity
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-12)


def test_greville_reproduces_linear_functions():
    t = open_uniform_knots(9, 3)
    x = np.linspace(0, 1, 23)
    np.testing.assert_allclose(collocation(t, 3, x) @ greville(t, 3), x, atol=1e-14)


# ---------------------------------------------------------------- true matrices
def _golden_stencils():
    out = {}
    with open(os.path.join(GOLDEN, "cardinal_stencils.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            out[(int(tok[0]), tok[1])] = np.array([float(v) for v in tok[3:]]) / float(tok[2])
    return out


@pytest.mark.parametrize("p", [2, 3])
def test_golden_1d_stencils_are_cardinal_bspline_values(p):
    """The fixture equals Phi_{2p+1} and -Phi''_{2p+1} at the integers (scipy)."""
    g = _golden_stencils()
    n = 2 * p + 1
    phi = BSpline.basis_element(np.arange(n + 2) - (n + 1) / 2.0, extrapolate=False)
    z = np.arange(-p, p + 1, dtype=float)
    np.testing.assert_allclose(np.nan_to_num(phi(z)), g[(p, "M")], atol=1e-14)
    np.testing.assert_allclose(-np.nan_to_num(phi.derivative(2)(z)), g[(p, "K")], atol=1e-13)


@pytest.mark.parametrize("dim,p,n_el", [(2, 2, 12), (2, 3, 15), (3, 2, 10)])
def test_identity_map_interior_rows_are_tensor_cardinal_stencils(dim, p, n_el):
    g = _golden_stencils()
    sp = Space(dim, p, n_el, IdentityMap(dim), ConstCoef())
    h = sp.h
    m1, k1 = h * g[(p, "M")], g[(p, "K")] / h
    # rows whose whole stencil is made of cardinal functions: 0-based [2p, m-2p-1]
    lo, hi = 2 * p, sp.m - 2 * p - 1
    rows = np.array([[lo] * dim, [hi] * dim, [(lo + hi) // 2] * dim, [lo] + [hi] * (dim - 1)])
    TK, TM = true_rows(sp, rows)
    if dim == 2:
        M_ref = np.einsum('b,a->ba', m1, m1).ravel()        # [d2, d1] -> colex
        K_ref = (np.einsum('b,a->ba', m1, k1) + np.einsum('b,a->ba', k1, m1)).ravel()
    else:
        M_ref = np.einsum('c,b,a->cba', m1, m1, m1).ravel()
        K_ref = (np.einsum('c,b,a->cba', m1, m1, k1) + np.einsum('c,b,a->cba', m1, k1, m1)
                 + np.einsum('c,b,a->cba', k1, m1, m1)).ravel()
    for r in range(len(rows)):
        np.testing.assert_allclose(TM[r], M_ref, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(TK[r], K_ref, rtol=1e-12, atol=1e-14)


def test_mass_total_is_domain_volume_annulus():
    """sum_ij M_ij = |Omega| = 3 pi / 4 for the quarter annulus (partition of unity)."""
    sp = Space(2, 2, 16, AnnulusQuarter(), SinCosCoef())
    _, TM = true_rows(sp, sp.all_rows())
    assert abs(TM.sum() - 0.75 * np.pi) < 1e-13


def test_mass_total_is_domain_volume_perturbed_cube():
    """det J = 1 + 0.1 (g_s + g_t + g_u) integrates to 1: |Omega| = 1."""
    theta = inputs.theta_lognormal(n=6, dim=3)
    sp = Space(3, 2, 6, CubeSinePerturbed(0.1), BsplineThetaCoef(theta))
    _, TM = true_rows(sp, sp.all_rows())
    # (p+1)-point Gauss does not integrate the sine terms exactly; it is accurate to ~h^6
    assert abs(TM.sum() - 1.0) < 1e-5
    sp_fine = Space(3, 2, 6, CubeSinePerturbed(0.1), ConstCoef(), quad_pts=8)
    _, TMf = true_rows(sp_fine, sp_fine.all_rows())
    assert abs(TMf.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("case", ["annulus_sincos", "cube_theta"])
def test_stiffness_rows_sum_to_zero_and_symmetric(case):
    """Eq. RowSumProperty: constants are in the kernel of K; K and M are symmetric."""
    if case == "annulus_sincos":
        sp = Space(2, 3, 14, AnnulusQuarter(), SinCosCoef())
    else:
        sp = Space(3, 2, 6, CubeSinePerturbed(0.1), BsplineThetaCoef(inputs.theta_lognormal(n=5)))
    TK, TM = true_rows(sp, sp.all_rows())
    assert np.abs(TK.sum(1)).max() < 1e-13 * np.abs(TK).max()
    K = stencil_to_csr(sp, TK)
    M = stencil_to_csr(sp, TM)
    assert abs(K - K.T).max() < 1e-14 * np.abs(TK).max()
    assert abs(M - M.T).max() < 1e-16 + 1e-14 * np.abs(TM).max()
    assert (TM >= -1e-18).all()                      # B-spline mass entries are non-negative


def test_stiffness_annihilates_linear_functions_away_from_boundary():
    """Identity map, c = 1: a(x_1, phi_i) = 0 when phi_i vanishes on the boundary."""
    sp = Space(2, 3, 12, IdentityMap(2), ConstCoef())
    TK, _ = true_rows(sp, sp.all_rows())
    K = stencil_to_csr(sp, TK)
    gam = greville(sp.knots, sp.p)
    rows = sp.all_rows()
    u = gam[rows[:, 0]]                                      # coefficients of x_1
    Ku = K @ u
    inner = np.all((rows >= 1) & (rows <= sp.m - 2), axis=1)
    assert np.abs(Ku[inner]).max() < 1e-13
    assert np.abs(Ku[~inner]).max() > 1e-3                   # boundary flux rows do not vanish


def test_brute_force_entries_tiny_mesh():
    """Entries vs adaptive quadrature with scipy B-splines and a sympy Jacobian (n_el = 4p+2)."""
    import sympy as sy
    from scipy.integrate import dblquad
    p, n_el = 2, 10
    sp = Space(2, p, n_el, AnnulusQuarter(), ConstCoef(), quad_pts=p + 1)
    sp_hi = Space(2, p, n_el, AnnulusQuarter(), ConstCoef(), quad_pts=14)
    s, t = sy.symbols('s t')
    F = sy.Matrix([(1 + s) * sy.cos(sy.pi * t / 2), (1 + s) * sy.sin(sy.pi * t / 2)])
    J = F.jacobian([s, t])
    detJ = sy.simplify(J.det())
    G = sy.simplify(detJ * (J.inv() * J.inv().T))
    fdet = sy.lambdify((s, t), detJ)
    fG = sy.lambdify((s, t), G)
    knots = open_uniform_knots(n_el, p)

    def basis(k, deriv=0):
        c = np.zeros(sp.m)
        c[k] = 1.0
        b = BSpline(knots, c, p)
        return b.derivative() if deriv else b

    pairs = [((0, 0), (1, 2)), ((5, 5), (6, 7)), ((11, 3), (10, 1)), ((4, 6), (4, 6))]
    rows = np.array([a for a, _ in pairs])
    TK, TM = true_rows(sp, rows)
    TKh, _ = true_rows(sp_hi, rows)
    for r, (i, j) in enumerate(pairs):
        bi = [basis(i[0]), basis(i[1])]
        bj = [basis(j[0]), basis(j[1])]
        di = [basis(i[0], 1), basis(i[1], 1)]
        dj = [basis(j[0], 1), basis(j[1], 1)]

        def fm(tt, ss):
            return bi[0](ss) * bi[1](tt) * bj[0](ss) * bj[1](tt) * fdet(ss, tt)

        def fk(tt, ss):
            gi = np.array([di[0](ss) * bi[1](tt), bi[0](ss) * di[1](tt)])
            gj = np.array([dj[0](ss) * bj[1](tt), bj[0](ss) * dj[1](tt)])
            return gi @ np.array(fG(ss, tt), dtype=float) @ gj

        lo = [max(0, min(i[k], j[k]) - p) for k in range(2)]
        hi = [min(n_el, max(i[k], j[k]) + 1) for k in range(2)]
        m_ref = k_ref = 0.0
        for es in range(lo[0], hi[0]):
            for et in range(lo[1], hi[1]):
                a = (es / n_el, (es + 1) / n_el, et / n_el, (et + 1) / n_el)
                m_ref += dblquad(fm, a[0], a[1], a[2], a[3], epsabs=1e-14, epsrel=1e-13)[0]
                k_ref += dblquad(fk, a[0], a[1], a[2], a[3], epsabs=1e-14, epsrel=1e-13)[0]
        dt = (j[0] - i[0] + p) + (j[1] - i[1] + p) * (2 * p + 1)
        # mass integrand is polynomial (det J linear in s): p+1 Gauss points are exact
        assert abs(TM[r, dt] - m_ref) < 1e-13 * max(1.0, abs(m_ref)) + 1e-16
        # stiffness has a 1/(1+s) factor: converges with more points
        assert abs(TKh[r, dt] - k_ref) < 1e-10 * max(1.0, abs(k_ref))
        assert abs(TK[r, dt] - k_ref) < 1e-3 * max(1e-3, abs(k_ref))


# ---------------------------------------------------------------- surrogate
def test_sampling_rule_config1_and_rounding():
    """Sec. 5.1: L = m - 4p interior points, every (L-1)/ceil((L-1)/M)-th, rounded."""
    got = sample_indices(66, 2, 4) - 4
    ref = [0, 4, 8, 11, 15, 19, 23, 27, 30, 34, 38, 42, 46, 49, 53, 57]
    assert list(got) == ref
    # L - 1 = 3, M = 2: spacing 1.5, the tie j = 1 rounds away from zero to 2
    assert list(sample_indices(8, 1, 2) - 2) == [0, 2, 3]
    # M = 1 samples every interior point
    assert list(sample_indices(30, 3, 1)) == list(range(6, 24))
    # both end points of the interior set are always sampled
    for m, p, M in [(131, 3, 8), (98, 2, 6), (515, 3, 8), (66, 2, 4)]:
        s = sample_indices(m, p, M)
        assert s[0] == 2 * p and s[-1] == m - 2 * p - 1
        assert np.all(np.diff(s) <= int(np.ceil((m - 4 * p - 1) / np.ceil((m - 4 * p - 1) / M))))


def _interp_case(dim):
    if dim == 2:
        sp = Space(2, 2, 40, AnnulusQuarter(), SinCosCoef())
        return sp, Surrogate(sp, 3, 5)
    sp = Space(3, 2, 20, CubeSinePerturbed(0.1), BsplineThetaCoef(inputs.theta_lognormal(n=6)))
    return sp, Surrogate(sp, 2, 4)


@pytest.mark.parametrize("dim", [2, 3])
def test_interpolation_matches_scipy_with_same_knots(dim):
    """Coefficients equal scipy's interpolating spline applied direction by direction."""
    sp, S = _interp_case(dim)
    t = sp.D // 2 + 3
    vals = S.sK[t]
    C = vals
    for k in range(dim):
        spl = make_interp_spline(S.xs, np.moveaxis(C, k, 0), k=S.q, t=S.iknots, axis=0)
        C = np.moveaxis(spl.c, 0, k)          # scipy puts the interpolation axis first
    np.testing.assert_allclose(C, S.cK[t], rtol=1e-11, atol=1e-13 * np.abs(vals).max())
    knots = interp_knots(S.xs, S.q)
    assert len(knots) == len(S.xs) + S.q + 1


@pytest.mark.parametrize("dim", [2, 3])
def test_interpolant_reproduces_samples_in_every_dimension(dim):
    """Sec. 3.3: the surrogate stencil function interpolates the sampled values."""
    sp, S = _interp_case(dim)
    grids = np.meshgrid(*([S.samp] * dim), indexing='ij')
    pts = np.stack([g.ravel() for g in grids], axis=1)
    for t in (sp.D // 2, sp.D - 1, sp.D // 2 + 5):
        got = S.evaluate('K', t, pts).reshape((len(S.samp),) * dim)
        np.testing.assert_allclose(got, S.sK[t], rtol=1e-12, atol=1e-14 * np.abs(S.sK[t]).max())


def _surrogate_case(dim=2):
    if dim == 2:
        sp = Space(2, 2, 64, AnnulusQuarter(), SinCosCoef(0.5))
        return sp, Surrogate(sp, 2, 4)
    sp = Space(3, 2, 20, CubeSinePerturbed(0.1), BsplineThetaCoef(inputs.theta_lognormal(n=6)))
    return sp, Surrogate(sp, 2, 4)


@pytest.mark.parametrize("dim", [2, 3])
def test_surrogate_equals_true_at_sample_rows(dim):
    """Interpolation reproduces the sampled values (Sec. 3.3): upper entries and the mass diagonal."""
    sp, S = _surrogate_case(dim)
    g = np.meshgrid(*([S.samp] * dim), indexing='ij')
    rows = np.stack([gg.ravel() for gg in g], 1)
    SK, SM = S.rows(rows)
    TK, TM = true_rows(sp, rows)
    t0 = (sp.D - 1) // 2
    dl = sp.deltas()
    for t in range(t0, sp.D):
        cols = rows + dl[t]
        ok = S.in_interior(cols)
        if t > t0:
            np.testing.assert_allclose(SK[ok, t], TK[ok, t], rtol=1e-12, atol=1e-13 * np.abs(TK).max())
        np.testing.assert_allclose(SM[ok, t], TM[ok, t], rtol=1e-12, atol=1e-14 * np.abs(TM).max())


def test_surrogate_sampling_length_one_is_exact():
    """M = 1 is the paper's reference: every interior row is sampled, K~ = K, M~ = M."""
    sp = Space(2, 2, 24, AnnulusQuarter(), SinCosCoef())
    S = Surrogate(sp, 3, 1)
    SK, SM = S.rows(sp.all_rows())
    TK, TM = true_rows(sp, sp.all_rows())
    assert np.abs(SK - TK).max() < 1e-12 * np.abs(TK).max()
    assert np.abs(SM - TM).max() < 1e-13 * np.abs(TM).max()


def test_annulus_constant_speed_mass_surrogate_is_exact():
    """Quarter annulus, c = 1: M_delta(x~) is affine in x~_1 and constant in x~_2, so q >= 1
    interpolation reproduces it: M~ = M to rounding while K~ != K."""
    sp = Space(2, 2, 64, AnnulusQuarter(), ConstCoef())
    S = Surrogate(sp, 2, 4)
    SK, SM = S.rows(sp.all_rows())
    TK, TM = true_rows(sp, sp.all_rows())
    assert np.abs(SM - TM).max() < 1e-13 * np.abs(TM).max()
    assert np.abs(SK - TK).max() > 1e-9 * np.abs(TK).max()


def test_surrogate_stiffness_kernel_and_symmetry():
    """Eq. DefinitionOfSurrogateMatrixSymmetricKernel: K~ symmetric and K~ 1 = 0."""
    sp, S = _surrogate_case()
    SK, SM = S.rows(sp.all_rows())
    K = stencil_to_csr(sp, SK)
    M = stencil_to_csr(sp, SM)
    # surrogate entries are mirrored exactly; true entries carry quadrature rounding
    assert abs(K - K.T).max() < 1e-14 * np.abs(SK).max()
    assert abs(M - M.T).max() < 1e-14 * np.abs(SM).max()
    assert np.abs(K @ np.ones(sp.N)).max() < 1e-14 * np.abs(SK).max() * sp.D


def test_consistency_error_decays_like_H_to_q_plus_1():
    """Sec. 5.2 / theorem of Sec. 4: consistency error O(H^{q+1}) at fixed h."""
    sp = Space(2, 2, 96, AnnulusQuarter(), ConstCoef())
    rows = sp.all_rows()
    TK, _ = true_rows(sp, rows)
    for q in (1, 2):
        Hs, errs = [], []
        for M in (3, 6, 12):
            S = Surrogate(sp, q, M)
            SK, _ = S.rows(rows)
            Hs.append(S.sampling_length())
            errs.append(np.abs(SK - TK).max() / np.abs(TK).max())
        slope = np.polyfit(np.log(Hs), np.log(errs), 1)[0]
        assert slope > q + 1 - 0.6, (q, slope, errs)


# ---------------------------------------------------------------- time stepping
def _small_wave(surrogate=True):
    sp = Space(2, 2, 16, AnnulusQuarter(), ConstCoef())
    if surrogate:
        S = Surrogate(sp, 2, 2)
        SK, SM = S.rows(sp.all_rows())
    else:
        SK, SM = true_rows(sp, sp.all_rows())
    return sp, SK, SM


def test_pcg_matches_direct_solve():
    sp, SK, SM = _small_wave()
    M = stencil_to_csr(sp, SM)
    b = inputs.vectors(sp.N)[0]
    x, it, rel = pcg(M, b, np.zeros(sp.N), 1.0 / M.diagonal(), 1e-13, 1000)
    x_ref = spla.spsolve(M.tocsc(), b)
    assert rel <= 1e-13 and it > 0
    np.testing.assert_allclose(x, x_ref, rtol=1e-10, atol=1e-10 * np.abs(x_ref).max())


def test_leapfrog_conserves_discrete_energy():
    sp, SK, SM = _small_wave()
    lf = Leapfrog(sp, SK, SM, dt=0.2 / sp.n_el, rtol=1e-14)
    u0 = gaussian_pulse(sp, AnnulusQuarter()(inputs.pulse_centre())[0], 0.15)
    es = []
    u_prev, u = None, u0
    for k in (1, 5, 20, 40):
        u, u_prev, _ = lf.run(u0, k)
        es.append(lf.energy(u_prev, u))
    es = np.array(es)
    assert np.abs(es - es[0]).max() < 1e-10 * abs(es[0])


def test_leapfrog_eigenmode_closed_form():
    """For an eigenpair K~ v = lam M~ v the scheme gives u^n = cos(n w) v, cos w = 1 - dt^2 lam / 2."""
    import scipy.linalg as sla
    sp, SK, SM = _small_wave()
    K = stencil_to_csr(sp, SK).toarray()
    M = stencil_to_csr(sp, SM).toarray()
    lam, V = sla.eigh(K, M)
    k = 7
    v = V[:, k]
    dt = 0.2 / sp.n_el
    lf = Leapfrog(sp, SK, SM, dt=dt, rtol=1e-15, max_it=2000)
    n = 30
    u, _, _ = lf.run(v, n)
    w = np.arccos(1.0 - 0.5 * dt * dt * lam[k])
    np.testing.assert_allclose(u, np.cos(n * w) * v, atol=1e-9 * np.abs(v).max())


def test_cg_start_reproduces_polynomials_in_time():
    """The extrapolated CG start is exact on accelerations a^n that are polynomials in
    n of the extrapolation degree (and not on one degree higher), and the degree drops
    to what the history allows."""
    from oracle.wave import cg_start
    rng = np.random.default_rng(7)
    n = 12
    for deg in (0, 1, 2, 3, 6):
        c = rng.standard_normal((deg + 2, 11))
        poly = lambda t, d: sum(c[i] * float(t) ** i for i in range(d + 1))
        hist = [poly(n - 1 - j, deg) for j in range(deg + 1)]
        want = poly(n, deg)
        np.testing.assert_allclose(cg_start(hist, deg, 11), want, rtol=0, atol=1e-9 * np.abs(want).max())
        # one degree more is not reproduced by this order
        hist1 = [poly(n - 1 - j, deg + 1) for j in range(deg + 1)]
        assert np.abs(cg_start(hist1, deg, 11) - poly(n, deg + 1)).max() > 1e-3 * np.abs(c[deg + 1]).max()
    h = [rng.standard_normal(11) for _ in range(3)]
    assert np.array_equal(cg_start([], 2, 11), np.zeros(11))
    assert np.array_equal(cg_start(h[:1], 2, 11), h[0])
    np.testing.assert_allclose(cg_start(h[:2], 2, 11), 2 * h[0] - h[1])
    np.testing.assert_allclose(cg_start(h, 2, 11), 3 * h[0] - 3 * h[1] + h[2])


def test_leapfrog_extrapolated_start_same_solution_fewer_iterations():
    """The CG start changes the work, not the solution: at a tight tolerance the states
    of guess orders 0 and 2 agree; at a loose one order 2 needs fewer iterations."""
    sp, SK, SM = _small_wave()
    dt = 0.2 / sp.n_el
    u0 = gaussian_pulse(sp, AnnulusQuarter()(inputs.pulse_centre())[0], 0.15)
    ua, _, _ = Leapfrog(sp, SK, SM, dt, rtol=1e-14, max_it=2000, guess_order=0).run(u0, 30)
    ub, _, _ = Leapfrog(sp, SK, SM, dt, rtol=1e-14, max_it=2000, guess_order=2).run(u0, 30)
    assert np.linalg.norm(ua - ub) <= 1e-12 * np.linalg.norm(ua)
    l0 = Leapfrog(sp, SK, SM, dt, rtol=1e-8, max_it=2000, guess_order=0)
    l2 = Leapfrog(sp, SK, SM, dt, rtol=1e-8, max_it=2000, guess_order=2)
    l0.run(u0, 30)
    l2.run(u0, 30)
    assert sum(l2.iters) < sum(l0.iters)
