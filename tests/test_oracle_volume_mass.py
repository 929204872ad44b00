"""Pins of the oracle's volume-preserving surrogate mass (Sec. 3.4, remark on
volume preservation): M~ = D + M~_0 with D_ii = integral of B_i over Omega.

Independent checks: the closed-form integral of a B-spline on the identity map
(knot span / (p+1) per direction), the domain volume |Omega| (perturbed cube: 1,
quarter annulus: 3 pi / 4), the M = 1 reduction to the true mass matrix, and
symmetry / row sums read off the assembled sparse matrix.
"""
import numpy as np

from oracle.assembly import Space, lumped_mass, stencil_to_csr, true_rows
from oracle.geometry import AnnulusQuarter, ConstCoef, CubeSinePerturbed, IdentityMap, SinCosCoef
from oracle.surrogate import Surrogate


def _knots(p, n_el):
    # open uniform knots on [0, 1], written out here independently of the oracle
    return np.concatenate([np.zeros(p + 1), np.arange(1, n_el) / n_el, np.ones(p + 1)])


def test_lumped_mass_identity_map_is_product_of_knot_spans():
    """On the identity map integral B_i = prod_k (t_{i_k+p+1} - t_{i_k}) / (p+1)."""
    for dim, p, n_el in [(2, 2, 10), (2, 3, 12), (3, 2, 8)]:
        sp = Space(dim, p, n_el, IdentityMap(dim), ConstCoef())
        rows = sp.all_rows()
        t = _knots(p, n_el)
        one_d = (t[p + 1:p + 1 + sp.m] - t[:sp.m]) / (p + 1)
        ref = np.prod(one_d[rows], axis=1)
        np.testing.assert_allclose(lumped_mass(sp, rows), ref, rtol=1e-13, atol=1e-17)


def test_volume_preserving_mass_total_is_domain_volume():
    """sum_ij M~ = sum_i D_ii = |Omega| for the surrogate, not only for the true matrix.

    Perturbed cube, |Omega| = 1 (det J = 1 + 0.1 (g_s + g_t + g_u) with g odd about
    the cube centre, so the symmetric Gauss rule on the even element grid gives 1 to
    rounding); the plain surrogate M~ misses the volume by its interpolation error,
    the volume-preserving one does not."""
    sp = Space(3, 2, 10, CubeSinePerturbed(0.1), ConstCoef())
    S = Surrogate(sp, 2, 2)
    rows = sp.all_rows()
    _, SM = S.rows(rows)
    _, SMv = S.rows_volume_preserving(rows)
    vol_plain = stencil_to_csr(sp, SM).sum()
    vol_vp = stencil_to_csr(sp, SMv).sum()
    assert abs(vol_vp - 1.0) < 1e-12
    assert abs(vol_plain - 1.0) > 1e3 * abs(vol_vp - 1.0)


def test_volume_preserving_mass_annulus_volume_and_row_sums():
    """Quarter annulus: |Omega| = 3 pi / 4; row sums of M~ equal D_ii; M~ symmetric."""
    sp = Space(2, 3, 16, AnnulusQuarter(), SinCosCoef())
    S = Surrogate(sp, 3, 2)
    rows = sp.all_rows()
    _, SMv = S.rows_volume_preserving(rows)
    A = stencil_to_csr(sp, SMv)
    assert abs(A.sum() - 0.75 * np.pi) < 1e-13
    D = lumped_mass(sp, rows)
    np.testing.assert_allclose(np.asarray(A.sum(axis=1)).ravel(), D, rtol=1e-12, atol=1e-16)
    assert abs(A - A.T).max() < 1e-16


def test_volume_preserving_mass_with_unit_sampling_is_the_true_mass():
    """M = 1: every off-diagonal entry is true, so D_ii - sum_{j != i} M_ij = M_ii."""
    sp = Space(2, 2, 16, AnnulusQuarter(), SinCosCoef())
    S = Surrogate(sp, 2, 1)
    rows = sp.all_rows()
    _, SMv = S.rows_volume_preserving(rows)
    _, TM = true_rows(sp, rows)
    assert np.abs(SMv - TM).max() < 1e-13 * np.abs(TM).max()
