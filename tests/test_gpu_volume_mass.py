"""Volume-preserving surrogate mass (IGA_MASS_VOLUME_PRESERVING, Sec. 3.4 remark on
volume preservation) on the GPU against the oracle's rows_volume_preserving().

Tolerances as in the other FP64 parity tests: 1e-12 relative to the largest
entry for fields, |Omega| to 1e-12 relative, direct-solve agreement to 1e-10.
"""
import functools

import numpy as np
import pytest

import inputs
from oracle.assembly import lumped_mass, stencil_to_csr, true_rows
from tests.oracle_cases import oracle_surrogate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

CASES = {
    "annulus64_p2": lambda: W.scaled("annulus64_p2"),
    "annulus40_p3_sincos": lambda: W.scaled("annulus512_p3", n_el=40),
    "cube20_p2_theta": lambda: W.scaled("cube96_p2", n_el=20),
    # finer sampling: with M = 6 on this small mesh the volume-preserving M~ is indefinite
    "cube20_p2_theta_M2": lambda: W.scaled("cube96_p2", n_el=20, M=2),
}
VOLUME = {"annulus64_p2": 0.75 * np.pi, "annulus40_p3_sincos": 0.75 * np.pi, "cube20_p2_theta": 1.0,
          "cube20_p2_theta_M2": 1.0}


@functools.lru_cache(maxsize=None)
def oracle_vp(name):
    w = CASES[name]()
    sp, S = oracle_surrogate(w)
    rows = sp.all_rows()
    _, SMv = S.rows_volume_preserving(rows)
    return sp, SMv


@functools.lru_cache(maxsize=None)
def gpu_vp(name, extra=0):
    w = CASES[name]()
    space = W.make_space(w)
    ops = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], iga.IGA_MASS_VOLUME_PRESERVING | extra)
    return space, ops


def mass_fields(ops):
    info = iga.iga_ops_info_get(ops)
    t = torch.empty((info.nM, info.N), dtype=torch.float64, device="cuda")
    iga.iga_ops_copy_fields(ops, iga.IGA_OP_M, iga.IGA_F64, t)
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_volume_preserving_mass_fields_match_oracle(name):
    sp, SMv = oracle_vp(name)
    _, ops = gpu_vp(name)
    t0 = (sp.D - 1) // 2
    want = SMv[:, t0:].T
    got = mass_fields(ops)
    assert np.array_equal(got == 0.0, want == 0.0)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("name", list(CASES))
def test_volume_preserving_mass_total_is_domain_volume(name):
    """1^T M~ 1 through the matrix-free apply equals |Omega| (det J integrated exactly
    by the Gauss rule on these maps and even element counts)."""
    _, ops = gpu_vp(name)
    N = iga.iga_ops_info_get(ops).N
    one = torch.ones((1, N), dtype=torch.float64, device="cuda")
    y = torch.empty_like(one)
    iga.iga_stencil_apply(ops, iga.IGA_OP_M, iga.IGA_F64, one, y, 1)
    torch.cuda.synchronize()
    vol = float(y.sum())
    assert abs(vol - VOLUME[name]) <= 1e-12 * VOLUME[name]


def test_volume_preserving_row_sums_are_the_lumped_mass():
    sp, _ = oracle_vp("cube20_p2_theta")
    _, ops = gpu_vp("cube20_p2_theta")
    N = sp.N
    one = torch.ones((1, N), dtype=torch.float64, device="cuda")
    y = torch.empty_like(one)
    iga.iga_stencil_apply(ops, iga.IGA_OP_M, iga.IGA_F64, one, y, 1)
    torch.cuda.synchronize()
    D = lumped_mass(sp, sp.all_rows())
    np.testing.assert_allclose(y.cpu().numpy()[0], D, rtol=1e-12, atol=1e-12 * D.max())


def test_volume_preserving_with_true_only_is_the_true_mass():
    sp, _ = oracle_vp("annulus40_p3_sincos")
    _, ops = gpu_vp("annulus40_p3_sincos", iga.IGA_TRUE_ONLY)
    _, TM = true_rows(sp, sp.all_rows())
    t0 = (sp.D - 1) // 2
    want = TM[:, t0:].T
    assert np.abs(mass_fields(ops) - want).max() <= 1e-12 * np.abs(want).max()


def test_mass_solve_with_volume_preserving_mass_matches_direct_solve():
    import scipy.sparse.linalg as spla
    sp, SMv = oracle_vp("cube20_p2_theta_M2")
    _, ops = gpu_vp("cube20_p2_theta_M2")
    M = stencil_to_csr(sp, SMv).tocsc()
    b = inputs.vectors(sp.N, 2)
    ref = np.stack([spla.spsolve(M, bb) for bb in b])
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    iga.iga_mass_solve(ops, iga.IGA_F64, bg, xg, 2, 1e-13, 2000)
    x = xg.cpu().numpy()
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()


def test_indefinite_volume_preserving_mass_is_reported_by_cg():
    """cube n_el = 20 with M = 6: the row-sum diagonal collects the interpolation error of
    all off-diagonal entries and the volume-preserving M~ has a negative eigenvalue
    (about -7e-8 against a smallest diagonal of 1e-6, by scipy eigsh on the oracle
    matrix); the CG reports the non-positive curvature instead of returning garbage."""
    _, ops = gpu_vp("cube20_p2_theta")
    N = iga.iga_ops_info_get(ops).N
    b = torch.tensor(inputs.vectors(N, 2), device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(iga.IgaError) as ei:
        iga.iga_mass_solve(ops, iga.IGA_F64, b, x, 2, 1e-13, 2000)
    assert ei.value.code == iga.IGA_ERR_NONFINITE
