"""On-the-fly evaluation of the stencil functions inside the apply (IGA_PATH_ONTHEFLY,
Sec. 3.3 matrix-free use of the stencil-function data) against the FP64 oracle's
surrogate matrices and against the stored-field apply, through the C ABI.

Tolerances are those of the other apply tests on the |A| |x| bound of each row: FP64
1e-12, FP32 2e-5 against the oracle; FP64 1e-13 between the two GPU forms (same
values, other summation order).  The meshes have rows of both kinds (surrogate-only
stencils and band rows) in every case.
"""
import functools

import numpy as np
import pytest

import inputs
from oracle.assembly import stencil_to_csr
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
    "cube14_p1": lambda: W.scaled("cube96_p2", n_el=14, p=1, q=1, M=3),
}


@functools.lru_cache(maxsize=None)
def oracle_ops(name):
    w = CASES[name]()
    sp, S = oracle_surrogate(w)
    SK, SM = S.rows(sp.all_rows())
    return sp, stencil_to_csr(sp, SK), stencil_to_csr(sp, SM)


@functools.lru_cache(maxsize=None)
def gpu_ops(name, flags=0):
    w = CASES[name]()
    space = W.make_space(w)
    return space, iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], flags)


def _apply(ops, which, dtype, path, x):
    iga.iga_ops_set_path(ops, path)
    tdt = torch.float64 if dtype == iga.IGA_F64 else torch.float32
    xg = torch.tensor(x, dtype=tdt, device="cuda")
    yg = torch.empty_like(xg)
    iga.iga_stencil_apply(ops, which, dtype, xg, yg, x.shape[0])
    torch.cuda.synchronize()
    iga.iga_ops_set_path(ops, iga.IGA_PATH_AUTO)
    return yg.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("which", ["K", "M"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_onthefly_apply_matches_oracle_and_stored_fields(name, which, dtype):
    sp, K, M = oracle_ops(name)
    _, ops = gpu_ops(name)
    w = iga.IGA_OP_K if which == "K" else iga.IGA_OP_M
    dt = iga.IGA_F64 if dtype == "f64" else iga.IGA_F32
    A = K if which == "K" else M
    x = inputs.vectors(sp.N, 2)
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    ref = (A @ x.T).T
    bound = (abs(A) @ np.abs(x).T).T
    yo = _apply(ops, w, dt, iga.IGA_PATH_ONTHEFLY, x)
    ys = _apply(ops, w, dt, iga.IGA_PATH_ROWS, x)
    tol = 1e-12 if dtype == "f64" else 2e-5
    assert np.all(np.abs(yo - ref) <= tol * bound + 1e-300)
    if dtype == "f64":
        assert np.all(np.abs(yo - ys) <= 1e-13 * bound + 1e-300)


def test_onthefly_volume_preserving_mass_equals_stored_fields():
    sp, _, _ = oracle_ops("cube20_p2_theta")
    _, ops = gpu_ops("cube20_p2_theta", iga.IGA_MASS_VOLUME_PRESERVING)
    x = inputs.vectors(sp.N, 1)
    yo = _apply(ops, iga.IGA_OP_M, iga.IGA_F64, iga.IGA_PATH_ONTHEFLY, x)
    ys = _apply(ops, iga.IGA_OP_M, iga.IGA_F64, iga.IGA_PATH_ROWS, x)
    assert np.abs(yo - ys).max() <= 1e-13 * np.abs(ys).max()


def test_onthefly_needs_a_surrogate_ops():
    _, ops = gpu_ops("annulus64_p2", iga.IGA_TRUE_ONLY)
    with pytest.raises(iga.IgaError):
        iga.iga_ops_set_path(ops, iga.IGA_PATH_ONTHEFLY)
