"""Brick kernels of the 3-D FP32 operators (IGA_PATH_BRICK) vs the FP64 oracle and
vs the row kernels (IGA_PATH_ROWS), through the C ABI.

Tolerance: the FP32 bar of the other apply tests, 2e-5 of the |A| |x| bound of each
row.  Sizes cover an m that is a multiple of 4 and 8, odd m, p = 1 and p = 2, a
lognormal B-spline wave speed and several bricks with clipped edges.
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
    "cube12_p2": lambda: W.scaled("cube96_p2", n_el=12, M=3),            # m = 14
    "cube20_p2_theta": lambda: W.scaled("cube96_p2", n_el=20),           # m = 22
    "cube27_p2_odd": lambda: W.scaled("cube96_p2", n_el=27, M=4),        # m = 29
    "cube14_p1": lambda: W.scaled("cube96_p2", n_el=14, p=1, q=1, M=3),  # m = 15
}


@functools.lru_cache(maxsize=None)
def oracle_ops(name):
    w = CASES[name]()
    sp, S = oracle_surrogate(w)
    SK, SM = S.rows(sp.all_rows())
    return sp, stencil_to_csr(sp, SK), stencil_to_csr(sp, SM)


@functools.lru_cache(maxsize=None)
def gpu_ops(name):
    w = CASES[name]()
    space = W.make_space(w)
    ops = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], 0)
    return space, ops


def _apply(ops, which, path, x):
    iga.iga_ops_set_path(ops, path)
    xg = torch.tensor(x, dtype=torch.float32, device="cuda")
    yg = torch.empty_like(xg)
    iga.iga_stencil_apply(ops, which, iga.IGA_F32, xg, yg, x.shape[0])
    torch.cuda.synchronize()
    iga.iga_ops_set_path(ops, iga.IGA_PATH_AUTO)
    return yg.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
def test_brick_plan_present(name):
    _, ops = gpu_ops(name)
    nb, threads, stages, smem = iga.iga_ops_brick_info(ops)
    assert nb >= 1 and 64 <= threads <= 1024 and stages in (2, 3) and 0 < smem <= 227 * 1024


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("which", ["K", "M"])
def test_brick_apply_vs_oracle_and_rows(name, which):
    sp, K, M = oracle_ops(name)
    _, ops = gpu_ops(name)
    w = iga.IGA_OP_K if which == "K" else iga.IGA_OP_M
    A = K if which == "K" else M
    x = inputs.vectors(sp.N, 3).astype(np.float32)
    xr = x.astype(np.float64)
    ref = (A @ xr.T).T
    bound = (abs(A) @ np.abs(xr).T).T
    yb = _apply(ops, w, iga.IGA_PATH_BRICK, x)
    yr = _apply(ops, w, iga.IGA_PATH_ROWS, x)
    assert np.all(np.abs(yb - ref) <= 2e-5 * bound + 1e-30)
    assert np.all(np.abs(yb - yr) <= 2e-5 * bound + 1e-30)


@pytest.mark.parametrize("which", ["K", "M"])
def test_brick_apply_constant_vector(which):
    # K~ 1 = 0 exactly in the difference form; M~ 1 = the row sums
    sp, K, M = oracle_ops("cube20_p2_theta")
    _, ops = gpu_ops("cube20_p2_theta")
    w = iga.IGA_OP_K if which == "K" else iga.IGA_OP_M
    x = np.ones((1, sp.N), dtype=np.float32)
    yb = _apply(ops, w, iga.IGA_PATH_BRICK, x)
    if which == "K":
        assert np.all(yb == 0.0)
    else:
        ref = np.asarray(M.sum(axis=1)).ravel()
        assert np.all(np.abs(yb[0] - ref) <= 2e-5 * np.abs(ref))


def test_brick_apply_deterministic():
    sp, _, _ = oracle_ops("cube27_p2_odd")
    _, ops = gpu_ops("cube27_p2_odd")
    x = inputs.vectors(sp.N, 1).astype(np.float32)
    a = _apply(ops, iga.IGA_OP_M, iga.IGA_PATH_BRICK, x)
    b = _apply(ops, iga.IGA_OP_M, iga.IGA_PATH_BRICK, x)
    assert np.array_equal(a, b)


def test_path_selection_errors():
    # a 2-D ops has no brick form
    w = W.scaled("annulus64_p2", n_el=12)
    space = W.make_space(w)
    ops = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], 0)
    assert iga.iga_ops_brick_info(ops) == (0, 0, 0, 0)
    with pytest.raises(iga.IgaError):
        iga.iga_ops_set_path(ops, iga.IGA_PATH_BRICK)
    with pytest.raises(iga.IgaError):
        iga.iga_ops_set_path(ops, 7)
    iga.iga_ops_set_path(ops, iga.IGA_PATH_ROWS)
    iga.iga_ops_destroy(ops)
    iga.iga_space_destroy(space)


# ---------------------------------------------------------------- brick form of the mass solve
def _solve(ops, path, b, x0, rtol, max_it, allow_nc=False):
    iga.iga_ops_set_path(ops, path)
    bg = torch.tensor(b[None], device="cuda")
    xg = torch.tensor(x0[None], device="cuda")
    rc, iters, rel = iga.iga_mass_solve(ops, iga.IGA_F32, bg, xg, 1, rtol, max_it, allow_not_converged=allow_nc)
    iga.iga_ops_set_path(ops, iga.IGA_PATH_AUTO)
    return rc, xg.cpu().numpy()[0].astype(np.float64), iters[0], rel[0]


@pytest.mark.parametrize("name", ["cube12_p2", "cube20_p2_theta", "cube27_p2_odd", "cube14_p1"])
def test_brick_pcg_iterates_match_oracle_pcg(name):
    """Fixed 25 iterations (rtol = 0) of the brick-form persistent PCG against the FP64
    oracle PCG on the same FP32-rounded operator and inputs (FP32 bar 2e-5 of the largest
    iterate entry) and against the row-kernel persistent PCG (same recurrence and
    precision; the FP32 mass apply sums in another order)."""
    from oracle.wave import pcg
    sp, _, M = oracle_ops(name)
    _, ops = gpu_ops(name)
    M = M.copy()
    dinv = (1.0 / M.diagonal()).astype(np.float32).astype(np.float64)
    M.data = M.data.astype(np.float32).astype(np.float64)
    b = inputs.vectors(sp.N, 1)[0].astype(np.float32)
    x0 = (0.1 * inputs.vectors(sp.N, 1, seed=99)[0]).astype(np.float32)
    xr, it, _ = pcg(M, b.astype(np.float64), x0.astype(np.float64), dinv, 0.0, 25)
    rc, xb, ib, _ = _solve(ops, iga.IGA_PATH_BRICK, b, x0, 0.0, 25)
    _, xw, iw, _ = _solve(ops, iga.IGA_PATH_ROWS, b, x0, 0.0, 25)
    assert ib == 25 and iw == 25 and it == 25
    scale = np.abs(xr).max()
    assert np.abs(xb - xr).max() <= 2e-5 * scale
    assert np.abs(xb - xw).max() <= 2e-5 * scale


def test_brick_pcg_converges_like_rows_and_is_deterministic():
    sp, _, M = oracle_ops("cube27_p2_odd")
    _, ops = gpu_ops("cube27_p2_odd")
    b = inputs.vectors(sp.N, 1)[0].astype(np.float32)
    x0 = np.zeros(sp.N, dtype=np.float32)
    _, xb, ib, rb = _solve(ops, iga.IGA_PATH_BRICK, b, x0, 1e-6, 500)
    _, xb2, ib2, _ = _solve(ops, iga.IGA_PATH_BRICK, b, x0, 1e-6, 500)
    _, xw, iw, rw = _solve(ops, iga.IGA_PATH_ROWS, b, x0, 1e-6, 500)
    assert rb <= 1e-6 and rw <= 1e-6 and abs(ib - iw) <= 1
    assert ib == ib2 and np.array_equal(xb, xb2)
    # true residual of the FP32-stored solution: its rounding alone leaves about
    # 6e-8 |M| |x|, here ~6e-6 ||b|| (the recursive FP64 residual is the one below 1e-6)
    r = b.astype(np.float64) - M @ xb
    assert np.linalg.norm(r) <= 2e-5 * np.linalg.norm(b)
    assert np.abs(xb - xw).max() <= 1e-4 * np.abs(xw).max()


def test_brick_pcg_zero_rhs_and_non_convergence():
    sp, _, _ = oracle_ops("cube20_p2_theta")
    _, ops = gpu_ops("cube20_p2_theta")
    b = np.zeros(sp.N, dtype=np.float32)
    _, x, it, _ = _solve(ops, iga.IGA_PATH_BRICK, b, np.ones(sp.N, dtype=np.float32), 1e-6, 50)
    assert it == 0 and np.all(x == 0.0)
    b = inputs.vectors(sp.N, 1)[0].astype(np.float32)
    rc, _, it, rel = _solve(ops, iga.IGA_PATH_BRICK, b, np.zeros(sp.N, dtype=np.float32), 1e-9, 2,
                            allow_nc=True)
    assert rc == iga.IGA_ERR_NOT_CONVERGED and it == 2 and rel > 1e-9
