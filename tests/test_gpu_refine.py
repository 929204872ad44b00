"""FP64 mass solves by iterative refinement (IGA_SOLVE_REFINE: FP64 residual with the
FP64 fields, FP32 Jacobi-PCG corrections) against the FP64 Jacobi-PCG, through the C
ABI.  The stopping rule is the FP64 residual, so the refined solve meets the same
tolerance; the solutions agree to the tolerance times the condition of M~."""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W


def _ops(name, **kw):
    w = W.scaled(name, **kw)
    sp = W.make_space(w)
    return sp, iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])


@pytest.mark.parametrize("name,kw,nrhs", [("cube96_p2", dict(n_el=20, M=2), 5), ("annulus512_p3", dict(n_el=40), 1),
                                          ("cube96_p2", dict(n_el=40), 1)])
def test_refined_solve_meets_the_fp64_residual(name, kw, nrhs):
    sp, ops = _ops(name, **kw)
    try:
        N = iga.iga_ops_info_get(ops).N
        b = torch.tensor(inputs.vectors(N, nrhs), device="cuda")
        x_ref = torch.zeros_like(b)
        x = torch.zeros_like(b)
        iga.iga_mass_solve(ops, iga.IGA_F64, b, x_ref, nrhs, 1e-12, 5000)
        _, it, rel = iga.iga_mass_solve(ops, iga.IGA_F64, b, x, nrhs, 1e-12, 5000, flags=iga.IGA_SOLVE_REFINE)
        r = torch.empty_like(b)
        iga.iga_stencil_apply(ops, iga.IGA_OP_M, iga.IGA_F64, x, r, nrhs)
        torch.cuda.synchronize()
        res = (torch.linalg.norm(b - r, dim=1) / torch.linalg.norm(b, dim=1)).cpu().numpy()
        assert np.all(rel <= 1e-12) and np.all(res <= 1.5e-12), (rel, res)
        assert np.all(it > 0)
        scale = x_ref.abs().max().item()
        assert (x - x_ref).abs().max().item() <= 1e-9 * scale
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(sp)


def test_refined_solve_zero_rhs_and_limit():
    sp, ops = _ops("cube96_p2", n_el=20, M=2)
    try:
        N = iga.iga_ops_info_get(ops).N
        b = torch.zeros((1, N), dtype=torch.float64, device="cuda")
        x = torch.ones_like(b)
        _, it, rel = iga.iga_mass_solve(ops, iga.IGA_F64, b, x, 1, 1e-12, 100, flags=iga.IGA_SOLVE_REFINE)
        torch.cuda.synchronize()
        assert float(x.abs().max()) == 0.0 and rel[0] == 0.0
        b = torch.tensor(inputs.vectors(N, 1), device="cuda")
        x = torch.zeros_like(b)
        rc, _, rel = iga.iga_mass_solve(ops, iga.IGA_F64, b, x, 1, 1e-15, 1, flags=iga.IGA_SOLVE_REFINE,
                                        allow_not_converged=True)
        assert rc == iga.IGA_ERR_NOT_CONVERGED and rel[0] > 1e-15
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(sp)
