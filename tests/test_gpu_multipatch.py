"""Multi-patch operators (C ABI) against the oracle's multi-patch assembly on the same
patches: numbering bit-exact, global applies to 1e-12 (FP64) / 2e-5 (FP32) relative
to the |A| |x| scale, the mass solve against a sparse direct solve of the oracle's
global matrix, and the domain volume through the matrix-free apply."""
import numpy as np
import pytest

import inputs
from oracle.assembly import Space, true_rows
from oracle.geometry import AnnulusSector, ConstCoef
from oracle.multipatch import assemble_global, global_numbering
from oracle.surrogate import Surrogate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga

HALF_PI = 0.5 * np.pi


def four_pieces():
    sectors = [(1.0, 1.5, 0.0, HALF_PI / 2), (1.5, 2.0, 0.0, HALF_PI / 2),
               (1.0, 1.5, HALF_PI / 2, HALF_PI), (1.5, 2.0, HALF_PI / 2, HALF_PI)]
    return sectors, [1.0] * 4, [(0, 1, 1, 0, 0), (2, 1, 3, 0, 0), (0, 3, 2, 2, 0), (1, 3, 3, 2, 0)]


def three_sectors():
    e = np.linspace(0.0, HALF_PI, 4)
    return ([(1.0, 2.0, e[l], e[l + 1]) for l in range(3)], [1.0, 2.0, 1.0],
            [(0, 3, 1, 2, 0), (1, 3, 2, 2, 0)])


class Setup:
    def __init__(self, sectors, cs, ifs, p, n_el, q=2, M=2, true_only=False):
        self.spaces = [Space(2, p, n_el, AnnulusSector(*sc), ConstCoef(c)) for sc, c in zip(sectors, cs)]
        self.maps, self.G = global_numbering([s.m for s in self.spaces], ifs)
        tk, tm = [], []
        for sp in self.spaces:
            if true_only:
                K, Mm = true_rows(sp, sp.all_rows())
            else:
                K, Mm = Surrogate(sp, q, M).rows(sp.all_rows())
            tk.append(K)
            tm.append(Mm)
        self.K = assemble_global(self.spaces, tk, self.maps, self.G)
        self.M = assemble_global(self.spaces, tm, self.maps, self.G)
        self.gspaces = [iga.iga_space_create(2, p, n_el, iga.IGA_MAP_ANNULUS_SECTOR, 0.0, iga.IGA_COEF_CONST, c,
                                             sector=sc) for sc, c in zip(sectors, cs)]
        flags = iga.IGA_TRUE_ONLY if true_only else 0
        self.gops = [iga.iga_surrogate_assemble(s, p, q, M, flags) for s in self.gspaces]
        self.mp = iga.iga_multipatch_create(self.gops, ifs)

    def close(self):
        iga.iga_multipatch_destroy(self.mp)
        for o in self.gops:
            iga.iga_ops_destroy(o)
        for s in self.gspaces:
            iga.iga_space_destroy(s)


def apply(st, which, dtype, x):
    xt = torch.tensor(x, dtype=torch.float64 if dtype == iga.IGA_F64 else torch.float32, device="cuda")
    y = torch.empty_like(xt)
    iga.iga_multipatch_apply(st.mp, which, dtype, xt, y, xt.shape[0])
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("case", ["four_pieces_p1_true", "three_sectors_p2"])
def test_multipatch_numbering_and_applies_match_oracle(case):
    if case == "four_pieces_p1_true":
        st = Setup(*four_pieces(), p=1, n_el=6, true_only=True)
    else:
        st = Setup(*three_sectors(), p=2, n_el=16)
    try:
        assert iga.iga_multipatch_size(st.mp) == st.G
        for l, sp in enumerate(st.spaces):
            assert np.array_equal(iga.iga_multipatch_global_index(st.mp, l, sp.N), st.maps[l])
        x = inputs.vectors(st.G, 3)
        for which, A in ((iga.IGA_OP_K, st.K), (iga.IGA_OP_M, st.M)):
            scale = (abs(A) @ np.abs(x).T).T
            ref = (A @ x.T).T
            got = apply(st, which, iga.IGA_F64, x)
            assert np.all(np.abs(got - ref) <= 1e-12 * scale.max()), which
            got32 = apply(st, which, iga.IGA_F32, x)
            assert np.all(np.abs(got32 - ref) <= 2e-5 * scale.max()), which
    finally:
        st.close()


def test_multipatch_volume_and_constant_kernel_through_the_apply():
    st = Setup(*three_sectors(), p=2, n_el=16)
    try:
        one = np.ones((1, st.G))
        assert abs(apply(st, iga.IGA_OP_M, iga.IGA_F64, one).sum() - 0.75 * np.pi) <= 1e-12
        assert np.abs(apply(st, iga.IGA_OP_K, iga.IGA_F64, one)).max() <= 1e-12 * abs(st.K).max()
    finally:
        st.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_multipatch_mass_solve_matches_direct_solve(dtype):
    import scipy.sparse.linalg as spla
    st = Setup(*three_sectors(), p=2, n_el=16)
    try:
        b = inputs.vectors(st.G, 2)
        ref = np.stack([spla.spsolve(st.M.tocsc(), bb) for bb in b])
        dt = iga.IGA_F64 if dtype == "f64" else iga.IGA_F32
        tdt = torch.float64 if dtype == "f64" else torch.float32
        bg = torch.tensor(b, dtype=tdt, device="cuda")
        xg = torch.zeros_like(bg)
        rtol = 1e-13 if dtype == "f64" else 1e-6
        rc, iters, rel = iga.iga_multipatch_mass_solve(st.mp, dt, bg, xg, 2, rtol, 3000)
        assert np.all(rel <= rtol) and np.all(iters > 0)
        tol = 1e-10 if dtype == "f64" else 2e-5
        assert np.abs(xg.double().cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    finally:
        st.close()


def test_multipatch_rejects_unequal_sides():
    a = iga.iga_space_create(2, 2, 16, iga.IGA_MAP_ANNULUS_SECTOR, 0.0, iga.IGA_COEF_CONST, 1.0,
                             sector=(1.0, 2.0, 0.0, 0.5))
    b = iga.iga_space_create(2, 2, 18, iga.IGA_MAP_ANNULUS_SECTOR, 0.0, iga.IGA_COEF_CONST, 1.0,
                             sector=(1.0, 2.0, 0.5, 1.0))
    oa = iga.iga_surrogate_assemble(a, 2, 2, 2)
    ob = iga.iga_surrogate_assemble(b, 2, 2, 2)
    try:
        with pytest.raises(iga.IgaError) as ei:
            iga.iga_multipatch_create([oa, ob], [(0, 3, 1, 2, 0)])
        assert ei.value.code == iga.IGA_ERR_ARG
    finally:
        for o in (oa, ob):
            iga.iga_ops_destroy(o)
        for s in (a, b):
            iga.iga_space_destroy(s)
