"""3-D multi-patch operators (C ABI) against the oracle's multi-patch assembly on the same
box patches (Sec. 3.2 / 3.4 multi-patch remarks, glued along faces): the numbering
bit-exact (including the orientation codes of turned and swapped faces), global applies to
1e-12 (FP64) / 2e-5 (FP32) relative to the |A| |x| scale, the domain volume and the
constant kernel through the matrix-free apply, and the mass solve against a sparse
direct solve of the oracle's global matrix."""
import numpy as np
import pytest

import inputs
from oracle.assembly import Space, true_rows
from oracle.geometry import BoxMap, ConstCoef
from oracle.multipatch import assemble_global, global_numbering
from oracle.surrogate import Surrogate
from tests.test_oracle_multipatch_3d import eight_boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga


def two_boxes():
    """[0, 1]^3 cut at x = 1/2, wave speed 1 on the left and 2 on the right."""
    return [((0.0, 0.0, 0.0), (0.5, 1.0, 1.0)), ((0.5, 0.0, 0.0), (0.5, 1.0, 1.0))], [1.0, 2.0], [(0, 1, 1, 0, 0)]


class Setup:
    def __init__(self, boxes, cs, ifs, p, n_el, q=2, M=2, true_only=False, spaces=None):
        self.spaces = spaces or [Space(3, p, n_el, BoxMap(o, e), ConstCoef(c)) for (o, e), c in zip(boxes, cs)]
        self.maps, self.G = global_numbering([s.m for s in self.spaces], ifs, dim=3)
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
        self.gspaces = [iga.iga_space_create(3, p, n_el, iga.IGA_MAP_BOX, 0.0, iga.IGA_COEF_CONST, c,
                                             box=tuple(o) + tuple(e)) for (o, e), c in zip(boxes, cs)]
        flags = iga.IGA_TRUE_ONLY if true_only else 0
        self.gops = [iga.iga_surrogate_assemble(s, p, q, M, flags) for s in self.gspaces]
        self.mp = iga.iga_multipatch_create(self.gops, ifs)

    def close(self):
        iga.iga_multipatch_destroy(self.mp)
        for o in self.gops:
            iga.iga_ops_destroy(o)
        for s in self.gspaces:
            iga.iga_space_destroy(s)


def eight_box_setup():
    k, p = 6, 1
    coef = ConstCoef(1.3)
    spaces, _, ifs = eight_boxes(k, p, coef)
    boxes = [(sp.geometry.origin, sp.geometry.extent) for sp in spaces]
    return Setup(boxes, [1.3] * 8, ifs, p=p, n_el=k, true_only=True, spaces=spaces)


def apply(st, which, dtype, x):
    xt = torch.tensor(x, dtype=torch.float64 if dtype == iga.IGA_F64 else torch.float32, device="cuda")
    y = torch.empty_like(xt)
    iga.iga_multipatch_apply(st.mp, which, dtype, xt, y, xt.shape[0])
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("case", ["eight_boxes_p1_true", "two_boxes_p2"])
def test_multipatch_3d_numbering_and_applies_match_oracle(case):
    st = eight_box_setup() if case == "eight_boxes_p1_true" else Setup(*two_boxes(), p=2, n_el=10)
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
        one = np.ones((1, st.G))
        assert abs(apply(st, iga.IGA_OP_M, iga.IGA_F64, one).sum() - 1.0) <= 1e-12
        assert np.abs(apply(st, iga.IGA_OP_K, iga.IGA_F64, one)).max() <= 1e-12 * abs(st.K).max()
    finally:
        st.close()


@pytest.mark.parametrize("orient", [4, 5, 6, 7])
def test_multipatch_3d_swapped_face_numbering_matches_oracle(orient):
    """Orientation codes with the swap bit (no box map turns a face that way, so this is a
    numbering check: the library follows the oracle's rule, which the oracle's own tests pin
    by hand)."""
    boxes, cs = [((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), ((1.0, 0.0, 0.0), (1.0, 1.0, 1.0))], [1.0, 1.0]
    for fa, fb in ((1, 0), (5, 2), (3, 4)):
        ifs = [(0, fa, 1, fb, orient)]
        sp = [Space(3, 1, 6, BoxMap(o, e), ConstCoef(c)) for (o, e), c in zip(boxes, cs)]
        maps, G = global_numbering([s.m for s in sp], ifs, dim=3)
        gs = [iga.iga_space_create(3, 1, 6, iga.IGA_MAP_BOX, 0.0, iga.IGA_COEF_CONST, 1.0, box=o + e)
              for o, e in boxes]
        go = [iga.iga_surrogate_assemble(s, 1, 1, 1, iga.IGA_TRUE_ONLY) for s in gs]
        mp = iga.iga_multipatch_create(go, ifs)
        try:
            assert iga.iga_multipatch_size(mp) == G == 2 * 7 ** 3 - 7 ** 2
            for l in range(2):
                assert np.array_equal(iga.iga_multipatch_global_index(mp, l, sp[l].N), maps[l])
        finally:
            iga.iga_multipatch_destroy(mp)
            for o in go:
                iga.iga_ops_destroy(o)
            for s in gs:
                iga.iga_space_destroy(s)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_multipatch_3d_mass_solve_matches_direct_solve(dtype):
    import scipy.sparse.linalg as spla
    st = Setup(*two_boxes(), p=2, n_el=10)
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


def test_multipatch_3d_rejects_bad_orientation_and_mixed_dimensions():
    a = iga.iga_space_create(3, 1, 6, iga.IGA_MAP_BOX, 0.0, iga.IGA_COEF_CONST, 1.0, box=(0, 0, 0, 1, 1, 1))
    b = iga.iga_space_create(3, 1, 6, iga.IGA_MAP_BOX, 0.0, iga.IGA_COEF_CONST, 1.0, box=(1, 0, 0, 1, 1, 1))
    c = iga.iga_space_create(2, 1, 6, iga.IGA_MAP_IDENTITY, 0.0, iga.IGA_COEF_CONST, 1.0)
    ops = [iga.iga_surrogate_assemble(s, 1, 1, 1, iga.IGA_TRUE_ONLY) for s in (a, b, c)]
    try:
        for patches, ifs in (([ops[0], ops[1]], [(0, 1, 1, 0, 8)]), ([ops[0], ops[1]], [(0, 6, 1, 0, 0)]),
                             ([ops[0], ops[2]], [(0, 1, 1, 0, 0)])):
            with pytest.raises(iga.IgaError) as ei:
                iga.iga_multipatch_create(patches, ifs)
            assert ei.value.code == iga.IGA_ERR_ARG
    finally:
        for o in ops:
            iga.iga_ops_destroy(o)
        for s in (a, b, c):
            iga.iga_space_destroy(s)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_multipatch_3d_leapfrog_matches_oracle(dtype):
    """Leapfrog on the glued two-box operator (Ricker source in one box, receivers in both,
    one on the shared face) against the oracle's global leapfrog: state and traces to
    1e-10 (FP64) / 2e-5 (FP32)."""
    import scipy.sparse.linalg as spla
    from oracle.multipatch import global_point_values, leapfrog_global
    st = Setup(*two_boxes(), p=2, n_el=10)
    try:
        lam = spla.eigsh(st.K.tocsc(), k=1, M=st.M.tocsc(), which="LM", return_eigenvectors=False)[0]
        dt, nsteps = 0.5 / np.sqrt(lam), 40
        src_patch, src_s = 0, (0.7, 0.45, 0.55)
        rec_patch = [0, 1, 1]
        rec_s = [(0.5, 0.5, 0.5), (0.3, 0.6, 0.4), (0.0, 0.5, 0.5)]
        S = global_point_values(st.spaces, st.maps, st.G, src_patch, src_s)
        R = [global_point_values(st.spaces, st.maps, st.G, l, s) for l, s in zip(rec_patch, rec_s)]
        u_ref, tr_ref = leapfrog_global(st.K, st.M, dt, np.zeros(st.G), nsteps, source=(S, 10.0, 0.1, 1.0),
                                        receivers=R, rtol=1e-13)
        dt_ = iga.IGA_F64 if dtype == "f64" else iga.IGA_F32
        u = torch.zeros(st.G, dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")
        rtol = 1e-13 if dtype == "f64" else 1e-7
        tr, iters = iga.iga_multipatch_leapfrog(st.mp, dt_, dt, nsteps, u, src_patch, src_s, 10.0, 0.1, 1.0,
                                                rec_patch, rec_s, cg_rtol=rtol, cg_max_it=3000)
        torch.cuda.synchronize()
        ug = u.double().cpu().numpy()
        tol = 1e-10 if dtype == "f64" else 2e-5
        assert iters > nsteps
        assert np.linalg.norm(ug - u_ref) <= tol * np.linalg.norm(u_ref)
        assert np.abs(tr - tr_ref).max() <= tol * np.abs(u_ref).max()
    finally:
        st.close()
