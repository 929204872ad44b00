"""Pins of the oracle's 3-D multi-patch assembly (Sec. 3.2 and 3.4 remarks on multi-patch
geometries, with faces instead of sides) against facts independent of its code path:

* for p = 1 the C0-glued space of the unit cube cut into 2 x 2 x 2 boxes is the
  single-patch space of the cube on the doubled mesh, so the true matrices agree entry
  by entry after renumbering by physical node position.  One box runs its first two
  parametric directions against x and y (a half turn about the z axis), so its faces
  meet their neighbours' with reversed entries (orientation bits 0 and 1);
* the face entry orders and the orientation codes against hand-written index lists;
* the global size is the local count minus the identified face functions.
"""
import numpy as np

from oracle.assembly import Space, stencil_to_csr, true_rows
from oracle.geometry import BoxMap, ConstCoef
from oracle.multipatch import assemble_global, global_numbering, oriented, side_indices

TURNED = 3   # the box at (x, y, z) = (1, 1, 0) of the 2 x 2 x 2 split, turned half about z


def eight_boxes(k, p, coef):
    """Pieces l = px + 2 py + 4 pz of [0, 1]^3 (k elements per direction each) and the
    interfaces that glue every pair of neighbours across their common face."""
    spaces, where = [], []
    for l in range(8):
        px, py, pz = l % 2, (l // 2) % 2, l // 4
        if l == TURNED:
            mp = BoxMap((0.5 * (px + 1), 0.5 * (py + 1), 0.5 * pz), (-0.5, -0.5, 0.5))
        else:
            mp = BoxMap((0.5 * px, 0.5 * py, 0.5 * pz), (0.5, 0.5, 0.5))
        spaces.append(Space(3, p, k, mp, coef))
        where.append((px, py, pz))

    def face(l, axis, high):
        """Side of piece l on its physical face (axis, high) and whether the piece is
        turned (its in-face entry indices along x and y run against x and y)."""
        turned = l == TURNED
        side = 2 * axis + (1 - high if (turned and axis < 2) else high)
        return side, turned

    ifs = []
    for l in range(8):
        for axis in range(3):
            c = list(where[l])
            if c[axis] == 1:
                continue
            c[axis] = 1
            n = c[0] + 2 * c[1] + 4 * c[2]
            sa, fa = face(l, axis, 1)
            sb, fb = face(n, axis, 0)
            # entries (u, v) run over the two remaining axes; when exactly one of the two
            # pieces is turned, the ones along x or y meet reversed
            rest = [a for a in range(3) if a != axis]
            orient = 0
            if fa != fb:
                orient = (1 if rest[0] < 2 else 0) | (2 if rest[1] < 2 else 0)
            ifs.append((l, sa, n, sb, orient))
    return spaces, where, ifs


def test_face_orders_and_orientations_by_hand():
    m = 3
    assert list(side_indices(m, 0, 3)) == [0, 3, 6, 9, 12, 15, 18, 21, 24]      # i1 = 0: (i2, i3)
    assert list(side_indices(m, 3, 3)) == [6, 7, 8, 15, 16, 17, 24, 25, 26]     # i2 = 2: (i1, i3)
    assert list(side_indices(m, 5, 3)) == list(range(18, 27))                  # i3 = 2: (i1, i2)
    assert list(side_indices(4, 1, 2)) == [3, 7, 11, 15]
    # entry u + 3 v of side a meets: swap -> v + 3 u; bit 0 -> (2 - u) + 3 v; bit 1 -> u + 3 (2 - v)
    assert list(oriented(m, 3, 4)) == [0, 3, 6, 1, 4, 7, 2, 5, 8]
    assert list(oriented(m, 3, 1)) == [2, 1, 0, 5, 4, 3, 8, 7, 6]
    assert list(oriented(m, 3, 2)) == [6, 7, 8, 3, 4, 5, 0, 1, 2]
    assert list(oriented(m, 3, 7)) == [8, 5, 2, 7, 4, 1, 6, 3, 0]
    # two 3 x 3 x 3 patches glued face 1 -> face 0 with a swap: size and the pairs
    maps, G = global_numbering([3, 3], [(0, 1, 1, 0, 4)], dim=3)
    assert G == 2 * 27 - 9
    a, b = side_indices(3, 1, 3), side_indices(3, 0, 3)
    for u in range(3):
        for v in range(3):
            assert maps[0][a[u + 3 * v]] == maps[1][b[v + 3 * u]]


def test_p1_eight_boxes_equal_the_single_patch():
    k, p = 6, 1
    coef = ConstCoef(1.3)
    spaces, where, ifs = eight_boxes(k, p, coef)
    maps, G = global_numbering([s.m for s in spaces], ifs, dim=3)
    single = Space(3, p, 2 * k, BoxMap((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), coef)
    assert G == single.N
    tabs_k, tabs_m = [], []
    for sp in spaces:
        TK, TM = true_rows(sp, sp.all_rows())
        tabs_k.append(TK)
        tabs_m.append(TM)
    K = assemble_global(spaces, tabs_k, maps, G).toarray()
    M = assemble_global(spaces, tabs_m, maps, G).toarray()
    perm = np.empty(G, dtype=np.int64)
    for l, (sp, g) in enumerate(zip(spaces, maps)):
        loc = sp.all_rows().copy()
        if l == TURNED:
            loc[:, 0] = k - loc[:, 0]
            loc[:, 1] = k - loc[:, 1]
        perm[g] = single.linear(loc + k * np.asarray(where[l]))
    TK1, TM1 = true_rows(single, single.all_rows())
    K1 = stencil_to_csr(single, TK1).toarray()[np.ix_(perm, perm)]
    M1 = stencil_to_csr(single, TM1).toarray()[np.ix_(perm, perm)]
    assert np.abs(M.sum() - 1.0) <= 1e-13
    assert np.abs(K - K1).max() <= 1e-12 * np.abs(K1).max()
    assert np.abs(M - M1).max() <= 1e-13 * np.abs(M1).max()


def test_global_leapfrog_equals_the_single_patch_leapfrog():
    """With one patch and no interface the global leapfrog is the single-patch oracle
    leapfrog (pinned by its own tests): same steps, sources, receivers and traces."""
    from oracle.geometry import AnnulusSector
    from oracle.multipatch import global_point_values, leapfrog_global
    from oracle.wave import Leapfrog
    sp = Space(2, 2, 10, AnnulusSector(), ConstCoef(1.0))
    SK, SM = true_rows(sp, sp.all_rows())
    maps, G = global_numbering([sp.m], [], dim=2)
    K, M = stencil_to_csr(sp, SK), stencil_to_csr(sp, SM)
    dt, nsteps = 0.01, 25
    src, rec = (0.4, 0.6), [(0.5, 0.5), (0.2, 0.9)]
    lf = Leapfrog(sp, SK, SM, dt, rtol=1e-14, max_it=2000)
    u_ref, _, tr_ref = lf.run(np.zeros(sp.N), nsteps, sources=[(src, 10.0, 0.1, 2.0)], receivers=rec)
    S = global_point_values([sp], maps, G, 0, src)
    R = [global_point_values([sp], maps, G, 0, r) for r in rec]
    u, tr = leapfrog_global(K, M, dt, np.zeros(G), nsteps, source=(S, 10.0, 0.1, 2.0), receivers=R, rtol=1e-14)
    assert np.abs(u[maps[0]] - u_ref).max() <= 1e-12 * np.abs(u_ref).max()
    assert np.abs(tr - tr_ref).max() <= 1e-12 * np.abs(u_ref).max()
