"""Pins of the oracle's multi-patch assembly (Sec. 3.2 and 3.4 remarks on multi-patch
geometries) against facts independent of its code path:

* for p = 1 the C0-glued space of four quarter-annulus pieces is the single-patch
  space of the whole quarter annulus on the same mesh, so the true matrices agree
  entry by entry after renumbering (renumbering by physical node position);
* the mass total is |Omega| = 3 pi / 4, constants lie in the kernel of the
  stiffness, both matrices are symmetric;
* the global size is the local count minus the identified side functions.
"""
import numpy as np

from oracle.assembly import Space, stencil_to_csr, true_rows
from oracle.geometry import AnnulusSector, ConstCoef, SinCosCoef
from oracle.multipatch import assemble_global, global_numbering
from oracle.surrogate import Surrogate

HALF_PI = 0.5 * np.pi


def four_piece_setup(k, p, coef):
    # pieces (radius half, angle half): 0 = (inner, low), 1 = (outer, low), 2 = (inner, high), 3 = (outer, high)
    pieces = [(1.0, 1.5, 0.0, HALF_PI / 2), (1.5, 2.0, 0.0, HALF_PI / 2),
              (1.0, 1.5, HALF_PI / 2, HALF_PI), (1.5, 2.0, HALF_PI / 2, HALF_PI)]
    spaces = [Space(2, p, k, AnnulusSector(*pc), coef) for pc in pieces]
    ifs = [(0, 1, 1, 0, 0), (2, 1, 3, 0, 0), (0, 3, 2, 2, 0), (1, 3, 3, 2, 0)]
    return spaces, ifs


def test_p1_four_pieces_equal_the_single_patch():
    k, p = 6, 1
    coef = SinCosCoef(0.5)
    spaces, ifs = four_piece_setup(k, p, coef)
    maps, G = global_numbering([s.m for s in spaces], ifs)
    single = Space(2, p, 2 * k, AnnulusSector(), coef)
    assert G == single.N
    tabs_k, tabs_m = [], []
    for sp in spaces:
        TK, TM = true_rows(sp, sp.all_rows())
        tabs_k.append(TK)
        tabs_m.append(TM)
    K = assemble_global(spaces, tabs_k, maps, G).toarray()
    M = assemble_global(spaces, tabs_m, maps, G).toarray()
    # renumber by position: piece (rho, alpha), local (i1, i2) -> single (rho k + i1, alpha k + i2)
    perm = np.empty(G, dtype=np.int64)
    for l, (sp, g) in enumerate(zip(spaces, maps)):
        rho, alpha = l % 2, l // 2
        loc = sp.all_rows()
        perm[g] = single.linear(np.stack([rho * k + loc[:, 0], alpha * k + loc[:, 1]], axis=1))
    TK1, TM1 = true_rows(single, single.all_rows())
    K1 = stencil_to_csr(single, TK1).toarray()[np.ix_(perm, perm)]
    M1 = stencil_to_csr(single, TM1).toarray()[np.ix_(perm, perm)]
    assert np.abs(K - K1).max() <= 1e-12 * np.abs(K1).max()
    assert np.abs(M - M1).max() <= 1e-13 * np.abs(M1).max()


def test_three_sector_surrogate_invariants():
    """p = 2, three angular sectors with a speed jump across the interfaces (c = 1, 2, 1),
    surrogate per patch: M~ total = |Omega| (the annulus mass stencils are affine in s and
    reproduced exactly), K~ 1 = 0, both symmetric, global size 3 m^2 - 2 m."""
    n_el, p, q, M_s = 16, 2, 2, 2
    edges = np.linspace(0.0, HALF_PI, 4)
    cs = [1.0, 2.0, 1.0]
    spaces = [Space(2, p, n_el, AnnulusSector(1.0, 2.0, edges[l], edges[l + 1]), ConstCoef(cs[l]))
              for l in range(3)]
    ifs = [(0, 3, 1, 2, 0), (1, 3, 2, 2, 0)]
    m = spaces[0].m
    maps, G = global_numbering([s.m for s in spaces], ifs)
    assert G == 3 * m * m - 2 * m
    tk, tm = [], []
    for sp in spaces:
        SK, SM = Surrogate(sp, q, M_s).rows(sp.all_rows())
        tk.append(SK)
        tm.append(SM)
    K = assemble_global(spaces, tk, maps, G)
    Mm = assemble_global(spaces, tm, maps, G)
    assert abs(Mm.sum() - 0.75 * np.pi) < 1e-13
    assert np.abs(K @ np.ones(G)).max() <= 1e-12 * abs(K).max()
    assert abs(K - K.T).max() <= 1e-14 * abs(K).max()
    assert abs(Mm - Mm.T).max() <= 1e-16


def test_reversed_interface_glues_mirrored_entries():
    """Sector 1 parameterised the other way round in both directions (r = 2 - s,
    angle 0.9 - 0.5 t: positive det J, the shared radial side is now t = 1 and runs
    inwards) glued with the reversed flag gives the same global matrix as the plain
    gluing of the plain map, after renumbering."""
    n_el, p = 6, 2
    a = Space(2, p, n_el, AnnulusSector(1.0, 2.0, 0.0, 0.4), ConstCoef())
    b = Space(2, p, n_el, AnnulusSector(1.0, 2.0, 0.4, 0.9), ConstCoef())
    b_rev = Space(2, p, n_el, AnnulusSector(2.0, 1.0, 0.9, 0.4), ConstCoef())
    maps, G = global_numbering([a.m, b.m], [(0, 3, 1, 2, 0)])
    maps_r, G_r = global_numbering([a.m, b_rev.m], [(0, 3, 1, 3, 1)])
    assert G == G_r
    Ma = [true_rows(sp, sp.all_rows())[1] for sp in (a, b)]
    Mr = [true_rows(sp, sp.all_rows())[1] for sp in (a, b_rev)]
    A = assemble_global([a, b], Ma, maps, G).toarray()
    B = assemble_global([a, b_rev], Mr, maps_r, G_r).toarray()
    # renumber: patch 0 identical; patch 1 local (i1, i2) of b <-> (m-1-i1, m-1-i2) of b_rev
    perm = np.empty(G, dtype=np.int64)
    perm[maps[0]] = maps_r[0]
    loc = b.all_rows()
    perm[maps[1]] = maps_r[1][b.linear(np.stack([b.m - 1 - loc[:, 0], b.m - 1 - loc[:, 1]], axis=1))]
    assert np.abs(A - B[np.ix_(perm, perm)]).max() <= 1e-14 * np.abs(A).max()
