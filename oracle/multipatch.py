"""Multi-patch assembly (oracle; test infrastructure only).

Sec. 3.2 (remark on multi-patch geometries) and Sec. 3.4 (remark after
Eq. DefinitionOfSurrogateMatrixSymmetricKernel): the domain is split into patches,
each the image of the parametric square under its own map, with its own stencil
functions; the patch matrices (true or surrogate) are built patch by patch and
added into the global matrix of the C0-conforming multi-patch space, whose basis
functions on a shared side are identified across the patches.

Global numbering (the rule the library follows as well): local functions of all
patches are visited patch by patch, each patch in colexicographic order; the
functions glued by the interfaces form equivalence classes, and a class receives
the next global index when its first member is visited.

Sides of a 2-D patch: 0 = {i_1 = 0}, 1 = {i_1 = m-1}, 2 = {i_2 = 0}, 3 = {i_2 = m-1};
the functions along a side are ordered by the other index, and a reversed
interface pairs entry k of one side with entry m-1-k of the other.
"""
import numpy as np
import scipy.sparse as sps

from .assembly import stencil_to_csr


def side_indices(m, side):
    """Linear (colex) local indices of the m functions on one side of a 2-D patch."""
    k = np.arange(m)
    if side == 0:
        return k * m
    if side == 1:
        return k * m + (m - 1)
    if side == 2:
        return k
    if side == 3:
        return (m - 1) * m + k
    raise ValueError("side must be 0..3")


def global_numbering(ms, interfaces):
    """Local-to-global maps (list of arrays, one per patch) and the global size.

    ms: functions per direction of each patch; interfaces: (patch_a, side_a,
    patch_b, side_b, reversed) tuples, the glued sides having the same m."""
    offs = np.concatenate([[0], np.cumsum([m * m for m in ms])])
    parent = np.arange(offs[-1])

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for pa, sa, pb, sb, rev in interfaces:
        if ms[pa] != ms[pb]:
            raise ValueError("glued sides need the same number of functions")
        ia = offs[pa] + side_indices(ms[pa], sa)
        ib = offs[pb] + side_indices(ms[pb], sb)
        if rev:
            ib = ib[::-1]
        for a, b in zip(ia, ib):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    glob = -np.ones(offs[-1], dtype=np.int64)
    cls = {}
    n = 0
    for k in range(offs[-1]):
        r = find(k)
        if r not in cls:
            cls[r] = n
            n += 1
        glob[k] = cls[r]
    return [glob[offs[l]:offs[l + 1]] for l in range(len(ms))], n


def assemble_global(spaces, tables, maps, n_global):
    """Sum over patches of P_l^T A_l P_l for patch matrices given in stencil storage
    (tables[l]: rows of patch l in colex order, shape (N_l, D))."""
    A = sps.csr_matrix((n_global, n_global))
    for sp, T, g in zip(spaces, tables, maps):
        Al = stencil_to_csr(sp, T).tocoo()
        A = A + sps.csr_matrix((Al.data, (g[Al.row], g[Al.col])), shape=(n_global, n_global))
    return A.tocsr()
