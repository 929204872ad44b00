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

Sides of a patch: side 2k is {i_(k+1) = 0} and side 2k+1 is {i_(k+1) = m-1}, so 2-D
patches have sides 0..3 (m functions each) and 3-D patches faces 0..5 (m^2 functions each).
The functions on a side are ordered colexicographically by the remaining indices.  The
orientation code of an interface says which entry of side b meets entry (u, v) of side a
(u the faster index): bit 2 swaps u and v, then bit 0 reverses u and bit 1 reverses v.  In
2-D only bit 0 exists (the reversed flag).
"""
import numpy as np
import scipy.sparse as sps

from .assembly import stencil_to_csr


def side_indices(m, side, dim=2):
    """Linear (colex) local indices of the functions on one side of a patch with m
    functions per direction, ordered colex by the remaining indices."""
    axis, top = divmod(side, 2)
    if not (0 <= axis < dim):
        raise ValueError("side must be 0..%d" % (2 * dim - 1))
    f = np.arange(m ** (dim - 1))
    coords = [f % m, f // m]             # the remaining indices, the first one fastest
    idx = [None] * dim
    idx[axis] = np.full(f.shape, m - 1 if top else 0)
    for r, k in enumerate([k for k in range(dim) if k != axis]):
        idx[k] = coords[r]
    return sum(idx[k] * m ** k for k in range(dim))


def oriented(m, dim, orient):
    """Position, in side b's order, of the partner of each entry of side a."""
    if dim == 2:
        if orient not in (0, 1):
            raise ValueError("2-D interfaces take orient 0 or 1")
        k = np.arange(m)
        return m - 1 - k if orient else k
    if not (0 <= orient < 8):
        raise ValueError("3-D interfaces take orient 0..7")
    v, u = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    u, v = u.ravel(), v.ravel()          # entry u + m v of side a
    if orient & 4:
        u, v = v, u
    if orient & 1:
        u = m - 1 - u
    if orient & 2:
        v = m - 1 - v
    return u + m * v


def global_numbering(ms, interfaces, dim=2):
    """Local-to-global maps (list of arrays, one per patch) and the global size.

    ms: functions per direction of each patch; interfaces: (patch_a, side_a,
    patch_b, side_b, orient) tuples, the glued sides having the same m."""
    offs = np.concatenate([[0], np.cumsum([m ** dim for m in ms])])
    parent = np.arange(offs[-1])

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for pa, sa, pb, sb, orient in interfaces:
        if ms[pa] != ms[pb]:
            raise ValueError("glued sides need the same number of functions")
        m = ms[pa]
        ia = offs[pa] + side_indices(m, sa, dim)
        ib = (offs[pb] + side_indices(m, sb, dim))[oriented(m, dim, orient)]
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


def global_point_values(spaces, maps, n_global, patch, s):
    """Global basis values at parametric point s of one patch: the patch's local values
    B_i(s) placed at the global indices of its functions."""
    from .wave import point_values
    g = np.zeros(n_global)
    g[maps[patch]] += point_values(spaces[patch], s)
    return g


def leapfrog_global(K, M, dt, u0, nsteps, source=None, receivers=(), rtol=1e-13, max_it=5000):
    """Leapfrog on the global multi-patch matrices, the scheme of oracle.wave.Leapfrog
    (u^{n+1} = 2 u^n - u^{n-1} + dt^2 a^n, M a^n = f^n - K u^n, u^1 = u^0 + dt^2/2 a^0,
    Jacobi-PCG started at a^{n-1}).  source: (S, f0, t0, amp) with S the global point
    values of the source; receivers: global point-value vectors.  Returns
    (u^nsteps, traces[nrec, nsteps]) with traces[:, n] taken from u^{n+1}."""
    from .wave import pcg, ricker
    dinv = 1.0 / M.diagonal()
    u = np.asarray(u0, dtype=np.float64).copy()
    u_prev = None
    a = np.zeros_like(u)
    R = np.array(receivers).reshape(len(receivers), u.size)
    traces = np.zeros((len(receivers), nsteps))
    for n in range(nsteps):
        f = np.zeros_like(u)
        if source is not None:
            S, f0, t0, amp = source
            f = amp * ricker(n * dt, f0, t0) * S
        a, _, _ = pcg(M, f - K @ u, a, dinv, rtol, max_it)
        u_new = u + 0.5 * dt * dt * a if n == 0 else 2.0 * u - u_prev + dt * dt * a
        u_prev, u = u, u_new
        if len(receivers):
            traces[:, n] = R @ u
    return u, traces
