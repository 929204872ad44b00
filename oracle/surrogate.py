"""Surrogate stencil functions and surrogate matrices (oracle; test infrastructure only).

Steps, in the paper's order:
1. Cardinal points x~_k = (k - (p+1)/2) h (Sec. 3.1) and the interior set Omega~
   (Sec. 3.3): 1-based k in [2p+1, m-2p] per direction, L = m - 4p points.
2. Sampling (Sec. 5.1): along each direction take every (L-1)/ceil((L-1)/M)-th
   of the L points, rounded to the nearest integer, starting at a corner, so
   both end points are sampled.  Rounding is half away from zero and decided
   in exact integer arithmetic.
3. Sample values M_delta(x~_s), K_delta(x~_s) are the true matrix rows at the
   sample rows (Eq. StencilRoughDefinition).
4. Each stencil function is interpolated by tensor B-splines of degree q whose
   knots are taken from the sample points (Sec. 3.3): end knots of multiplicity
   q+1 at the first / last sample, interior knots by de Boor's knot averaging
   t_{j+q+1} = (x_{j+1} + ... + x_{j+q}) / q.
5. Surrogate matrices by Eq. DefinitionOfSurrogateMatrixSymmetric (mass) and
   Eq. DefinitionOfSurrogateMatrixSymmetricKernel (stiffness): an entry is a
   surrogate value iff both x~_i and x~_j lie in Omega~; the upper triangle
   (colex i < j, i <= j for the mass) evaluates the surrogate at x~_i, the lower
   triangle mirrors it, every other entry is the true one, and the stiffness
   diagonal is minus the off-diagonal row sum on every row.
"""
import numpy as np

from .assembly import lumped_mass, true_rows
from .bspline import collocation


def interior_range(m, p):
    """0-based first and last index of Omega~ in one direction (1-based [2p+1, m-2p])."""
    return 2 * p, m - 2 * p - 1


def cardinal_point(k0, p, h):
    """x~ of 0-based index k0 (1-based k = k0 + 1): (k - (p+1)/2) h."""
    return (k0 + 1 - 0.5 * (p + 1)) * h


def sample_indices(m, p, M):
    """0-based sampled indices along one direction (Sec. 5.1)."""
    lo, hi = interior_range(m, p)
    L = hi - lo + 1
    if L < 1:
        raise ValueError("empty interior")
    if L == 1:
        return np.array([lo])
    n = -(-(L - 1) // M)                      # ceil((L-1)/M) intervals
    # round(j (L-1)/n) half away from zero == floor((2 j (L-1) + n) / (2 n)) for j >= 0
    j = np.arange(n + 1)
    offs = (2 * j * (L - 1) + n) // (2 * n)
    return lo + offs


def mesh_dependent_sampling_length(h, p, q, a=0.0, b=0.0, C=1.0, eps=0.1):
    """Sampling length M(h) of Eq. MeshDependentSamplingLength (Sec. 5.2):
    M(h) = max{1, floor(C h^(eps - 1 + (p + a)/(q + b)))}, in FP64."""
    if not (h > 0 and q + b > 0 and C > 0 and eps > 0):
        raise ValueError("need h > 0, q + b > 0, C > 0, eps > 0")
    return max(1, int(np.floor(C * h ** (eps - 1.0 + (p + a) / (q + b)))))


def _true_rows_chunk(args):
    space, rows = args
    return true_rows(space, rows)


def parallel_true_rows(space, rows, pool=None, chunks=64):
    """true_rows() of many rows, optionally split into chunks over an executor's map();
    rows are independent, so the result is the same as one call."""
    if pool is None or len(rows) < 2 * chunks:
        return true_rows(space, rows)
    parts = np.array_split(np.asarray(rows), chunks)
    out = list(pool.map(_true_rows_chunk, [(space, p) for p in parts]))
    return np.concatenate([o[0] for o in out]), np.concatenate([o[1] for o in out])


def interp_knots(xs, q):
    """Knot vector of order q+1 for interpolation at abscissae xs (de Boor averaging)."""
    xs = np.asarray(xs, dtype=np.float64)
    ns = len(xs)
    inner = [xs[j + 1:j + q + 1].mean() for j in range(ns - q - 1)]
    return np.concatenate([np.full(q + 1, xs[0]), inner, np.full(q + 1, xs[-1])])


class Surrogate:
    """Surrogate K~ and M~ of a Space for interpolation degree q and sampling length M."""

    def __init__(self, space, q, M, pool=None):
        """pool: optional executor whose map() runs the true-row quadrature of chunks of
        the sample rows in parallel (the same arithmetic, row by row)."""
        self.space, self.q, self.M = space, q, M
        sp = space
        self.lo, self.hi = interior_range(sp.m, sp.p)
        self.samp = sample_indices(sp.m, sp.p, M)          # same in every direction
        ns = len(self.samp)
        if ns < q + 1:
            raise ValueError("need at least q+1 samples per direction")
        self.xs = cardinal_point(self.samp, sp.p, sp.h)
        self.iknots = interp_knots(self.xs, q)
        # collocation matrix A[r, c] = beta_c(xs_r); the interpolant's coefficients
        # solve A C = values along each direction
        self.A = collocation(self.iknots, q, self.xs)
        # 3. sample values: true rows at every sample row (tensor grid of samples)
        grids = np.meshgrid(*([self.samp] * sp.dim), indexing='ij')
        srows = np.stack([g.ravel(order='F') for g in grids], axis=1)   # colex order
        TK, TM = parallel_true_rows(sp, srows, pool)
        shape = (ns,) * sp.dim
        # samples[t] is a (ns,)*dim array indexed [s_1, .., s_d]
        self.sK = TK.T.reshape((sp.D,) + shape[::-1]).transpose([0] + list(range(sp.dim, 0, -1)))
        self.sM = TM.T.reshape((sp.D,) + shape[::-1]).transpose([0] + list(range(sp.dim, 0, -1)))
        # 4. coefficients of every stencil function: solve along each direction
        self.cK = np.array([self._coefficients(v) for v in self.sK])
        self.cM = np.array([self._coefficients(v) for v in self.sM])

    def _coefficients(self, vals):
        """Tensor interpolation: solve A C = values along each direction in turn."""
        C = vals
        for k in range(self.space.dim):
            Ck = np.moveaxis(C, k, 0)
            shp = Ck.shape
            Ck = np.linalg.solve(self.A, Ck.reshape(shp[0], -1)).reshape(shp)
            C = np.moveaxis(Ck, 0, k)
        return C

    def evaluate(self, which, t, points):
        """Surrogate stencil function t of K ('K') or M ('M') at interior multi-indices (R, dim)."""
        sp = self.space
        C = (self.cK if which == 'K' else self.cM)[t]
        pts = np.asarray(points).reshape(-1, sp.dim)
        E = [collocation(self.iknots, self.q, cardinal_point(pts[:, k], sp.p, sp.h))
             for k in range(sp.dim)]
        if sp.dim == 2:
            return np.einsum('ra,rb,ab->r', E[0], E[1], C)
        return np.einsum('ra,rb,rc,abc->r', E[0], E[1], E[2], C)

    def in_interior(self, idx):
        idx = np.asarray(idx)
        return np.all((idx >= self.lo) & (idx <= self.hi), axis=-1)

    def rows(self, rows):
        """Surrogate rows (stencil storage) SK, SM for multi-indices rows (R, dim)."""
        sp = self.space
        rows = np.asarray(rows, dtype=np.int64).reshape(-1, sp.dim)
        TK, TM = true_rows(sp, rows)
        SK, SM = TK.copy(), TM.copy()
        dl = sp.deltas()
        t0 = (sp.D - 1) // 2
        row_in = self.in_interior(rows)
        for t, delta in enumerate(dl):
            cols = rows + delta[None, :]
            both = row_in & self.in_interior(cols)
            if not both.any():
                continue
            if t > t0 or (t == t0):
                # upper triangle (colex i < j) and the diagonal: evaluate at x~_i
                vk = self.evaluate('K', t, rows[both]) if t != t0 else None
                vm = self.evaluate('M', t, rows[both])
            else:
                # lower triangle: [A~]_ij = [A~]_ji = A~_{-delta}(x~_j)
                tm = sp.D - 1 - t
                vk = self.evaluate('K', tm, cols[both])
                vm = self.evaluate('M', tm, cols[both])
            if vk is not None:
                SK[both, t] = vk
            SM[both, t] = vm
        # kernel preservation: diagonal = - sum of the off-diagonal row entries (every row)
        off = np.ones(sp.D, dtype=bool)
        off[t0] = False
        SK[:, t0] = -SK[:, off].sum(axis=1)
        return SK, SM

    def rows_volume_preserving(self, rows):
        """Surrogate rows with the volume-preserving mass (Sec. 3.4, remark on
        volume preservation): M~ = D + M~_0, D_ii = integral of B_i, and M~_0 built
        like K~ (Eq. DefinitionOfSurrogateMatrixSymmetricKernel) from the mass
        stencil functions: the off-diagonal entries are those of M~ and the
        diagonal of M~_0 is minus its off-diagonal row sum.  Hence
        [M~]_ii = D_ii - sum_{j != i} [M~]_ij and sum_ij [M~]_ij = |Omega|.
        Returns SK, SM (SK as in rows())."""
        sp = self.space
        rows = np.asarray(rows, dtype=np.int64).reshape(-1, sp.dim)
        SK, SM = self.rows(rows)
        t0 = (sp.D - 1) // 2
        off = np.ones(sp.D, dtype=bool)
        off[t0] = False
        SM[:, t0] = lumped_mass(sp, rows) - SM[:, off].sum(axis=1)
        return SK, SM

    def sampling_length(self):
        """H of Eq. Hdefn: the largest spacing of the interpolation knots."""
        u = np.unique(self.iknots)
        return float(np.max(np.diff(u)))
