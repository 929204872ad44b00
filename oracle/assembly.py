"""True stiffness and mass matrices by element-loop Gauss quadrature (oracle; test infrastructure only).

Definitions followed:
* K_ij = a(phi_j, phi_i) = int_{[0,1]^d} c^2 (J^-T grad phi_j) . (J^-T grad phi_i) det J ds
  and M_ij = m(phi_j, phi_i) = int phi_j phi_i det J ds (Eq. weakforms, Eq. SurrogateEoM,
  with the c^2 weight of Eq. LinearWaveEnergy and unit density).
* Tensor-product B-spline basis on open uniform knots, colexicographic global
  index i = i_1 + (i_2 - 1) m + ... (Sec. 3.1).
* Element-wise Gauss quadrature with `quad_pts` points per direction (p+1 by
  default), the standard element loop of Sec. 5.1.

Rows are returned in "stencil" storage: T[r, t] = A(i_r, i_r + delta_t), where
delta_t in {-p..p}^d is enumerated colexicographically (delta_1 fastest), i.e.
t = sum_k (delta_k + p) (2p+1)^(k-1); entries whose column falls outside the
index grid are 0.  This is the row view [A]_ij = A_delta(x_i) of
Eq. StencilRoughDefinition.
"""
import itertools

import numpy as np

from .bspline import collocation, gauss_legendre, open_uniform_knots


class Space:
    """Tensor-product B-spline space of degree p with n_el elements per direction."""

    def __init__(self, dim, p, n_el, geometry, coef, quad_pts=None):
        self.dim = dim
        self.p = p
        self.n_el = n_el
        self.m = n_el + p                       # basis functions per direction
        self.N = self.m ** dim
        self.h = 1.0 / n_el                     # h = 1/(m-p), Sec. 3.1
        self.knots = open_uniform_knots(n_el, p)
        self.geometry = geometry
        self.coef = coef
        self.quad_pts = quad_pts if quad_pts is not None else p + 1
        self.D = (2 * p + 1) ** dim              # #stencil offsets, Sec. 3.2

    # ---- index helpers -------------------------------------------------
    def deltas(self):
        """All offsets delta in colexicographic order, shape (D, dim)."""
        r = range(-self.p, self.p + 1)
        out = [tuple(reversed(t)) for t in itertools.product(r, repeat=self.dim)]
        return np.array(out, dtype=np.int64)

    def linear(self, multi):
        """Colexicographic linear index (0-based) of multi-indices (..., dim)."""
        multi = np.asarray(multi, dtype=np.int64)
        idx = np.zeros(multi.shape[:-1], dtype=np.int64)
        for k in range(self.dim - 1, -1, -1):
            idx = idx * self.m + multi[..., k]
        return idx

    def multi(self, lin):
        lin = np.asarray(lin, dtype=np.int64)
        out = []
        for _ in range(self.dim):
            out.append(lin % self.m)
            lin = lin // self.m
        return np.stack(out, axis=-1)

    def all_rows(self):
        return self.multi(np.arange(self.N))

    # ---- element quadrature -------------------------------------------
    def _tables_1d(self, elems_1d):
        """Gauss points and local basis values / derivatives on the given 1-D elements.

        Returns x[e, g] (parametric coordinates), w[e, g] (weights incl. h) and
        V[e, g, a], G[e, g, a] for the p+1 local functions a = 0..p of element e
        (global 1-D index e + a).
        """
        gx, gw = gauss_legendre(self.quad_pts)
        e = np.asarray(elems_1d)
        x = (e[:, None] + gx[None, :]) * self.h
        w = np.broadcast_to(gw[None, :] * self.h, x.shape)
        Bv = collocation(self.knots, self.p, x.ravel()).reshape(x.shape + (self.m,))
        Bd = collocation(self.knots, self.p, x.ravel(), 1).reshape(x.shape + (self.m,))
        loc = e[:, None] + np.arange(self.p + 1)[None, :]
        V = np.take_along_axis(Bv, loc[:, None, :].repeat(self.quad_pts, 1), axis=2)
        G = np.take_along_axis(Bd, loc[:, None, :].repeat(self.quad_pts, 1), axis=2)
        return x, w, V, G

    def element_volumes(self, elems):
        """Ve[e, a] = int_element phi_a det J ds for the (p+1)^dim local functions a
        (colex local index, as in element_matrices) of elements elems (nE, dim)."""
        elems = np.asarray(elems, dtype=np.int64).reshape(-1, self.dim)
        d, p, nq = self.dim, self.p, self.quad_pts
        tabs = [self._tables_1d(elems[:, k]) for k in range(d)]
        gidx = [tuple(reversed(g)) for g in itertools.product(range(nq), repeat=d)]
        aidx = [tuple(reversed(a)) for a in itertools.product(range(p + 1), repeat=d)]
        nE, NQ, NL = len(elems), len(gidx), len(aidx)
        s = np.empty((nE, NQ, d))
        w = np.ones((nE, NQ))
        for qi, g in enumerate(gidx):
            for k in range(d):
                s[:, qi, k] = tabs[k][0][:, g[k]]
                w[:, qi] *= tabs[k][1][:, g[k]]
        _, J = self.geometry(s)
        detJ = np.linalg.det(J)
        val = np.ones((nE, NQ, NL))
        for qi, g in enumerate(gidx):
            for ai, a in enumerate(aidx):
                for k in range(d):
                    val[:, qi, ai] *= tabs[k][2][:, g[k], a[k]]
        return np.einsum('eqa,eq->ea', val, w * detJ)

    def element_matrices(self, elems):
        """Element stiffness and mass matrices for element multi-indices elems (nE, dim).

        Returns Ke, Me of shape (nE, nloc, nloc), nloc = (p+1)^dim, with local
        index a = a_1 + a_2 (p+1) + ... (colex) of global function elem + a.
        Ke[a, b] = a(phi_b, phi_a), Me[a, b] = m(phi_b, phi_a).
        """
        elems = np.asarray(elems, dtype=np.int64).reshape(-1, self.dim)
        d, p, nq = self.dim, self.p, self.quad_pts
        tabs = [self._tables_1d(elems[:, k]) for k in range(d)]
        # tensor quadrature points, colex over (g_1, .., g_d)
        gidx = list(itertools.product(range(nq), repeat=d))
        gidx = [tuple(reversed(g)) for g in gidx]
        aidx = [tuple(reversed(a)) for a in itertools.product(range(p + 1), repeat=d)]
        nE, NQ, NL = len(elems), len(gidx), len(aidx)
        s = np.empty((nE, NQ, d))
        w = np.ones((nE, NQ))
        for qi, g in enumerate(gidx):
            for k in range(d):
                s[:, qi, k] = tabs[k][0][:, g[k]]
                w[:, qi] *= tabs[k][1][:, g[k]]
        x, J = self.geometry(s)
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        c2 = self.coef.c2(s, x)
        # G = c^2 det J J^-1 J^-T: grad phi_i^T G grad phi_j is the pulled-back integrand
        Gm = (c2 * detJ)[..., None, None] * np.einsum('eqak,eqbk->eqab', Jinv, Jinv)
        val = np.ones((nE, NQ, NL))
        grad = np.ones((nE, NQ, NL, d))
        for qi, g in enumerate(gidx):
            for ai, a in enumerate(aidx):
                for k in range(d):
                    v = tabs[k][2][:, g[k], a[k]]
                    dv = tabs[k][3][:, g[k], a[k]]
                    val[:, qi, ai] *= v
                    for l in range(d):
                        grad[:, qi, ai, l] *= dv if l == k else v
        Ke = np.einsum('eqak,eqkl,eqbl,eq->eab', grad, Gm, grad, w)
        Me = np.einsum('eqa,eqb,eq->eab', val, val, w * detJ)
        return Ke, Me, np.array(aidx, dtype=np.int64)


def true_rows(space, rows, chunk=4096):
    """Rows of the true K and M in stencil storage (definition of Eq. KeyIdentity).

    rows: (R, dim) multi-indices.  Returns TK, TM of shape (R, D) with
    TK[r, t] = K(i_r, i_r + delta_t).  Each entry is the sum, over every element
    of supp(phi_i), of the element-matrix entry (element-loop assembly).
    """
    rows = np.asarray(rows, dtype=np.int64).reshape(-1, space.dim)
    d, p, ne = space.dim, space.p, space.n_el
    P = 2 * p + 1
    # every (row, support element) pair: element e = i - a with local index a in {0..p}^d
    loc = np.array([tuple(reversed(a)) for a in itertools.product(range(p + 1), repeat=d)],
                   dtype=np.int64)                                   # (nloc, d), colex
    pr_row = np.repeat(np.arange(len(rows)), len(loc))
    pr_a = np.tile(np.arange(len(loc)), len(rows))
    pr_e = rows[pr_row] - loc[pr_a]
    ok = np.all((pr_e >= 0) & (pr_e < ne), axis=1)
    pr_row, pr_a, pr_e = pr_row[ok], pr_a[ok], pr_e[ok]
    e_lin = np.zeros(len(pr_e), dtype=np.int64)
    for k in range(d - 1, -1, -1):
        e_lin = e_lin * ne + pr_e[:, k]
    uniq, pr_ei = np.unique(e_lin, return_inverse=True)
    elems = np.stack([(uniq // ne ** k) % ne for k in range(d)], axis=1)
    nloc = len(loc)
    Ke = np.empty((len(elems), nloc, nloc))
    Me = np.empty((len(elems), nloc, nloc))
    for c0 in range(0, len(elems), chunk):
        k_, m_, _ = space.element_matrices(elems[c0:c0 + chunk])
        Ke[c0:c0 + chunk] = k_
        Me[c0:c0 + chunk] = m_
    TK = np.zeros((len(rows), space.D))
    TM = np.zeros((len(rows), space.D))
    for b in range(nloc):
        # column function e + b, offset delta = e + b - i = b - a
        delta = loc[b][None, :] - loc[pr_a]
        t = np.zeros(len(delta), dtype=np.int64)
        for k in range(d - 1, -1, -1):
            t = t * P + (delta[:, k] + p)
        np.add.at(TK, (pr_row, t), Ke[pr_ei, pr_a, b])
        np.add.at(TM, (pr_row, t), Me[pr_ei, pr_a, b])
    return TK, TM


def stencil_to_csr(space, T, rows=None):
    """Sparse matrix from stencil storage (rows default to all rows, in linear order)."""
    import scipy.sparse as sp
    if rows is None:
        rows = space.all_rows()
    rows = np.asarray(rows)
    dl = space.deltas()
    ii, jj, vv = [], [], []
    for t, delta in enumerate(dl):
        cols = rows + delta[None, :]
        ok = np.all((cols >= 0) & (cols < space.m), axis=1)
        ii.append(space.linear(rows[ok]))
        jj.append(space.linear(cols[ok]))
        vv.append(T[ok, t])
    A = sp.csr_matrix((np.concatenate(vv), (np.concatenate(ii), np.concatenate(jj))),
                      shape=(space.N, space.N))
    return A


def lumped_mass(space, rows):
    """D_ii = integral over Omega of B_i = int_{[0,1]^d} phi_i det J ds (Sec. 3.4,
    remark on volume preservation), by the element Gauss rule of the space summed
    over the elements of supp(phi_i).  rows: (R, dim) multi-indices; returns (R,).
    """
    rows = np.asarray(rows, dtype=np.int64).reshape(-1, space.dim)
    d, p, ne = space.dim, space.p, space.n_el
    loc = np.array([tuple(reversed(a)) for a in itertools.product(range(p + 1), repeat=d)],
                   dtype=np.int64)
    out = np.zeros(len(rows))
    for ai, a in enumerate(loc):
        e = rows - a[None, :]                          # element whose local function a is phi_i
        ok = np.all((e >= 0) & (e < ne), axis=1)
        if ok.any():
            out[ok] += space.element_volumes(e[ok])[:, ai]
    return out
