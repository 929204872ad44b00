"""Geometry maps F: [0,1]^d -> Omega and wave-speed coefficients (oracle; test infrastructure only).

The weak forms of Eq. weakforms are pulled back to the parametric domain with
the Jacobian J of the map; the acoustic energy of Eq. LinearWaveEnergy weights
the stiffness by c^2.  Maps and coefficients here are the smooth analytic ones
of the synthetic workloads (a smooth map is the paper's requirement in
Sec. 3.5 for smooth stencil functions).

Every map returns, for parametric points s of shape (..., d), the physical
points x (..., d) and the Jacobian J[..., a, b] = dx_a / ds_b.
"""
import numpy as np

from .bspline import collocation, open_uniform_knots


class IdentityMap:
    def __init__(self, dim):
        self.dim = dim

    def __call__(self, s):
        s = np.asarray(s, dtype=np.float64)
        J = np.broadcast_to(np.eye(self.dim), s.shape + (self.dim,)).copy()
        return s.copy(), J


class AnnulusQuarter:
    """F(s,t) = ((1+s) cos(pi t/2), (1+s) sin(pi t/2)): quarter annulus 1 < |x| < 2."""
    dim = 2

    def __call__(self, s):
        s = np.asarray(s, dtype=np.float64)
        r = 1.0 + s[..., 0]
        a = 0.5 * np.pi * s[..., 1]
        x = np.stack([r * np.cos(a), r * np.sin(a)], axis=-1)
        J = np.empty(s.shape + (2,))
        J[..., 0, 0] = np.cos(a)
        J[..., 0, 1] = -r * 0.5 * np.pi * np.sin(a)
        J[..., 1, 0] = np.sin(a)
        J[..., 1, 1] = r * 0.5 * np.pi * np.cos(a)
        return x, J


class AnnulusSector:
    """F(s,t) = (r cos a, r sin a), r = r0 + (r1 - r0) s, a = a0 + (a1 - a0) t: one patch of
    an annulus split into sectors (multi-patch remark of Sec. 3.2); r0 = 1, r1 = 2, a0 = 0,
    a1 = pi/2 is the quarter annulus."""
    dim = 2

    def __init__(self, r0=1.0, r1=2.0, a0=0.0, a1=0.5 * np.pi):
        self.r0, self.r1, self.a0, self.a1 = r0, r1, a0, a1

    def __call__(self, s):
        s = np.asarray(s, dtype=np.float64)
        dr, da = self.r1 - self.r0, self.a1 - self.a0
        r = self.r0 + dr * s[..., 0]
        a = self.a0 + da * s[..., 1]
        x = np.stack([r * np.cos(a), r * np.sin(a)], axis=-1)
        J = np.empty(s.shape + (2,))
        J[..., 0, 0] = dr * np.cos(a)
        J[..., 0, 1] = -r * da * np.sin(a)
        J[..., 1, 0] = dr * np.sin(a)
        J[..., 1, 1] = r * da * np.cos(a)
        return x, J


class BoxMap:
    """x_k = o_k + e_k s_k: an axis-aligned box, one patch of a multi-patch brick (the
    multi-patch remark of Sec. 3.2 in three dimensions); J = diag(e).  A negative e_k
    runs the parametric direction against the physical one (det J = prod e_k > 0)."""

    def __init__(self, origin, extent):
        self.origin = np.asarray(origin, dtype=np.float64)
        self.extent = np.asarray(extent, dtype=np.float64)
        self.dim = len(self.origin)

    def __call__(self, s):
        s = np.asarray(s, dtype=np.float64)
        x = self.origin + self.extent * s
        J = np.zeros(s.shape + (self.dim,))
        for k in range(self.dim):
            J[..., k, k] = self.extent[k]
        return x, J


class CubeSinePerturbed:
    """x_k = s_k + eps * sin(pi s) sin(pi t) sin(pi u) for each coordinate k (unit cube)."""
    dim = 3

    def __init__(self, eps=0.1):
        self.eps = eps

    def __call__(self, s):
        s = np.asarray(s, dtype=np.float64)
        sn = np.sin(np.pi * s)
        cs = np.cos(np.pi * s)
        g = sn[..., 0] * sn[..., 1] * sn[..., 2]
        grad = np.stack([np.pi * cs[..., 0] * sn[..., 1] * sn[..., 2],
                         np.pi * sn[..., 0] * cs[..., 1] * sn[..., 2],
                         np.pi * sn[..., 0] * sn[..., 1] * cs[..., 2]], axis=-1)
        x = s + self.eps * g[..., None]
        J = np.broadcast_to(np.eye(3), s.shape + (3,)).copy()
        J += self.eps * grad[..., None, :]   # every row of J gets eps * grad g
        return x, J


class ConstCoef:
    def __init__(self, c=1.0):
        self.c = float(c)

    def c2(self, s, x):
        return np.full(s.shape[:-1], self.c * self.c)


class SinCosCoef:
    """c(x) = 1 + a sin(2 pi x) cos(2 pi y), evaluated at the physical point x = F(s)."""

    def __init__(self, a=0.5):
        self.a = a

    def c2(self, s, x):
        c = 1.0 + self.a * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])
        return c * c


class BsplineThetaCoef:
    """c(s) = sum_k theta_k B_k(s): tensor B-spline of degree `deg` on the parametric cube.

    theta has shape (n_1, ..., n_d) indexed [k_1, ..., k_d] (k_1 = first parametric
    direction); each direction uses an open uniform knot vector with n_j - deg
    elements.
    """

    def __init__(self, theta, deg=3):
        self.theta = np.asarray(theta, dtype=np.float64)
        self.deg = deg
        self.knots = [open_uniform_knots(n - deg, deg) for n in self.theta.shape]

    def c(self, s):
        s = np.asarray(s, dtype=np.float64)
        flat = s.reshape(-1, s.shape[-1])
        d = flat.shape[1]
        mats = [collocation(self.knots[k], self.deg, flat[:, k]) for k in range(d)]
        if d == 2:
            val = np.einsum('ra,rb,ab->r', mats[0], mats[1], self.theta)
        else:
            val = np.einsum('ra,rb,rc,abc->r', mats[0], mats[1], mats[2], self.theta)
        return val.reshape(s.shape[:-1])

    def c2(self, s, x):
        c = self.c(s)
        return c * c
