"""Receiver misfit of the surrogate wave model and its directional derivative (oracle; test infrastructure only).

Misfit over shots s, receivers r and recorded steps n = 1..N (traces of
oracle.wave.Leapfrog):
    J(theta) = dt/2 sum_s sum_r sum_n (d_{s,r}^n(theta) - d_obs_{s,r}^n)^2.
theta are the B-spline coefficients of the wave speed c(s) = sum_k theta_k B_k(s);
only K~ depends on theta (the mass has no coefficient).

Directional derivative J'(theta; v) by forward-mode differentiation of every
step (tangent-linear model):
* K_ij = int c^2 grad phi_i^T G^ grad phi_j is quadratic in theta, so
  dK/dtheta . v is the stiffness assembled with c^2 replaced by 2 c c_v,
  c_v = sum_k v_k B_k;
* the surrogate construction (sample rows, interpolation, mirroring, row-sum
  diagonal; Eq. DefinitionOfSurrogateMatrixSymmetricKernel) is linear in the true
  entries, so dK~/dtheta . v is that construction applied to dK/dtheta . v;
* tangent leapfrog: u'^{n+1} = 2u'^n - u'^{n-1} + dt^2 a'^n, M~ a'^n = -K~' u^n - K~ u'^n,
  first step u'^1 = dt^2/2 a'^0, u'^0 = 0;
* J' = dt sum_s sum_r sum_n (d^n - d_obs^n) d'^n.
"""
import numpy as np

from .assembly import Space, stencil_to_csr
from .geometry import BsplineThetaCoef
from .surrogate import Surrogate
from .wave import Leapfrog, pcg, point_values, ricker


class TangentCoef:
    """'c^2' of the tangent stiffness: 2 c(s) c_v(s) (theta base point, v direction)."""

    def __init__(self, theta, v, deg=3):
        self.c = BsplineThetaCoef(theta, deg)
        self.cv = BsplineThetaCoef(v, deg)

    def c2(self, s, x):
        return 2.0 * self.c.c(s) * self.cv.c(s)


def _space(base, coef):
    return Space(base.dim, base.p, base.n_el, base.geometry, coef, base.quad_pts)


def surrogate_operators(base, theta, q, M, direction=None):
    """(SK, SM) of the surrogate for coefficient theta; with a direction v also SK'."""
    sp = _space(base, BsplineThetaCoef(theta))
    S = Surrogate(sp, q, M)
    SK, SM = S.rows(sp.all_rows())
    if direction is None:
        return SK, SM
    spt = _space(base, TangentCoef(theta, direction))
    St = Surrogate(spt, q, M)
    SKt, _ = St.rows(spt.all_rows())
    return SK, SM, SKt


def misfit(base, theta, q, M, dt, nsteps, sources, receivers, d_obs, rtol=1e-14, max_it=5000):
    """J(theta) and the traces; sources: list of (s_src, f0, t0, amp) (one per shot)."""
    SK, SM = surrogate_operators(base, theta, q, M)
    J = 0.0
    traces = []
    for k, src in enumerate(sources):
        lf = Leapfrog(_space(base, BsplineThetaCoef(theta)), SK, SM, dt, rtol=rtol, max_it=max_it)
        _, _, tr = lf.run(np.zeros(base.N), nsteps, sources=[src], receivers=receivers)
        traces.append(tr)
        J += 0.5 * dt * np.sum((tr - d_obs[k]) ** 2)
    return J, np.array(traces)


def tangent(base, theta, v, q, M, dt, nsteps, sources, receivers, d_obs, rtol=1e-14, max_it=5000):
    """J'(theta; v) by the tangent-linear leapfrog."""
    SK, SM, SKt = surrogate_operators(base, theta, q, M, direction=v)
    K = stencil_to_csr(base, SK)
    Kt = stencil_to_csr(base, SKt)
    Mm = stencil_to_csr(base, SM)
    dinv = 1.0 / Mm.diagonal()
    R = np.array([point_values(base, s) for s in receivers])
    Jp = 0.0
    for k, (s_src, f0, t0, amp) in enumerate(sources):
        bsrc = point_values(base, s_src)
        u = np.zeros(base.N)
        ut = np.zeros(base.N)
        u_prev = ut_prev = None
        a_prev = np.zeros(base.N)
        at_prev = np.zeros(base.N)
        for n in range(nsteps):
            f = amp * ricker(n * dt, f0, t0) * bsrc
            a, _, _ = pcg(Mm, f - K @ u, a_prev, dinv, rtol, max_it)
            at, _, _ = pcg(Mm, -(Kt @ u) - K @ ut, at_prev, dinv, rtol, max_it)
            if n == 0:
                u_new = u + 0.5 * dt * dt * a
                ut_new = ut + 0.5 * dt * dt * at
            else:
                u_new = 2.0 * u - u_prev + dt * dt * a
                ut_new = 2.0 * ut - ut_prev + dt * dt * at
            u_prev, u = u, u_new
            ut_prev, ut = ut, ut_new
            a_prev, at_prev = a, at
            Jp += dt * (R @ u - d_obs[k][:, n]) @ (R @ ut)
    return Jp
