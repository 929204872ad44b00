"""Consistent-mass Jacobi-PCG and leapfrog time stepping (oracle; test infrastructure only).

The paper's acoustic model (Eq. GeneralSystem with the energy of
Eq. LinearWaveEnergy, unit density, homogeneous Neumann data on the whole
boundary) discretised with the surrogate matrices gives M~ u'' + K~ u = f
(Eq. SurrogateEoMSurrogate without the time-harmonic terms; Sec. 4.6 discusses
time stepping with surrogate matrices).  The time integrator, source and
receiver model are the workload's:

* leapfrog  u^{n+1} = 2 u^n - u^{n-1} + dt^2 a^n,  M~ a^n = f^n - K~ u^n,
  started by the second-order Taylor step u^1 = u^0 + dt v^0 + dt^2/2 a^0;
* a^n by Jacobi-preconditioned CG on M~ with initial guess a^{n-1} (0 at n = 0),
  stopping when ||r_k||_2 <= rtol ||b||_2 or after max_it iterations
  (rtol = 0 runs exactly max_it iterations);
* Ricker point source f_i^n = r(t_n) B_i(s_src), r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2)
  exp(-pi^2 f0^2 (t-t0)^2), t_n = n dt;
* Gaussian initial pulse u^0_i = exp(-|F(gamma_i) - x_c|^2 / (2 w^2)) at the
  Greville points gamma_i, v^0 = 0;
* receiver traces d_r^n = sum_i u_i^n B_i(s_r), recorded for n = 1..nsteps.
"""
from math import comb

import numpy as np
import scipy.sparse as sps

from .assembly import stencil_to_csr
from .bspline import collocation, greville


def pcg(A, b, x0, dinv, rtol, max_it):
    """Jacobi-PCG for SPD A.  Returns (x, iterations, ||r||/||b||)."""
    x = x0.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - A @ x
    z = dinv * r
    pvec = z.copy()
    rz = r @ z
    it = 0
    while it < max_it:
        if rtol > 0 and np.linalg.norm(r) <= rtol * bn:
            break
        q = A @ pvec
        alpha = rz / (pvec @ q)
        x += alpha * pvec
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        pvec = z + beta * pvec
        it += 1
    return x, it, np.linalg.norm(r) / bn


def ricker(t, f0, t0):
    a = (np.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def point_values(space, s):
    """Vector B_i(s) over all global basis functions for one parametric point s (dim,)."""
    vals = [collocation(space.knots, space.p, [s[k]])[0] for k in range(space.dim)]
    out = vals[0]
    for k in range(1, space.dim):
        out = np.multiply.outer(vals[k], out).ravel()        # colex: earlier dims fastest
    return out


def gaussian_pulse(space, xc, width):
    """u^0_i = g(F(gamma_i)) with g(x) = exp(-|x - xc|^2 / (2 width^2))."""
    gam = greville(space.knots, space.p)
    rows = space.all_rows()
    s = gam[rows]
    x, _ = space.geometry(s)
    return np.exp(-np.sum((x - np.asarray(xc)) ** 2, axis=-1) / (2.0 * width ** 2))


def cg_start(hist, order, n):
    """Start of step n's mass solve from the accelerations of the earlier steps,
    hist = [a^{n-1}, a^{n-2}, ...] (most recent first, as many as exist): zero
    before the first step, else the value one step ahead of the polynomial of
    degree k = min(order, len(hist) - 1) through the last k + 1 accelerations,
    sum_{j=0..k} (-1)^j C(k+1, j+1) a^{n-1-j} (Newton's backward differences:
    degree 0: a^{n-1}; 1: 2a^{n-1} - a^{n-2}; 2: 3a^{n-1} - 3a^{n-2} + a^{n-3}).
    The starting point is not part of the time-stepping scheme: every solve
    still runs to its tolerance."""
    if not hist:
        return np.zeros(n)
    k = min(order, len(hist) - 1)
    out = np.zeros(n)
    for j in range(k + 1):
        out += (-1) ** j * comb(k + 1, j + 1) * hist[j]
    return out


class Leapfrog:
    """Leapfrog on the (surrogate) stencil matrices SK, SM given for all rows."""

    def __init__(self, space, SK, SM, dt, rtol=1e-10, max_it=1000, guess_order=0):
        self.space = space
        self.guess_order = guess_order
        self.K = stencil_to_csr(space, SK)
        self.M = stencil_to_csr(space, SM)
        self.dinv = 1.0 / self.M.diagonal()
        self.dt = dt
        self.rtol, self.max_it = rtol, max_it
        self.iters = []

    def run(self, u0, nsteps, v0=None, sources=(), receivers=()):
        """sources: list of (s_src, f0, t0, amplitude); receivers: list of s_r.

        Returns (u^{nsteps}, u^{nsteps-1}, traces[nrec, nsteps]).
        """
        sp, dt = self.space, self.dt
        svec = [(point_values(sp, s), f0, t0, amp) for (s, f0, t0, amp) in sources]
        rvec = np.array([point_values(sp, s) for s in receivers]).reshape(len(receivers), sp.N)
        u = np.asarray(u0, dtype=np.float64).copy()
        v = np.zeros_like(u) if v0 is None else np.asarray(v0, dtype=np.float64)
        hist = []                   # a^{n-1}, a^{n-2}, a^{n-3} (most recent first)
        u_prev = None
        traces = np.zeros((len(receivers), nsteps))
        for n in range(nsteps):
            t = n * dt
            f = np.zeros(sp.N)
            for bvec, f0, t0, amp in svec:
                f += amp * ricker(t, f0, t0) * bvec
            b = f - self.K @ u
            a, it, _ = pcg(self.M, b, cg_start(hist, self.guess_order, sp.N), self.dinv, self.rtol, self.max_it)
            self.iters.append(it)
            if n == 0:
                u_new = u + dt * v + 0.5 * dt * dt * a
            else:
                u_new = 2.0 * u - u_prev + dt * dt * a
            u_prev, u = u, u_new
            hist = [a] + hist[:self.guess_order]
            if len(receivers):
                traces[:, n] = rvec @ u
        return u, u_prev, traces

    def energy(self, u_prev, u):
        """Discrete leapfrog energy between levels n and n+1 (conserved for f = 0)."""
        du = (u - u_prev) / self.dt
        return 0.5 * du @ (self.M @ du) + 0.5 * u_prev @ (self.K @ u)
