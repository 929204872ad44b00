"""Synthetic workloads shaped like the paper's problems, as plain parameter sets.

A workload names the space (dimension, degree, elements, geometry map,
wave-speed coefficient), the surrogate parameters (q, M) and the time stepping.
``make_space`` / ``make_ops`` build it on the GPU through the C ABI; the seeded
random inputs come from the ``inputs`` package.

Workloads (sizes of the benchmark problems):
  annulus64_p2   2-D p=2, 64^2 elements, quarter annulus, c = 1, q=2, M=4, dt = 0.2 h,
                 Gaussian pulse of width 0.05, 20 steps (FP64)
  annulus512_p3  2-D p=3, 512^2, quarter annulus, c = 1 + 0.5 sin(2 pi x) cos(2 pi y),
                 q=3, M=8, Ricker f0 = 10 at s = (0.5, 0.5), 2000 steps, CG tol 1e-10,
                 dt = 0.1 h (0.2 h exceeds the leapfrog stability limit, about 0.19 h)
  cube96_p2      3-D p=2, 96^3, sine-perturbed cube (amplitude 0.1), lognormal
                 (sigma 0.3) wave speed on a 16^3 cubic B-spline grid, q=2, M=6,
                 Ricker source at the cube centre, 500 FP32 steps, dt = 0.1 h (0.2 h exceeds
                 the leapfrog stability limit, about 0.19 h and falling with n_el)
"""
import numpy as np

import inputs

WORKLOADS = {
    "annulus64_p2": dict(dim=2, p=2, n_el=64, map="annulus", coef="const", q=2, M=4, steps=20,
                         source=False, pulse=True, dt_factor=0.2),
    "annulus512_p3": dict(dim=2, p=3, n_el=512, map="annulus", coef="sincos", q=3, M=8, steps=2000,
                          source=True, pulse=False, dt_factor=0.1),
    "cube96_p2": dict(dim=3, p=2, n_el=96, map="cube", coef="theta16", q=2, M=6, steps=500,
                      source=True, pulse=False, dt_factor=0.1),
}


def scaled(name, **over):
    """A copy of a named workload with some parameters replaced (e.g. smaller n_el)."""
    w = dict(WORKLOADS[name])
    w.update(over)
    return w


def theta_for(w):
    """Seeded theta coefficients (array [k_1, .., k_d]) for a B-spline coefficient, else None."""
    if w["coef"] == "theta16":
        return inputs.theta_lognormal(n=16, dim=w["dim"], sigma=0.3)
    if w["coef"] == "theta12":
        return inputs.theta_smooth(n=12, dim=w["dim"])
    return None


def make_space(w):
    from . import iga
    mk = {"annulus": iga.IGA_MAP_ANNULUS_QUARTER, "cube": iga.IGA_MAP_CUBE_SINE,
          "identity": iga.IGA_MAP_IDENTITY}[w["map"]]
    mp = 0.1 if w["map"] == "cube" else 0.0
    theta = theta_for(w)
    if w["coef"] == "const":
        return iga.iga_space_create(w["dim"], w["p"], w["n_el"], mk, mp, iga.IGA_COEF_CONST, 1.0)
    if w["coef"] == "sincos":
        return iga.iga_space_create(w["dim"], w["p"], w["n_el"], mk, mp, iga.IGA_COEF_SINCOS, 0.5)
    return iga.iga_space_create(w["dim"], w["p"], w["n_el"], mk, mp, iga.IGA_COEF_BSPLINE, 0.0,
                                theta=inputs.colex(theta), n_theta=theta.shape[0], theta_degree=3)


def source_position(w):
    return np.full(w["dim"], 0.5)


def dt_of(w):
    return w["dt_factor"] / w["n_el"]
