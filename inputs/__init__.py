"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module draws random numbers only; it holds none of the method's
arithmetic.  Every array is produced by numpy's PCG64 generator
(``numpy.random.default_rng(seed)``) with a fixed seed per quantity, so both
sides of a parity test receive identical inputs.

Layout convention: arrays over a tensor grid are returned with index
[k_1, ..., k_d] (first parametric direction first); ``colex`` flattens them
with k_1 fastest, the order the C ABI expects.
"""
import numpy as np

SEED_PULSE = 1
SEED_THETA_LOGNORMAL = 2
SEED_SHOTS_2D = 3
SEED_THETA_SMOOTH = 4
SEED_RECEIVERS = 5
SEED_THETA_OBS = 6
SEED_SHOTS_3D = 7
SEED_VECTORS = 11


def colex(a):
    """Flatten a [k_1, .., k_d] array with k_1 fastest (colexicographic order)."""
    return np.ascontiguousarray(np.asarray(a).ravel(order='F'))


def pulse_centre(dim=2, seed=SEED_PULSE):
    """Parametric centre of the initial Gaussian pulse, uniform in [0.25, 0.75]^dim."""
    return np.random.default_rng(seed).uniform(0.25, 0.75, size=dim)


def theta_lognormal(n=16, dim=3, sigma=0.3, seed=SEED_THETA_LOGNORMAL):
    """Wave-speed B-spline coefficients theta = exp(sigma z), z iid N(0,1), shape (n,)*dim."""
    z = np.random.default_rng(seed).standard_normal((n,) * dim)
    return np.exp(sigma * z)


def theta_smooth(n=12, dim=3, amp=0.05, seed=SEED_THETA_SMOOTH):
    """theta = 1 + amp z with z iid N(0,1) clipped to [-3, 3], shape (n,)*dim."""
    z = np.clip(np.random.default_rng(seed).standard_normal((n,) * dim), -3.0, 3.0)
    return 1.0 + amp * z


def shot_positions(nshot, dim=2, lo=0.1, hi=0.9, seed=SEED_SHOTS_2D):
    """Parametric source positions, uniform in [lo, hi]^dim, shape (nshot, dim)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=(nshot, dim))


def face_receivers(per_face=32, seed=SEED_RECEIVERS):
    """Receivers on the 6 faces of the parametric unit cube, shape (6*per_face, 3).

    On each face the two free coordinates are uniform in [0.05, 0.95].
    """
    rng = np.random.default_rng(seed)
    out = []
    for axis in range(3):
        for side in (0.0, 1.0):
            uv = rng.uniform(0.05, 0.95, size=(per_face, 2))
            pts = np.empty((per_face, 3))
            free = [k for k in range(3) if k != axis]
            pts[:, free[0]] = uv[:, 0]
            pts[:, free[1]] = uv[:, 1]
            pts[:, axis] = side
            out.append(pts)
    return np.concatenate(out)


def vectors(n, nrhs=1, seed=SEED_VECTORS):
    """Random test vectors, uniform in [-1, 1], shape (nrhs, n)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(nrhs, n))
