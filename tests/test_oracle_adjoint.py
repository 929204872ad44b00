"""Pin of the oracle's directional derivative of the receiver misfit (CPU only).

The tangent-linear leapfrog J'(theta; v) must match central finite differences
of the oracle's own J(theta) (an independent route: only J is evaluated).
"""
import numpy as np
import pytest

import inputs
from oracle.adjoint import misfit, tangent
from oracle.assembly import Space
from oracle.geometry import ConstCoef, CubeSinePerturbed


def _case():
    base = Space(3, 2, 10, CubeSinePerturbed(0.1), ConstCoef())
    theta = inputs.theta_smooth(n=6, dim=3)
    theta_obs = inputs.theta_smooth(n=6, dim=3, seed=inputs.SEED_THETA_OBS)
    shots = [(np.array([0.5, 0.5, 0.5]), 10.0, 0.1, 1.0), (np.array([0.3, 0.6, 0.4]), 10.0, 0.1, 1.0)]
    rec = list(inputs.face_receivers(per_face=2))
    dt, nsteps, q, M = 0.1 / 10, 8, 2, 2
    _, d_obs = misfit(base, theta_obs, q, M, dt, nsteps, shots, rec, np.zeros((2, len(rec), nsteps)))
    return base, theta, shots, rec, dt, nsteps, q, M, d_obs


@pytest.mark.parametrize("seed", [21, 22])
def test_tangent_matches_central_differences(seed):
    base, theta, shots, rec, dt, nsteps, q, M, d_obs = _case()
    v = np.random.default_rng(seed).standard_normal(theta.shape)
    Jp = tangent(base, theta, v, q, M, dt, nsteps, shots, rec, d_obs)
    eps = 1e-6
    Jplus, _ = misfit(base, theta + eps * v, q, M, dt, nsteps, shots, rec, d_obs)
    Jminus, _ = misfit(base, theta - eps * v, q, M, dt, nsteps, shots, rec, d_obs)
    fd = (Jplus - Jminus) / (2 * eps)
    assert abs(Jp) > 0
    assert abs(Jp - fd) <= 1e-6 * abs(Jp), (Jp, fd)


def test_misfit_vanishes_at_the_observation_model():
    base, theta, shots, rec, dt, nsteps, q, M, d_obs = _case()
    theta_obs = inputs.theta_smooth(n=6, dim=3, seed=inputs.SEED_THETA_OBS)
    J, _ = misfit(base, theta_obs, q, M, dt, nsteps, shots, rec, d_obs)
    assert J == 0.0
