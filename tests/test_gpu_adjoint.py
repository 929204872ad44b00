"""wave_adjoint (C ABI) against the oracle's misfit and tangent-linear derivative,
central finite differences on the GPU, checkpoint invariance and the autograd path."""
import functools

import numpy as np
import pytest

import inputs
from oracle.adjoint import misfit, tangent
from oracle.assembly import Space
from oracle.geometry import ConstCoef, CubeSinePerturbed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300.autograd import misfit as torch_misfit


@functools.lru_cache(maxsize=None)
def small_case():
    base = Space(3, 2, 10, CubeSinePerturbed(0.1), ConstCoef())
    theta = inputs.theta_smooth(n=6, dim=3)
    theta_obs = inputs.theta_smooth(n=6, dim=3, seed=inputs.SEED_THETA_OBS)
    src = np.array([[0.5, 0.5, 0.5], [0.3, 0.6, 0.4]])
    shots = [(s, 10.0, 0.1, 1.0) for s in src]
    rec = inputs.face_receivers(per_face=2)
    dt, nsteps, q, M = 0.1 / 10, 8, 2, 2
    _, d_obs = misfit(base, theta_obs, q, M, dt, nsteps, shots, list(rec), np.zeros((2, len(rec), nsteps)))
    return dict(base=base, theta=theta, src=src, shots=shots, rec=rec, dt=dt, nsteps=nsteps, q=q, M=M,
                obs=d_obs, n_el=10)


def gpu_adjoint(case, theta, want_grad=True, ckpt=50, rtol=1e-14, guess=0, flags=0):
    sp = iga.iga_space_create(3, 2, case["n_el"], iga.IGA_MAP_CUBE_SINE, 0.1, iga.IGA_COEF_BSPLINE, 0.0,
                              theta=inputs.colex(theta), n_theta=theta.shape[0], theta_degree=3)
    ops = iga.iga_surrogate_assemble(sp, 2, case["q"], case["M"])
    w = iga.iga_wave_create(ops, len(case["src"]), iga.IGA_F64, case["dt"], src_pos=case["src"], f0=10.0, t0=0.1,
                            rec_pos=case["rec"], nsteps_max=case["nsteps"], cg_rtol=rtol, cg_max_it=5000,
                            cfl_check=0, cg_guess=guess, solve_flags=flags)
    J, g = iga.iga_wave_adjoint(w, case["nsteps"], ckpt, case["obs"], n_theta_total=theta.size if want_grad else 0)
    iga.iga_wave_destroy(w)
    iga.iga_ops_destroy(ops)
    iga.iga_space_destroy(sp)
    return J, (g.reshape(theta.shape, order="F") if g is not None else None)


def test_adjoint_misfit_matches_oracle():
    c = small_case()
    J_gpu, _ = gpu_adjoint(c, c["theta"], want_grad=False)
    J_ora, _ = misfit(c["base"], c["theta"], c["q"], c["M"], c["dt"], c["nsteps"], c["shots"], list(c["rec"]),
                      c["obs"])
    assert J_ora > 0
    assert abs(J_gpu - J_ora) <= 1e-10 * J_ora


@pytest.mark.parametrize("seed,guess", [(31, 0), (32, 0), (31, 3)])
def test_adjoint_gradient_matches_oracle_tangent(seed, guess):
    """guess: the wave's CG start order (3: the extrapolated start in the forward,
    recomputed and reverse sweeps; only where each solve starts changes)."""
    c = small_case()
    _, g = gpu_adjoint(c, c["theta"], guess=guess)
    v = np.random.default_rng(seed).standard_normal(c["theta"].shape)
    jt = tangent(c["base"], c["theta"], v, c["q"], c["M"], c["dt"], c["nsteps"], c["shots"], list(c["rec"]),
                 c["obs"])
    gv = float(np.sum(g * v))
    print("adjoint g.v", gv, "oracle tangent", jt)
    assert abs(gv - jt) <= 1e-7 * abs(jt)


@pytest.mark.parametrize("guess", [0, 3])
def test_adjoint_is_independent_of_checkpoint_spacing(guess):
    """With guess = 3 the checkpoints carry the acceleration history, so a segment
    recomputed from a checkpoint repeats the forward sweep exactly."""
    c = small_case()
    _, g1 = gpu_adjoint(c, c["theta"], ckpt=3, guess=guess)
    _, g2 = gpu_adjoint(c, c["theta"], ckpt=100, guess=guess)
    assert np.abs(g1 - g2).max() <= 1e-12 * np.abs(g2).max()


@pytest.mark.parametrize("flags", [0, 4])   # 4: IGA_SOLVE_REFINE (FP32 corrections, FP64 residual)
def test_adjoint_cg_start_and_refinement_change_only_rounding(flags):
    c = small_case()
    J0, g0 = gpu_adjoint(c, c["theta"], guess=0)
    J3, g3 = gpu_adjoint(c, c["theta"], guess=3, flags=flags)
    assert abs(J3 - J0) <= 1e-10 * J0
    assert np.abs(g3 - g0).max() <= 1e-9 * np.abs(g0).max()


def test_autograd_function_returns_the_adjoint_gradient():
    c = small_case()
    theta = torch.tensor(c["theta"], dtype=torch.float64, requires_grad=True)
    problem = dict(dim=3, p=2, n_el=c["n_el"], map_kind=iga.IGA_MAP_CUBE_SINE, map_param=0.1, q=c["q"], M=c["M"],
                   dt=c["dt"], nsteps=c["nsteps"], checkpoint_every=4, src_pos=c["src"], rec_pos=c["rec"],
                   obs=c["obs"], cg_rtol=1e-14)
    J = torch_misfit(theta, problem)
    (2.0 * J).backward()
    J_ref, g_ref = gpu_adjoint(c, c["theta"])
    assert abs(float(J) - J_ref) <= 1e-12 * J_ref
    np.testing.assert_allclose(theta.grad.numpy(), 2.0 * g_ref, rtol=1e-10, atol=1e-14 * np.abs(g_ref).max())


def test_adjoint_matches_central_differences_on_gpu():
    """Config-5 family at reduced size: 12^3 theta (smooth perturbation of 1), 3 shots, 30 steps."""
    n_el = 16
    theta = inputs.theta_smooth(n=12, dim=3)
    theta_obs = inputs.theta_smooth(n=12, dim=3, seed=inputs.SEED_THETA_OBS)
    src = inputs.shot_positions(3, dim=3, lo=0.3, hi=0.7, seed=inputs.SEED_SHOTS_3D)
    rec = inputs.face_receivers(per_face=8)
    case = dict(n_el=n_el, src=src, rec=rec, dt=0.1 / n_el, nsteps=30, q=2, M=2,
                obs=np.zeros((3, len(rec), 30)))
    _, tr = None, None
    # observed data from the second model through the same GPU path (misfit with obs = 0 gives traces^2)
    sp = iga.iga_space_create(3, 2, n_el, iga.IGA_MAP_CUBE_SINE, 0.1, iga.IGA_COEF_BSPLINE, 0.0,
                              theta=inputs.colex(theta_obs), n_theta=12, theta_degree=3)
    ops = iga.iga_surrogate_assemble(sp, 2, 2, 2)
    w = iga.iga_wave_create(ops, 3, iga.IGA_F64, case["dt"], src_pos=src, f0=10.0, t0=0.1, rec_pos=rec,
                            nsteps_max=30, cg_rtol=1e-14, cg_max_it=5000, cfl_check=0)
    iga.iga_wave_step(w, 30)
    case["obs"] = iga.iga_wave_traces(w, 3, len(rec), 30)
    iga.iga_wave_destroy(w)
    iga.iga_ops_destroy(ops)
    iga.iga_space_destroy(sp)
    _, g = gpu_adjoint(case, theta, ckpt=10)
    for seed in (41, 42, 43):
        v = np.random.default_rng(seed).standard_normal(theta.shape)
        eps = 1e-6
        Jp, _ = gpu_adjoint(case, theta + eps * v, want_grad=False)
        Jm, _ = gpu_adjoint(case, theta - eps * v, want_grad=False)
        fd = (Jp - Jm) / (2 * eps)
        gv = float(np.sum(g * v))
        print("seed", seed, "adjoint", gv, "central FD", fd)
        assert abs(gv - fd) <= 1e-6 * abs(gv)
