"""torch.autograd.Function for the receiver misfit J(theta) of the surrogate wave model.

Forward and backward both cross the C ABI once: the forward evaluates J through
`iga_wave_adjoint` (which also produces the gradient by the discrete adjoint,
with checkpoints), the backward scales the stored gradient by the incoming
gradient.  theta are the wave-speed B-spline coefficients, shape (n,)*dim,
indexed [k_1, .., k_d].
"""
import numpy as np
import torch

from . import iga


class SurrogateWaveMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, problem):
        """problem: dict(dim, p, n_el, map_kind, map_param, q, M, dt, nsteps, checkpoint_every,
        src_pos [nshot][dim], rec_pos [nrec][dim], obs [nshot][nrec][nsteps], f0, t0, cg_rtol)."""
        th = theta.detach().to("cpu", torch.float64).numpy()
        flat = np.ascontiguousarray(th.ravel(order="F"))
        space = iga.iga_space_create(problem["dim"], problem["p"], problem["n_el"], problem["map_kind"],
                                     problem.get("map_param", 0.0), iga.IGA_COEF_BSPLINE, 0.0, theta=flat,
                                     n_theta=th.shape[0], theta_degree=3)
        ops = iga.iga_surrogate_assemble(space, problem["p"], problem["q"], problem["M"])
        nsteps = problem["nsteps"]
        src = np.asarray(problem["src_pos"], dtype=np.float64)
        wave = iga.iga_wave_create(ops, src.shape[0], iga.IGA_F64, problem["dt"], src_pos=src,
                                   f0=problem.get("f0", 10.0), t0=problem.get("t0", 0.1),
                                   rec_pos=problem["rec_pos"], nsteps_max=nsteps,
                                   cg_rtol=problem.get("cg_rtol", 1e-13), cg_max_it=problem.get("cg_max_it", 5000),
                                   cfl_check=0, cg_guess=problem.get("cg_guess", 0),
                                   solve_flags=problem.get("solve_flags", 0))
        want = ctx.needs_input_grad[0]
        J, g = iga.iga_wave_adjoint(wave, nsteps, problem.get("checkpoint_every", 50), problem["obs"],
                                    n_theta_total=flat.size if want else 0)
        iga.iga_wave_destroy(wave)
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(space)
        if want:
            grad = torch.from_numpy(g.reshape(th.shape, order="F").copy()).to(theta.device, theta.dtype)
            ctx.save_for_backward(grad)
        return torch.tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return gJ * grad, None


def misfit(theta, problem):
    return SurrogateWaveMisfit.apply(theta, problem)
