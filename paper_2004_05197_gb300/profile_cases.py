"""Small profiling cases for ncu.

    python -m paper_2004_05197_gb300.profile_cases [n_el]
    python -m paper_2004_05197_gb300.profile_cases assemble [n_el]
    python -m paper_2004_05197_gb300.profile_cases apply [n_el]

Workload: the cube96_p2 family at n_el (default 80: the FP32 fields exceed L2).
Default case, launch order: two K~ applies, then persistent PCG solves of exactly
10, 10 and 20 iterations (rtol 0), so that a capture of the last two separates the
per-solve and per-iteration DRAM traffic.  `assemble`: one surrogate assembly of
the space (band quadrature, sample rows, interpolation, evaluation).  `apply`
(default n_el 96): FP32 K~ then M~ applies, two launches each, first with the
brick kernels, then with the row kernels.
"""
import sys

import torch

import inputs
from paper_2004_05197_gb300 import iga
from paper_2004_05197_gb300 import workloads as W


def main(n_el=80):
    w = W.scaled("cube96_p2", n_el=n_el)
    sp = W.make_space(w)
    ops = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
    N = iga.iga_ops_info_get(ops).N
    x = torch.tensor(inputs.vectors(N, 1), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for _ in range(2):
        iga.iga_stencil_apply(ops, iga.IGA_OP_K, iga.IGA_F32, x, y, 1)
    for its in (10, 10, 20):
        a = torch.zeros_like(x)
        iga.iga_mass_solve(ops, iga.IGA_F32, x, a, 1, 0.0, its)
    torch.cuda.synchronize()
    print("ok N", N)


def assemble(n_el=40):
    w = W.scaled("cube96_p2", n_el=n_el)
    sp = W.make_space(w)
    ops = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
    torch.cuda.synchronize()
    print("ok N", iga.iga_ops_info_get(ops).N, "band ms", iga.iga_ops_info_get(ops).t_band_ms)


def applies(n_el=96):
    w = W.scaled("cube96_p2", n_el=n_el)
    sp = W.make_space(w)
    ops = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
    N = iga.iga_ops_info_get(ops).N
    x = torch.tensor(inputs.vectors(N, 1), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for path in (iga.IGA_PATH_BRICK, iga.IGA_PATH_ROWS):
        iga.iga_ops_set_path(ops, path)
        for which in (iga.IGA_OP_K, iga.IGA_OP_M):
            for _ in range(2):
                iga.iga_stencil_apply(ops, which, iga.IGA_F32, x, y, 1)
    torch.cuda.synchronize()
    print("ok N", N, "bricks", iga.iga_ops_brick_info(ops))


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "apply":
        applies(int(sys.argv[2]) if len(sys.argv) > 2 else 96)
    elif len(sys.argv) > 1 and sys.argv[1] == "assemble":
        assemble(int(sys.argv[2]) if len(sys.argv) > 2 else 40)
    else:
        main(int(sys.argv[1]) if len(sys.argv) > 1 else 80)
