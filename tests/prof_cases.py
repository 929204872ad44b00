"""Small profiling case for ncu (not a test): K~ applies and a short fixed PCG solve on a cube."""
import sys, os, numpy as np, torch
sys.path.insert(0, os.getcwd())
import inputs
from paper_2004_05197_gb300 import iga, workloads as W
n_el = int(sys.argv[1]) if len(sys.argv) > 1 else 80
w = W.scaled("cube96_p2", n_el=n_el)
sp = W.make_space(w)
ops = iga.iga_surrogate_assemble(sp, 2, 2, 6)
N = iga.iga_ops_info_get(ops).N
x = torch.tensor(inputs.vectors(N, 1), dtype=torch.float32, device="cuda")
y = torch.empty_like(x)
for _ in range(2):
    iga.iga_stencil_apply(ops, iga.IGA_OP_K, iga.IGA_F32, x, y, 1)
for _ in range(2):
    a = torch.zeros_like(x)
    iga.iga_mass_solve(ops, iga.IGA_F32, x, a, 1, 0.0, 10)
torch.cuda.synchronize()
print("ok N", N)
