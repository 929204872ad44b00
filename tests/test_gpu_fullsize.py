"""Parity at the full sizes of the benchmark workloads (3-D p = 2, 96^3 elements,
941,192 rows; 2-D p = 3, 512^2 elements, 265,225 rows) in the launch configuration
bench.py uses, on sampled outputs the oracle computes one by one:

* surrogate fields (FP64) of a seeded sample of rows -- interior, sample and band
  rows -- against the oracle's surrogate rows, 1e-12 relative to the largest entry;
* K~ x and M~ x at those rows, FP64 to 1e-12 and FP32 to 2e-5 of the |A| |x| row
  scale, from the oracle's full stencil rows;
* the persistent FP32 mass solve of the bench: its true residual, recomputed by the
  FP64 apply, meets the requested tolerance (a property that holds at any size).

The oracle's sample-row quadrature (4,096 rows per workload) runs on a pool of
processes started with spawn.
"""
import concurrent.futures as cf
import functools
import multiprocessing as mp
import os

import numpy as np
import pytest

import inputs
from oracle.surrogate import Surrogate, interior_range
from tests.oracle_cases import oracle_space

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

NAMES = ["cube96_p2", "annulus512_p3"]


@functools.lru_cache(maxsize=None)
def pool():
    return cf.ProcessPoolExecutor(max(1, min(16, os.cpu_count() or 1)), mp_context=mp.get_context("spawn"))


def _rows(args):
    S, rows = args
    return S.rows(rows)


def sampled_rows(sp, S, seed=123):
    """Seeded rows: 96 uniform, 32 on the sampling lattice, 32 outside Omega~."""
    rng = np.random.default_rng(seed)
    uni = sp.multi(rng.integers(0, sp.N, size=96))
    samp = S.samp
    lat = np.stack([rng.choice(samp, 32) for _ in range(sp.dim)], axis=1)
    lo, hi = interior_range(sp.m, sp.p)
    band = rng.integers(0, sp.m, size=(32, sp.dim))
    band[:, 0] = rng.choice(np.r_[0:lo, hi + 1:sp.m], 32)
    return np.concatenate([uni, lat, band])


@functools.lru_cache(maxsize=None)
def oracle_case(name):
    w = W.scaled(name)
    sp = oracle_space(w)
    S = Surrogate(sp, w["q"], w["M"], pool=pool())
    rows = sampled_rows(sp, S)
    parts = np.array_split(rows, 16)
    out = list(pool().map(_rows, [(S, p) for p in parts]))
    SK = np.concatenate([o[0] for o in out])
    SM = np.concatenate([o[1] for o in out])
    return sp, rows, SK, SM


@functools.lru_cache(maxsize=None)
def gpu_case(name):
    w = W.scaled(name)
    space = W.make_space(w)
    ops = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], 0)
    return space, ops


def fields_at(ops, which, dtype, lin):
    info = iga.iga_ops_info_get(ops)
    nf = info.nK if which == iga.IGA_OP_K else info.nM
    t = torch.empty((nf, info.N), dtype=torch.float64 if dtype == iga.IGA_F64 else torch.float32, device="cuda")
    iga.iga_ops_copy_fields(ops, which, dtype, t)
    out = t[:, torch.tensor(lin, device="cuda")].double().cpu().numpy()
    del t
    return out


@pytest.mark.parametrize("name", NAMES)
def test_fullsize_fields_at_sampled_rows(name):
    sp, rows, SK, SM = oracle_case(name)
    _, ops = gpu_case(name)
    lin = sp.linear(rows)
    t0 = (sp.D - 1) // 2
    gK = fields_at(ops, iga.IGA_OP_K, iga.IGA_F64, lin)
    gM = fields_at(ops, iga.IGA_OP_M, iga.IGA_F64, lin)
    oK, oM = SK[:, t0 + 1:].T, SM[:, t0:].T
    assert np.array_equal(gK == 0.0, oK == 0.0) and np.array_equal(gM == 0.0, oM == 0.0)
    assert np.abs(gK - oK).max() <= 1e-12 * np.abs(oK).max()
    assert np.abs(gM - oM).max() <= 1e-12 * np.abs(oM).max()


@pytest.mark.parametrize("name", NAMES)
def test_fullsize_applies_at_sampled_rows(name):
    sp, rows, SK, SM = oracle_case(name)
    _, ops = gpu_case(name)
    x = inputs.vectors(sp.N, 1)[0]
    nb = rows[:, None, :] + sp.deltas()[None, :, :]                       # (R, D, dim)
    inside = np.all((nb >= 0) & (nb < sp.m), axis=2)
    xn = np.where(inside, x[sp.linear(np.clip(nb, 0, sp.m - 1))], 0.0)
    lin = sp.linear(rows)
    for which, T in ((iga.IGA_OP_K, SK), (iga.IGA_OP_M, SM)):
        ref = np.sum(T * xn, axis=1)
        scale = np.sum(np.abs(T) * np.abs(xn), axis=1)
        for dtype, tol in ((iga.IGA_F64, 1e-12), (iga.IGA_F32, 2e-5)):
            tdt = torch.float64 if dtype == iga.IGA_F64 else torch.float32
            xg = torch.tensor(x[None], dtype=tdt, device="cuda")
            yg = torch.empty_like(xg)
            iga.iga_stencil_apply(ops, which, dtype, xg, yg, 1)
            got = yg[0, torch.tensor(lin, device="cuda")].double().cpu().numpy()
            assert np.all(np.abs(got - ref) <= tol * scale.max()), (which, dtype, np.abs(got - ref).max() / scale.max())


@pytest.mark.parametrize("name", NAMES)
def test_fullsize_mass_solve_residual(name):
    """The bench's FP32 persistent solve (rtol 1e-6) and an FP64 solve (rtol 1e-12): the
    residual b - M~ a recomputed with the FP64 fields meets the tolerance (FP32: up to the
    FP32 representation of M~ and a, bounded by about cond(M~) 2^-24)."""
    _, ops = gpu_case(name)
    N = iga.iga_ops_info_get(ops).N
    b = torch.tensor(inputs.vectors(N, 1), device="cuda")
    for dtype, rtol, bound in ((iga.IGA_F32, 1e-6, 5e-5), (iga.IGA_F64, 1e-12, 1e-11)):
        tdt = torch.float64 if dtype == iga.IGA_F64 else torch.float32
        a = torch.zeros((1, N), dtype=tdt, device="cuda")
        _, iters, rel = iga.iga_mass_solve(ops, dtype, b.to(tdt), a, 1, rtol, 5000)
        r = torch.empty_like(b)
        iga.iga_stencil_apply(ops, iga.IGA_OP_M, iga.IGA_F64, a.double(), r, 1)
        res = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
        assert rel[0] <= rtol and res <= bound, (dtype, rel[0], res)
