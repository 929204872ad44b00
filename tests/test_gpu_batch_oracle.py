"""Batched persistent stepping and single-shot FP64 waves against the FP64 oracle
leapfrog, on the mesh family of the batched workload (2-D p = 3 quarter annulus,
c = 1 + 0.5 sin(2 pi x) cos(2 pi y), q = 3, Ricker shots at seeded positions).

* iga_batch_step, two meshes of different size x 4 shots, FP32 (compensated state,
  FP64 residual): every shot's state and traces against the oracle run of that shot at
  the FP32 bar 2e-5 (relative L2 for the state; traces on the field's scale).
* FP64 single-shot waves, persistent and plain CG schedules: 1e-11 against the oracle,
  so that the FP64 GPU wave the bench uses as the reference of the batched FP32 error
  is itself pinned on this family.
"""
import functools

import numpy as np
import pytest

import inputs
from oracle.wave import Leapfrog
from tests.oracle_cases import oracle_surrogate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

SIZES = (16, 22)
NSHOT = 4
NSTEPS = 40
REC = np.array([[0.5, 0.5], [0.25, 0.75], [0.8, 0.3]])


def _w(n):
    return W.scaled("annulus512_p3", n_el=n, M=2)


@functools.lru_cache(maxsize=None)
def _oracle(n):
    w = _w(n)
    sp, S = oracle_surrogate(w)
    SK, SM = S.rows(sp.all_rows())
    return sp, SK, SM


@functools.lru_cache(maxsize=None)
def _oracle_shots(n, k, guess):
    sp, SK, SM = _oracle(n)
    w = _w(n)
    src = inputs.shot_positions(NSHOT, dim=2, seed=inputs.SEED_SHOTS_2D + 100 * k)
    out = []
    for s in src:
        lf = Leapfrog(sp, SK, SM, W.dt_of(w), rtol=1e-13, max_it=3000, guess_order=guess)
        u, _, tr = lf.run(np.zeros(sp.N), NSTEPS, sources=[(s, 10.0, 0.1, 1.0)], receivers=list(REC))
        out.append((u, tr))
    return src, out


def _ops(n):
    w = _w(n)
    sp = W.make_space(w)
    return w, sp, iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])


@pytest.mark.parametrize("guess", [0, 3])
def test_batch_matches_oracle_leapfrog(guess):
    made, waves, refs = [], [], []
    for k, n in enumerate(SIZES):
        w, sp, ops = _ops(n)
        src, ref = _oracle_shots(n, k, guess)
        wv = iga.iga_wave_create(ops, NSHOT, iga.IGA_F32, W.dt_of(w), src_pos=src, f0=10.0, t0=0.1, rec_pos=REC,
                                 nsteps_max=NSTEPS, cg_rtol=1e-6, cg_max_it=2000, cfl_check=0, cg_guess=guess)
        made.append((sp, ops))
        waves.append(wv)
        refs.append(ref)
    b = iga.iga_batch_create(waves)
    iga.iga_batch_step(b, NSTEPS, use_graph=True)
    for k, (sp_ops, wv, ref) in enumerate(zip(made, waves, refs)):
        ops = sp_ops[1]
        N = iga.iga_ops_info_get(ops).N
        u = torch.empty((NSHOT, N), dtype=torch.float32, device="cuda")
        iga.iga_wave_get_state(wv, u)
        torch.cuda.synchronize()
        ug = u.cpu().numpy().astype(np.float64)
        tg = iga.iga_wave_traces(wv, NSHOT, len(REC), NSTEPS)
        for s in range(NSHOT):
            ur, trr = ref[s]
            err = np.linalg.norm(ug[s] - ur) / np.linalg.norm(ur)
            terr = np.abs(tg[s] - trr).max() / np.abs(ur).max()
            print("mesh", SIZES[k], "shot", s, "state", err, "traces", terr)
            assert err <= 2e-5 and terr <= 2e-5
    iga.iga_batch_destroy(b)
    for wv in waves:
        iga.iga_wave_destroy(wv)
    for sp, ops in made:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(sp)


@pytest.mark.parametrize("schedule", ["persistent", "plain"])
def test_fp64_single_shot_matches_oracle_on_batched_family(schedule):
    n, k = SIZES[1], 1
    w, sp, ops = _ops(n)
    src, ref = _oracle_shots(n, k, 3)
    flags = iga.IGA_SOLVE_PLAIN if schedule == "plain" else 0
    wv = iga.iga_wave_create(ops, 1, iga.IGA_F64, W.dt_of(w), src_pos=src[:1], f0=10.0, t0=0.1, rec_pos=REC,
                             nsteps_max=NSTEPS, cg_rtol=1e-13, cg_max_it=3000, solve_flags=flags, cfl_check=0,
                             cg_guess=3)
    iga.iga_wave_step(wv, NSTEPS)
    N = iga.iga_ops_info_get(ops).N
    u = torch.empty((1, N), dtype=torch.float64, device="cuda")
    iga.iga_wave_get_state(wv, u)
    torch.cuda.synchronize()
    tg = iga.iga_wave_traces(wv, 1, len(REC), NSTEPS)[0]
    ur, trr = ref[0]
    ug = u.cpu().numpy()[0]
    assert np.linalg.norm(ug - ur) <= 1e-11 * np.linalg.norm(ur)
    assert np.abs(tg - trr).max() <= 1e-11 * np.abs(ur).max()
    iga.iga_wave_destroy(wv)
    iga.iga_ops_destroy(ops)
    iga.iga_space_destroy(sp)
