"""Batched persistent stepping (C ABI): several meshes of uneven size in one
cooperative launch match the same waves stepped one by one; the captured graph
replays bit-identically; the partition tuner keeps results within FP32 rounding."""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

SIZES = (24, 32, 40)
NSHOT = 4
NSTEPS = 30


def _problems():
    out = []
    for k, n in enumerate(SIZES):
        w = W.scaled("annulus512_p3", n_el=n, M=4)
        sp = W.make_space(w)
        ops = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
        src = inputs.shot_positions(NSHOT, dim=2, seed=inputs.SEED_SHOTS_2D + 100 * k)
        rec = np.array([[0.5, 0.5], [0.2, 0.8], [0.9, 0.1]])
        out.append((w, sp, ops, src, rec))
    return out


def _wave(prob, guess=0):
    w, sp, ops, src, rec = prob
    return iga.iga_wave_create(ops, NSHOT, iga.IGA_F32, W.dt_of(w), src_pos=src, f0=10.0, t0=0.1, rec_pos=rec,
                               nsteps_max=NSTEPS, cg_rtol=1e-6, cg_max_it=2000, cfl_check=0, cg_guess=guess)


def _state(wave, ops):
    N = iga.iga_ops_info_get(ops).N
    u = torch.empty((NSHOT, N), dtype=torch.float32, device="cuda")
    iga.iga_wave_get_state(wave, u)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("guess", [0, 2, 4])
def test_batch_matches_individual_waves_and_graph_replay_is_exact(guess):
    """guess: the waves' CG start order (2: quadratic extrapolation in time, whose three
    acceleration buffers rotate inside the kernel and across graph replays)."""
    probs = _problems()
    singles = [_wave(p, guess) for p in probs]
    for wv in singles:
        iga.iga_wave_step(wv, NSTEPS)
    batched = [_wave(p, guess) for p in probs]
    b = iga.iga_batch_create(batched)
    for _ in range(3):                       # 10 + 10 + 10 steps through the captured graph
        iga.iga_batch_step(b, NSTEPS // 3, use_graph=True)
    direct = [_wave(p, guess) for p in probs]
    b2 = iga.iga_batch_create(direct)
    iga.iga_batch_step(b2, NSTEPS, use_graph=False)
    for k, p in enumerate(probs):
        ops, rec = p[2], p[4]
        us, ub, ud = _state(singles[k], ops), _state(batched[k], ops), _state(direct[k], ops)
        err = np.linalg.norm(ub - us) / np.linalg.norm(us)
        print("mesh", SIZES[k], "batched vs single relative L2", err)
        assert err <= 1e-5
        tb = iga.iga_wave_traces(batched[k], NSHOT, len(rec), NSTEPS)
        ts = iga.iga_wave_traces(singles[k], NSHOT, len(rec), NSTEPS)
        assert tb.shape == ts.shape
        # a trace is a weighted sum of (p+1)^d coefficients (weights summing to one):
        # compared on the field's scale, as the states
        assert np.abs(tb - ts).max() <= 1e-5 * np.abs(us).max()
        # the same partition and the same per-block reduction order: replay is bit-identical
        assert np.array_equal(ub, ud)
    iga.iga_batch_destroy(b)
    iga.iga_batch_destroy(b2)


def test_batch_tuner_rebalances_and_keeps_results():
    probs = _problems()
    waves = [_wave(p) for p in probs]
    b = iga.iga_batch_create(waves)
    before = iga.iga_batch_partition(b, len(probs))
    iga.iga_batch_tune(b, trial_steps=3, rounds=2)
    after = iga.iga_batch_partition(b, len(probs))
    assert sum(before) == sum(after) and all(x >= 1 for x in after)
    for wv, p in zip(waves, probs):
        iga.iga_wave_reset(wv, p[2])
    iga.iga_batch_step(b, NSTEPS, use_graph=True)
    singles = [_wave(p) for p in probs]
    for wv in singles:
        iga.iga_wave_step(wv, NSTEPS)
    for k, p in enumerate(probs):
        err = np.linalg.norm(_state(waves[k], p[2]) - _state(singles[k], p[2])) / np.linalg.norm(_state(singles[k], p[2]))
        assert err <= 1e-5
    iga.iga_batch_destroy(b)


def test_batch_continues_waves_stepped_on_their_own_with_extrapolated_start():
    """A wave stepped alone for a few steps (its acceleration buffers rotated on the
    host) and then batched continues the same scheme as a wave stepped alone throughout."""
    probs = _problems()
    singles = [_wave(p, 4) for p in probs]
    for wv in singles:
        iga.iga_wave_step(wv, NSTEPS)
    mixed = [_wave(p, 4) for p in probs]
    for wv in mixed:
        iga.iga_wave_step(wv, 7)
    b = iga.iga_batch_create(mixed)
    iga.iga_batch_step(b, 11, use_graph=True)
    for wv in mixed:                         # back to single stepping, then batched again
        iga.iga_wave_step(wv, 4)
    iga.iga_batch_step(b, NSTEPS - 22, use_graph=True)
    for k, p in enumerate(probs):
        us, um = _state(singles[k], p[2]), _state(mixed[k], p[2])
        err = np.linalg.norm(um - us) / np.linalg.norm(us)
        print("mesh", SIZES[k], "mixed vs single relative L2", err)
        assert err <= 1e-5
    iga.iga_batch_destroy(b)
