"""CUDA path (through the C ABI) vs the FP64 oracle on the same seeded inputs.

Tolerances:
* index / layout work (sample indices, zero pattern of the fields) is bit-exact;
* FP64 floating point: 1e-12 relative to the largest entry of the operator (fields)
  or to the |A| |x| bound of the row (operator applies);
* FP32 paths: 2e-5 relative on the same scales.
The CG-based tests use rtol 1e-13 on both sides so that the solver error stays
below the comparison tolerance.
"""
import functools

import numpy as np
import pytest

import inputs
from oracle.assembly import stencil_to_csr, true_rows
from oracle.surrogate import sample_indices
from oracle.wave import Leapfrog, gaussian_pulse, pcg, point_values
from tests.oracle_cases import oracle_space, oracle_surrogate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

CASES = {
    "annulus64_p2": lambda: W.scaled("annulus64_p2"),
    "annulus40_p3_sincos": lambda: W.scaled("annulus512_p3", n_el=40),
    "cube20_p2_theta": lambda: W.scaled("cube96_p2", n_el=20),
    "minimal_p2_q1": lambda: W.scaled("annulus64_p2", n_el=10, q=1, M=100),
    # sampling fine enough for a definite K~ (M = 6 on n_el = 20 gives an indefinite K~)
    "cube20_p2_theta_M2": lambda: W.scaled("cube96_p2", n_el=20, M=2),
}


@functools.lru_cache(maxsize=None)
def oracle_full(name):
    w = CASES[name]()
    sp, S = oracle_surrogate(w)
    rows = sp.all_rows()
    SK, SM = S.rows(rows)
    TK, TM = true_rows(sp, rows)
    return sp, S, SK, SM, TK, TM


@functools.lru_cache(maxsize=None)
def gpu_ops(name, flags=0, M=None):
    w = CASES[name]()
    space = W.make_space(w)
    ops = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"] if M is None else M, flags)
    return space, ops


def fields(ops, which, dtype):
    info = iga.iga_ops_info_get(ops)
    nf = info.nK if which == iga.IGA_OP_K else info.nM
    t = torch.empty((nf, info.N), dtype=torch.float64 if dtype == iga.IGA_F64 else torch.float32,
                    device="cuda")
    iga.iga_ops_copy_fields(ops, which, dtype, t)
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_fields(sp, SK, SM):
    t0 = (sp.D - 1) // 2
    return SK[:, t0 + 1:].T, SM[:, t0:].T


@pytest.mark.parametrize("name", list(CASES))
def test_sample_indices_bit_exact(name):
    w = CASES[name]()
    _, ops = gpu_ops(name)
    m = w["n_el"] + w["p"]
    assert list(iga.iga_ops_sample_indices(ops)) == list(sample_indices(m, w["p"], w["M"]))


@pytest.mark.parametrize("name", list(CASES))
def test_fields_fp64_match_oracle(name):
    sp, S, SK, SM, _, _ = oracle_full(name)
    _, ops = gpu_ops(name)
    oK, oM = oracle_fields(sp, SK, SM)
    gK, gM = fields(ops, iga.IGA_OP_K, iga.IGA_F64), fields(ops, iga.IGA_OP_M, iga.IGA_F64)
    # layout: the zero pattern (columns outside the grid) is identical
    assert np.array_equal(gK == 0.0, oK == 0.0)
    assert np.array_equal(gM == 0.0, oM == 0.0)
    assert np.abs(gK - oK).max() <= 1e-12 * np.abs(oK).max()
    assert np.abs(gM - oM).max() <= 1e-12 * np.abs(oM).max()


@pytest.mark.parametrize("name", list(CASES))
def test_fields_match_oracle_per_entry(name):
    """Every stored entry on its own scale: |gpu - oracle| <= 1e-12 |oracle| + 1e-14 max|oracle|
    (the floor covers entries that cancel to nearly zero, whose rounding is set by the
    size of the terms that cancel)."""
    sp, S, SK, SM, _, _ = oracle_full(name)
    _, ops = gpu_ops(name)
    oK, oM = oracle_fields(sp, SK, SM)
    for g, o in ((fields(ops, iga.IGA_OP_K, iga.IGA_F64), oK), (fields(ops, iga.IGA_OP_M, iga.IGA_F64), oM)):
        bound = 1e-12 * np.abs(o) + 1e-14 * np.abs(o).max()
        ratio = (np.abs(g - o) / bound).max()
        print(name, "worst per-entry error / bound", ratio)
        assert ratio <= 1.0


@pytest.mark.parametrize("name", ["annulus64_p2", "cube20_p2_theta"])
def test_fields_fp32_are_rounded_fp64(name):
    _, ops = gpu_ops(name)
    for which in (iga.IGA_OP_K, iga.IGA_OP_M):
        f64 = fields(ops, which, iga.IGA_F64)
        f32 = fields(ops, which, iga.IGA_F32)
        assert np.array_equal(f32, f64.astype(np.float32))


@pytest.mark.parametrize("name", ["annulus40_p3_sincos", "cube20_p2_theta"])
def test_sample_tables_match_oracle(name):
    sp, S, *_ = oracle_full(name)
    _, ops = gpu_ops(name, flags=iga.IGA_KEEP_SAMPLES)
    info = iga.iga_ops_info_get(ops)
    for which, ref in ((iga.IGA_OP_K, S.sK), (iga.IGA_OP_M, S.sM)):
        t = torch.empty((info.D, info.n_sample_rows), dtype=torch.float64, device="cuda")
        iga.iga_ops_copy_samples(ops, which, t)
        got = t.cpu().numpy()
        want = np.stack([inputs.colex(ref[k]) for k in range(info.D)])
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("name", ["annulus64_p2", "cube20_p2_theta"])
def test_true_only_matches_oracle_true_matrix(name):
    sp, _, _, _, TK, TM = oracle_full(name)
    _, ops = gpu_ops(name, flags=iga.IGA_TRUE_ONLY)
    oK, oM = oracle_fields(sp, TK, TM)
    gK, gM = fields(ops, iga.IGA_OP_K, iga.IGA_F64), fields(ops, iga.IGA_OP_M, iga.IGA_F64)
    assert np.abs(gK - oK).max() <= 1e-12 * np.abs(oK).max()
    assert np.abs(gM - oM).max() <= 1e-12 * np.abs(oM).max()


def test_sampling_length_one_reproduces_true_matrix_on_gpu():
    _, ops1 = gpu_ops("annulus40_p3_sincos", M=1)
    _, opsT = gpu_ops("annulus40_p3_sincos", flags=iga.IGA_TRUE_ONLY)
    for which in (iga.IGA_OP_K, iga.IGA_OP_M):
        a, b = fields(ops1, which, iga.IGA_F64), fields(opsT, which, iga.IGA_F64)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_assembly_is_deterministic():
    w = CASES["cube20_p2_theta"]()
    space = W.make_space(w)
    a = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"])
    b = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"])
    for which in (iga.IGA_OP_K, iga.IGA_OP_M):
        assert np.array_equal(fields(a, which, iga.IGA_F64), fields(b, which, iga.IGA_F64))
    iga.iga_ops_destroy(a)
    iga.iga_ops_destroy(b)


def test_assembly_reuses_the_space_band_lists():
    """The band element lists are built once per space (one for the surrogate band, one
    for TRUE_ONLY): alternating assemblies on one space give the fields of fresh spaces."""
    name = "annulus40_p3_sincos"
    w = CASES[name]()
    space = W.make_space(w)
    a = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"])
    t = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], iga.IGA_TRUE_ONLY)
    b = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"])
    _, fresh = gpu_ops(name)
    _, fresh_t = gpu_ops(name, flags=iga.IGA_TRUE_ONLY)
    for which in (iga.IGA_OP_K, iga.IGA_OP_M):
        ref = fields(fresh, which, iga.IGA_F64)
        assert np.array_equal(fields(a, which, iga.IGA_F64), ref)
        assert np.array_equal(fields(b, which, iga.IGA_F64), ref)
        assert np.array_equal(fields(t, which, iga.IGA_F64), fields(fresh_t, which, iga.IGA_F64))
    assert iga.iga_ops_info_get(a).n_band_elements == iga.iga_ops_info_get(fresh).n_band_elements
    for o in (a, t, b):
        iga.iga_ops_destroy(o)
    iga.iga_space_destroy(space)


def _apply_case(name, which, dtype, nrhs):
    sp, S, SK, SM, _, _ = oracle_full(name)
    _, ops = gpu_ops(name)
    A = stencil_to_csr(sp, SK if which == iga.IGA_OP_K else SM)
    x = inputs.vectors(sp.N, nrhs)
    tdt = torch.float64 if dtype == iga.IGA_F64 else torch.float32
    xg = torch.tensor(x, dtype=tdt, device="cuda")
    yg = torch.empty_like(xg)
    iga.iga_stencil_apply(ops, which, dtype, xg, yg, nrhs)
    torch.cuda.synchronize()
    y = yg.cpu().numpy().astype(np.float64)
    xr = x if dtype == iga.IGA_F64 else x.astype(np.float32).astype(np.float64)
    ref = (A @ xr.T).T
    bound = (abs(A) @ np.abs(xr).T).T
    return y, ref, bound


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("which", ["K", "M"])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_stencil_apply_fp64(name, which, nrhs):
    w = iga.IGA_OP_K if which == "K" else iga.IGA_OP_M
    y, ref, bound = _apply_case(name, w, iga.IGA_F64, nrhs)
    assert np.all(np.abs(y - ref) <= 1e-12 * bound + 1e-300)


@pytest.mark.parametrize("name", ["annulus64_p2", "annulus40_p3_sincos", "cube20_p2_theta"])
@pytest.mark.parametrize("which", ["K", "M"])
def test_stencil_apply_fp32(name, which):
    w = iga.IGA_OP_K if which == "K" else iga.IGA_OP_M
    y, ref, bound = _apply_case(name, w, iga.IGA_F32, 4)
    assert np.all(np.abs(y - ref) <= 2e-5 * bound + 1e-30)


def test_stencil_apply_zero_rhs_and_alias():
    _, ops = gpu_ops("annulus64_p2")
    x = torch.zeros(4356, dtype=torch.float64, device="cuda")
    iga.iga_stencil_apply(ops, iga.IGA_OP_K, iga.IGA_F64, x, x.clone(), 0)
    with pytest.raises(iga.IgaError):
        iga.iga_stencil_apply(ops, iga.IGA_OP_K, iga.IGA_F64, x, x, 1)


@pytest.mark.parametrize("name", ["annulus64_p2", "cube20_p2_theta"])
def test_mass_solve_fp64_matches_direct_solve(name):
    import scipy.sparse.linalg as spla
    sp, S, SK, SM, _, _ = oracle_full(name)
    _, ops = gpu_ops(name)
    M = stencil_to_csr(sp, SM).tocsc()
    b = inputs.vectors(sp.N, 5)
    ref = np.stack([spla.spsolve(M, bb) for bb in b])
    bg = torch.tensor(b, device="cuda")
    xg = torch.zeros_like(bg)
    rc, iters, rel = iga.iga_mass_solve(ops, iga.IGA_F64, bg, xg, 5, 1e-13, 2000)
    x = xg.cpu().numpy()
    assert np.all(rel <= 1e-13) and np.all(iters > 0)
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()


SCHEDULES = {"persistent": 0, "graph": 2, "plain": 1}


@pytest.mark.parametrize("schedule", list(SCHEDULES))
def test_mass_solve_iterates_match_oracle_pcg(schedule):
    """Fixed iteration count (rtol = 0): GPU and oracle run the identical recurrence."""
    sp, S, SK, SM, _, _ = oracle_full("annulus40_p3_sincos")
    _, ops = gpu_ops("annulus40_p3_sincos")
    M = stencil_to_csr(sp, SM)
    b = inputs.vectors(sp.N, 1)[0]
    x0 = 0.1 * inputs.vectors(sp.N, 1, seed=99)[0]
    xr, it, _ = pcg(M, b, x0.copy(), 1.0 / M.diagonal(), 0.0, 25)
    bg = torch.tensor(b[None], device="cuda")
    xg = torch.tensor(x0[None], device="cuda")
    rc, iters, _ = iga.iga_mass_solve(ops, iga.IGA_F64, bg, xg, 1, 0.0, 25, flags=SCHEDULES[schedule])
    assert iters[0] == 25 and it == 25
    assert np.abs(xg.cpu().numpy()[0] - xr).max() <= 1e-11 * np.abs(xr).max()


@pytest.mark.parametrize("name", ["annulus40_p3_sincos", "cube20_p2_theta_M2"])
@pytest.mark.parametrize("schedule", list(SCHEDULES))
def test_mass_solve_fp32_iterates_match_oracle_pcg(name, schedule):
    """FP32 path (FP32 fields and vectors, FP64 residual, compensated FP32 dot products
    widened to FP64 across threads), fixed 25 iterations, against the FP64 oracle PCG on
    the same FP32-rounded operator and inputs: what is left is the FP32 rounding of the
    CG vectors, checked at the FP32 tolerance 2e-5 of the largest iterate entry."""
    sp, S, SK, SM, _, _ = oracle_full(name)
    _, ops = gpu_ops(name)
    M = stencil_to_csr(sp, SM)
    dinv = (1.0 / M.diagonal()).astype(np.float32).astype(np.float64)
    M.data = M.data.astype(np.float32).astype(np.float64)
    b = inputs.vectors(sp.N, 1)[0].astype(np.float32)
    x0 = (0.1 * inputs.vectors(sp.N, 1, seed=99)[0]).astype(np.float32)
    xr, it, _ = pcg(M, b.astype(np.float64), x0.astype(np.float64), dinv, 0.0, 25)
    bg = torch.tensor(b[None], device="cuda")
    xg = torch.tensor(x0[None], device="cuda")
    rc, iters, _ = iga.iga_mass_solve(ops, iga.IGA_F32, bg, xg, 1, 0.0, 25, flags=SCHEDULES[schedule])
    assert iters[0] == 25 and it == 25
    err = np.abs(xg.cpu().numpy()[0].astype(np.float64) - xr).max() / np.abs(xr).max()
    assert err <= 2e-5, err


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_mass_solve_plain_and_persistent_schedules_agree_bitwise(dtype):
    _, ops = gpu_ops("cube20_p2_theta")
    info = iga.iga_ops_info_get(ops)
    dt = iga.IGA_F64 if dtype == "f64" else iga.IGA_F32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    b = torch.tensor(inputs.vectors(info.N, 3), dtype=tdt, device="cuda")
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    rtol = 1e-12 if dtype == "f64" else 1e-6
    _, i1, r1 = iga.iga_mass_solve(ops, dt, b, x1, 3, rtol, 500)
    _, i2, r2 = iga.iga_mass_solve(ops, dt, b, x2, 3, rtol, 500, flags=iga.IGA_SOLVE_PLAIN)
    assert list(i1) == list(i2)
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("schedule", list(SCHEDULES))
def test_mass_solve_zero_rhs_gives_zero(schedule):
    _, ops = gpu_ops("annulus64_p2")
    b = torch.zeros((1, 4356), dtype=torch.float64, device="cuda")
    x = torch.ones_like(b)
    rc, iters, rel = iga.iga_mass_solve(ops, iga.IGA_F64, b, x, 1, 1e-10, 100, flags=SCHEDULES[schedule])
    assert iters[0] == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("schedule", list(SCHEDULES))
def test_mass_solve_reports_non_convergence(schedule):
    _, ops = gpu_ops("annulus64_p2")
    b = torch.tensor(inputs.vectors(4356, 1), device="cuda")
    x = torch.zeros_like(b)
    rc, iters, rel = iga.iga_mass_solve(ops, iga.IGA_F64, b, x, 1, 1e-12, 2, flags=SCHEDULES[schedule],
                                        allow_not_converged=True)
    assert rc == iga.IGA_ERR_NOT_CONVERGED and iters[0] == 2 and rel[0] > 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_mass_solve_graph_schedule_matches_persistent(dtype):
    """Same recurrence, different block partition of the dot products: results agree to
    the CG tolerance scale and the iteration counts to within one."""
    _, ops = gpu_ops("cube20_p2_theta")
    info = iga.iga_ops_info_get(ops)
    dt = iga.IGA_F64 if dtype == "f64" else iga.IGA_F32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    b = torch.tensor(inputs.vectors(info.N, 5), dtype=tdt, device="cuda")   # a 4-wide and a 1-wide chunk
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    rtol = 1e-12 if dtype == "f64" else 1e-6
    _, i1, r1 = iga.iga_mass_solve(ops, dt, b, x1, 5, rtol, 500)
    _, i2, r2 = iga.iga_mass_solve(ops, dt, b, x2, 5, rtol, 500, flags=iga.IGA_SOLVE_GRAPH)
    assert np.all(np.abs(i1 - i2) <= 1) and np.all(r2 <= rtol)
    tol = 1e-10 if dtype == "f64" else 2e-5
    assert float((x1 - x2).abs().max()) <= tol * float(x1.abs().max())
    # deterministic: a second graph solve is bitwise identical
    x3 = torch.zeros_like(b)
    _, i3, _ = iga.iga_mass_solve(ops, dt, b, x3, 5, rtol, 500, flags=iga.IGA_SOLVE_GRAPH)
    assert list(i3) == list(i2) and torch.equal(x3, x2)


def _wave_case(dtype, nsteps=20):
    name = "annulus64_p2"
    w = CASES[name]()
    sp, S, SK, SM, _, _ = oracle_full(name)
    _, ops = gpu_ops(name)
    dt = W.dt_of(w)
    centre = inputs.pulse_centre(2)
    # receivers near the pulse (so the traces carry signal) and one on the boundary
    rec = np.array([centre + [0.03, 0.0], centre + [0.0, -0.04], [0.0, centre[1]]])
    wave = iga.iga_wave_create(ops, 1, dtype, dt, init_kind=iga.IGA_INIT_GAUSS_PULSE,
                               pulse_centre=centre[None], pulse_width=0.05, rec_pos=rec,
                               nsteps_max=nsteps, cg_rtol=1e-13 if dtype == iga.IGA_F64 else 1e-6,
                               cg_max_it=3000)
    iga.iga_wave_step(wave, nsteps)
    tdt = torch.float64 if dtype == iga.IGA_F64 else torch.float32
    u = torch.empty((1, sp.N), dtype=tdt, device="cuda")
    iga.iga_wave_get_state(wave, u)
    torch.cuda.synchronize()
    traces = iga.iga_wave_traces(wave, 1, len(rec), nsteps)
    iga.iga_wave_destroy(wave)
    lf = Leapfrog(sp, SK, SM, dt, rtol=1e-13, max_it=3000)
    xc = sp.geometry(centre)[0]
    u0 = gaussian_pulse(sp, xc, 0.05)
    ur, _, tr = lf.run(u0, nsteps, receivers=list(rec))
    return u.cpu().numpy()[0].astype(np.float64), ur, traces[0], tr


def test_wave_fp64_matches_oracle():
    u, ur, tr, trr = _wave_case(iga.IGA_F64)
    assert np.linalg.norm(u - ur) <= 1e-11 * np.linalg.norm(ur)
    # every coefficient, not only the L2 norm of the state
    assert np.abs(u - ur).max() <= 1e-11 * np.abs(ur).max()
    # a trace is a weighted sum of (p+1)^d coefficients: compare on the field's scale
    assert np.abs(tr - trr).max() <= 1e-11 * np.abs(ur).max()


def test_wave_fp32_error_against_fp64_oracle():
    u, ur, tr, trr = _wave_case(iga.IGA_F32)
    err = np.linalg.norm(u - ur) / np.linalg.norm(ur)
    print("FP32 leapfrog relative L2 error after 20 steps:", err)
    assert err <= 1e-5
    assert np.abs(u - ur).max() <= 2e-5 * np.abs(ur).max()
    assert np.abs(tr - trr).max() <= 2e-5 * np.abs(ur).max()


@pytest.mark.parametrize("mode", ["f64", "f64_plain", "f64_graph", "f32", "f32_graph", "f64_guess2", "f32_guess2",
                                  "f64_guess1", "f32_guess3", "f64_guess6", "f32_guess6", "f32_graph_guess4",
                                  "f64_refine", "f64_refine_guess3"])
def test_wave_cube_ricker_source_matches_oracle(mode):
    """3-D, lognormal wave speed, Ricker point source at the centre (the bench workload family)."""
    name = "cube20_p2_theta_M2"
    w = CASES[name]()
    sp, S, SK, SM, _, _ = oracle_full(name)
    _, ops = gpu_ops(name)
    dt = W.dt_of(w)
    nsteps = 60
    src = W.source_position(w)
    rec = np.array([src + [0.05, 0.0, 0.0], src + [0.0, -0.1, 0.05]])
    f32 = mode.startswith("f32")
    dtype = iga.IGA_F32 if f32 else iga.IGA_F64
    flags = iga.IGA_SOLVE_PLAIN if "plain" in mode else iga.IGA_SOLVE_GRAPH if "graph" in mode else 0
    if "refine" in mode:
        flags |= iga.IGA_SOLVE_REFINE
    guess = int(mode[-1]) if "guess" in mode else 0
    wave = iga.iga_wave_create(ops, 1, dtype, dt, src_pos=src[None], f0=10.0, t0=0.1, rec_pos=rec,
                               nsteps_max=nsteps, cg_rtol=1e-6 if f32 else 1e-13,
                               cg_max_it=3000, solve_flags=flags, cg_guess=guess)
    iga.iga_wave_step(wave, nsteps)
    tdt = torch.float32 if f32 else torch.float64
    u = torch.empty((1, sp.N), dtype=tdt, device="cuda")
    iga.iga_wave_get_state(wave, u)
    torch.cuda.synchronize()
    tr = iga.iga_wave_traces(wave, 1, len(rec), nsteps)[0]
    iga.iga_wave_destroy(wave)
    lf = Leapfrog(sp, SK, SM, dt, rtol=1e-13, max_it=3000, guess_order=guess)
    ur, _, trr = lf.run(np.zeros(sp.N), nsteps, sources=[(src, 10.0, 0.1, 1.0)], receivers=list(rec))
    ug = u.cpu().numpy()[0].astype(np.float64)
    err = np.linalg.norm(ug - ur) / np.linalg.norm(ur)
    terr = np.abs(tr - trr).max() / np.abs(ur).max()
    print(mode, "relative L2 error", err, "trace error", terr)
    # FP32 parity tolerance 2e-5: storing M~ in FP32 perturbs each solve by about
    # cond(M~) * 2^-24 ~ 1e-5 whatever the CG tolerance
    tol = 2e-5 if f32 else 1e-11
    assert err <= tol and terr <= tol
    # the state in the max norm as well: no single coefficient off by more than tol
    assert np.abs(ug - ur).max() <= tol * np.abs(ur).max()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_multishot_wave_with_extrapolated_start_matches_single_shots(dtype):
    """Five shots in one wave (CG chunks of 4 + 1 right-hand sides) with the order-3 CG
    start: every shot equals the same shot stepped alone (FP64 1e-11: both solve to
    1e-13; FP32 2e-5: the chunks reduce in a different order and stop at different
    iterates within rtol 1e-6)."""
    name = "annulus40_p3_sincos"
    w = CASES[name]()
    _, ops = gpu_ops(name)
    N = iga.iga_ops_info_get(ops).N
    dt = W.dt_of(w)
    src = inputs.shot_positions(5, dim=2, seed=inputs.SEED_SHOTS_2D + 7)
    dt_code = iga.IGA_F64 if dtype == "f64" else iga.IGA_F32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    rtol = 1e-13 if dtype == "f64" else 1e-6
    nsteps = 25

    def run(pos):
        wv = iga.iga_wave_create(ops, len(pos), dt_code, dt, src_pos=pos, f0=10.0, t0=0.1, cg_rtol=rtol,
                                 cg_max_it=3000, cg_guess=3)
        iga.iga_wave_step(wv, nsteps)
        u = torch.empty((len(pos), N), dtype=tdt, device="cuda")
        iga.iga_wave_get_state(wv, u)
        torch.cuda.synchronize()
        iga.iga_wave_destroy(wv)
        return u.double().cpu().numpy()

    multi = run(src)
    tol = 1e-11 if dtype == "f64" else 2e-5
    for k in range(5):
        single = run(src[k:k + 1])[0]
        assert np.linalg.norm(multi[k] - single) <= tol * np.linalg.norm(single), k


def test_wave_rejects_cg_guess_out_of_range():
    _, ops = gpu_ops("annulus64_p2")
    for bad in (-1, 7):
        with pytest.raises(iga.IgaError):
            iga.iga_wave_create(ops, 1, iga.IGA_F64, 1e-3, cg_guess=bad)


@pytest.mark.parametrize("case", ["annulus40", "cube16_M6"])
def test_spectrum_extremes_match_dense_eigensolver(case):
    """Lanczos (K~, M~) extremes vs scipy's dense generalized symmetric eigensolver."""
    import scipy.linalg as sla
    w = W.scaled("annulus512_p3", n_el=40) if case == "annulus40" else W.scaled("cube96_p2", n_el=16)
    sp, S = oracle_surrogate(w)
    SK, SM = S.rows(sp.all_rows())
    lam = sla.eigh(stencil_to_csr(sp, SK).toarray(), stencil_to_csr(sp, SM).toarray(), eigvals_only=True)
    space = W.make_space(w)
    ops = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"])
    lo, hi = iga.iga_ops_spectrum(ops, iga.IGA_F64, 80)
    print(case, "lanczos", lo, hi, "dense", lam[0], lam[-1])
    assert abs(hi - lam[-1]) <= 1e-3 * lam[-1]
    assert abs(lo - lam[0]) <= 2e-3 * lam[-1]
    iga.iga_ops_destroy(ops)


def test_wave_refuses_unstable_time_step():
    _, ops = gpu_ops("annulus64_p2")
    lo, hi = iga.iga_ops_spectrum(ops, iga.IGA_F64, 60)
    wave = iga.iga_wave_create(ops, 1, iga.IGA_F64, 2.5 / np.sqrt(hi), cfl_check=1)
    with pytest.raises(iga.IgaError) as e:
        iga.iga_wave_step(wave, 1)
    assert e.value.code == iga.IGA_ERR_ARG
    st = iga.iga_wave_stats_get(wave)
    assert abs(st.lambda_max - hi) <= 1e-2 * hi
    iga.iga_wave_destroy(wave)
    ok = iga.iga_wave_create(ops, 1, iga.IGA_F64, 1.0 / np.sqrt(hi), cfl_check=1)
    iga.iga_wave_step(ok, 2)
    iga.iga_wave_destroy(ok)
