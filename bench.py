#!/usr/bin/env python
"""Benchmark of the surrogate-matrix IGA wave hot path on GB300.

One bench step is one pass of the whole hot path over the workload: surrogate
assembly (index sets, sample-row quadrature, band quadrature, interpolation,
surrogate evaluation) followed by `nsteps` leapfrog steps (K~ apply, Jacobi-PCG
on M~, update, receivers), all on the device.

Default workload: cube96_p2 (3-D p=2, 96^3 elements, sine-perturbed cube,
lognormal wave speed on a 16^3 cubic B-spline grid, q=2, M=6, Ricker source at
the centre, 500 FP32 time steps).  Its stencil fields (1.4 GB FP32 + FP64)
exceed the L2 cache, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs under torchrun as independent
replicas (one per GPU, no collective on the data path; weak scaling).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

# the CPU oracle legs run single-threaded (the thread count is reported)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "surrogate rows/s; wave shot-steps/s FP32-batched vs FP64 plain; % HBM peak"
HBM_FALLBACK_GBS = 6800.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


# ncu summaries of the two persistent PCG kernels, with the sources hashed when the
# counters were taken
PCG_PROFILES = {
    "pcg_persistent_kernel": (os.path.join(ROOT, "profiles", "stencil_apply_and_pcg_cube80_p2.md"),
                              ["solve.cu", "cg.cuh", "stencil.cuh"]),
    "pcg_brick_kernel": (os.path.join(ROOT, "profiles", "pcg_brick_kernel_cube80_p2.md"),
                         ["solve.cu", "cg.cuh", "pcg_brick.cuh", "brick.cuh"]),
}


def pcg_profiled_traffic(kernel):
    """DRAM bytes per row (per solve, per iteration) of a persistent PCG kernel from its
    committed ncu summary, or None when the kernel sources changed since the capture."""
    import hashlib
    try:
        path, sources = PCG_PROFILES[kernel]
        vals = {}
        with open(path) as f:
            for line in f:
                line = line.strip()
                for key in ("pcg_dram_bytes_per_row_init", "pcg_dram_bytes_per_row_iteration",
                            "kernel_sources_sha256_16"):
                    if line.startswith(key + ":"):
                        vals[key] = line.split(":", 1)[1].strip()
        h = hashlib.sha256()
        for name in sources:
            with open(os.path.join(ROOT, "paper_2004_05197_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
        if h.hexdigest()[:16] != vals.get("kernel_sources_sha256_16"):
            return None
        return float(vals["pcg_dram_bytes_per_row_init"]), float(vals["pcg_dram_bytes_per_row_iteration"])
    except Exception:
        return None


def max_over_ranks(ms, world, device):
    """The slowest rank's time (replicas: every rank times the same work on its GPU)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, ms_step, world):
    """Whole-job throughput: the units all ranks processed divided by the slowest time."""
    return world * units_per_rank / (ms_step / 1e3)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def cg_bytes(nM, R, es):
    """Algorithmic HBM bytes per row of one persistent PCG launch (Chronopoulos-Gear
    form; every field element read once per mass apply).

    init : apply r = b - M~x: fields nM*es + D^-1 es + per RHS (x, b read, u write: 3 es;
           r write: 8); apply w = M~u: fields nM*es + per RHS (u read, w write: 2 es)
    iter : phase 1 D^-1 es + per RHS (u, w, p, s, x read, p, s, x, u write: 9 es;
           r read + write: 16); phase 2 w = M~u: fields nM*es + per RHS (u read, w write: 2 es)
    """
    init = 2 * nM * es + es + R * (5 * es + 8)
    it = nM * es + es + R * (11 * es + 16)
    return init, it


def run_ours(args, rank, world, device):
    import numpy as np
    import torch

    import inputs
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

    w = W.scaled(args.workload)
    nsteps = args.nsteps or w["steps"]
    dt = W.dt_of(w)
    src = W.source_position(w)[None]
    rec = inputs.face_receivers(per_face=32) if w["dim"] == 3 else np.array([[0.5, 0.9], [0.9, 0.5]])
    stream = torch.cuda.current_stream()
    space = W.make_space(w)
    info_s = iga.iga_space_info_get(space)
    N = info_s.N

    def assemble():
        return iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], 0, stream)

    ops = assemble()
    sflags = iga.IGA_SOLVE_GRAPH if args.solve == "graph" else 0
    wave = iga.iga_wave_create(ops, args.nshot, iga.IGA_F32, dt, src_pos=np.repeat(src, args.nshot, 0),
                               f0=10.0, t0=0.1, rec_pos=rec, nsteps_max=nsteps, cg_rtol=args.cg_rtol,
                               cg_max_it=args.cg_max_it, cfl_check=2, solve_flags=sflags,
                               cg_guess=args.cg_guess)
    iga.iga_wave_set_timing(wave, True)

    def one_pass(old_ops):
        o = assemble()
        iga.iga_wave_reset(wave, o, stream)
        iga.iga_wave_step(wave, nsteps, stream)
        if old_ops is not None:
            iga.iga_ops_destroy(old_ops)
        return o

    for _ in range(args.warmup):
        ops = one_pass(ops)
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    asm_ms, cg_ms, force_ms, cg_it, cg_solves = 0.0, 0.0, 0.0, 0, 0
    launches0 = iga.iga_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t_host = time.perf_counter()
    for _ in range(args.steps):
        o = assemble()
        asm_ms += iga.iga_ops_info_get(o).t_total_ms
        iga.iga_wave_reset(wave, o, stream)
        iga.iga_wave_step(wave, nsteps, stream)
        st = iga.iga_wave_stats_get(wave)
        cg_ms += st.cg_ms
        force_ms += st.force_ms
        cg_it += st.cg_iterations
        cg_solves += st.cg_solves
        iga.iga_ops_destroy(ops)
        ops = o
    ev1.record(stream)
    torch.cuda.synchronize()
    t_host = time.perf_counter() - t_host
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    launches = iga.iga_launch_count() - launches0
    if args.solve == "graph":
        # the library counts one launch per solve graph; it runs init 1, init 2, zero-RHS,
        # finish and two kernels per iteration
        launches += 3 * cg_solves + 2 * cg_it
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, device)

    oinfo = iga.iga_ops_info_get(ops)
    K = args.steps
    ms_step = ms / K
    shot_steps = args.nshot * nsteps
    value = replica_value(shot_steps, ms_step, world)
    # dominant kernel: the persistent PCG launch (events around every launch, on its stream)
    init_b, it_b = cg_bytes(oinfo.nM, 1, 4)
    # one shot: every launch is one solve and the device counter holds its iterations
    cg_bytes_total = (cg_solves * init_b + cg_it * it_b) * N if args.nshot == 1 else None
    achieved = cg_bytes_total / (cg_ms / 1e3) / 1e9 if cg_bytes_total else None
    # which persistent kernel ran: the brick form for an FP32 single-RHS solve on an
    # operator whose M~ apply runs on bricks
    brick_paths = iga.iga_ops_brick_info(ops, with_paths=True)[4]
    if args.solve == "graph":
        kernel = "pcg graph (cgg_phase1_kernel + cgg_phase2_kernel)"
    else:
        kernel = "pcg_brick_kernel" if (args.nshot == 1 and brick_paths & 2) else "pcg_persistent_kernel"
    # ncu DRAM bytes of the same kernel on the n_el = 80 case, scaled to this launch by rows
    # and by the mean iterations per launch (traffic grows in proportion to both)
    prof = pcg_profiled_traffic(kernel) if (args.nshot == 1 and kernel in PCG_PROFILES) else None
    traffic = ((prof[0] + prof[1] * cg_it / max(1, cg_solves)) * N) if prof else None
    traffic_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, %s, scaled by rows and "
                   "iterations per launch" % os.path.relpath(PCG_PROFILES[kernel][0], ROOT)) if prof else None
    peaks = load_peaks()
    peak = peaks.get("hbm_gbs") if peaks else None
    peak_src = "measured" if peak else "fallback"
    peak = peak or HBM_FALLBACK_GBS
    comps = {
        "surrogate_rows_per_s": N / (asm_ms / K / 1e3),
        "assembly_ms": asm_ms / K,
        "assembly_split_ms": {"band": oinfo.t_band_ms, "sample_rows": oinfo.t_sample_ms,
                              "interpolation": oinfo.t_interp_ms, "evaluation": oinfo.t_eval_ms},
        "stepping_shot_steps_per_s": shot_steps / ((ms_step - asm_ms / K) / 1e3),
        "cg_iterations_per_step": cg_it / (K * nsteps * args.nshot),
        "cg_ms_per_step": cg_ms / (K * nsteps),
        "force_ms_per_step": force_ms / (K * nsteps),
        "host_s_per_step": t_host / K,
    }
    out = {
        "metric": METRIC, "value": value, "unit": "shot-steps/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, world),
        "components": comps,
        "roofline": {"bound": "hbm",
                     "kernel": kernel,
                     "achieved": achieved, "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": traffic_src,
                     "bytes_per_row_per_iteration": it_b, "launches": cg_solves,
                     "avg_launch_ms": cg_ms / max(1, cg_solves)},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    return out, (space, ops, wave, w, nsteps, dt, src, rec)


def stencil_apply_leg(ctx, args):
    """Stand-alone FP32 K~ and M~ applies (one right-hand side) on the bench operator:
    CUDA events on the launching stream around 20 back-to-back launches (the fields are
    larger than L2, so every launch streams them from HBM), algorithmic bytes = every
    stored field element once + x read + y written."""
    import torch

    from paper_2004_05197_gb300 import iga
    space, ops, wave, w, nsteps, dt, src, rec = ctx
    info = iga.iga_ops_info_get(ops)
    N = info.N
    peaks = load_peaks()
    peak = (peaks or {}).get("hbm_gbs") or HBM_FALLBACK_GBS
    stream = torch.cuda.current_stream()
    x = torch.rand((1, N), device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    res = {}
    for name, which, nf in (("K", iga.IGA_OP_K, info.nK), ("M", iga.IGA_OP_M, info.nM)):
        for _ in range(3):
            iga.iga_stencil_apply(ops, which, iga.IGA_F32, x, y, 1, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            iga.iga_stencil_apply(ops, which, iga.IGA_F32, x, y, 1, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        gbs = (nf * 4 + 8) * N / (us * 1e-6) / 1e9
        res["stencil_apply_fp32_" + name] = {"us": us, "fields": nf, "bytes_per_row": nf * 4 + 8,
                                            "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak}
    # on-the-fly evaluation of the stencil functions (IGA_PATH_ONTHEFLY) on the same
    # operator and vector: per apply the coefficient contraction over directions 1..d-1
    # and the row kernel (surrogate-only rows from the coefficients, the rest from fields)
    iga.iga_ops_set_path(ops, iga.IGA_PATH_ONTHEFLY)
    L = info.m - 4 * info.p
    deep = (L - 2 * info.p) ** info.dim / N
    for name, which in (("K", iga.IGA_OP_K), ("M", iga.IGA_OP_M)):
        us = _time_us(lambda: iga.iga_stencil_apply(ops, which, iga.IGA_F32, x, y, 1, stream), stream)
        res["onthefly_apply_fp32_" + name] = {"us": us, "over_stored": us / res["stencil_apply_fp32_" + name]["us"],
                                              "rows_from_coefficients": deep}
    iga.iga_ops_set_path(ops, iga.IGA_PATH_AUTO)
    return res


def _time_us(fn, stream, reps=20, warm=3):
    import torch
    for _ in range(warm):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / reps


def next_rows_leg(ctx, args):
    """--next-rows: measurements of the rows beyond the hot path.  (1) The
    volume-preserving mass M~ = D + M~_0 on the bench operator: assembly time, FP32 apply
    and FP32 Jacobi-PCG (rtol 1e-6, zero start) against the plain surrogate mass.
    (2) Multi-patch: the quarter annulus as four angular sector patches (p = 3, 256^2
    elements each, q = 3, M = 8, glued along three sides), global FP32 / FP64 applies and
    the FP32 mass solve, against one 256^2 patch."""
    import numpy as np
    import torch

    import inputs
    from paper_2004_05197_gb300 import iga
    space, ops, wave, w, nsteps, dt, src, rec = ctx
    stream = torch.cuda.current_stream()
    out = {}
    # (1) volume-preserving mass on the bench space
    vp = iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], iga.IGA_MASS_VOLUME_PRESERVING, stream)
    torch.cuda.synchronize()
    N = iga.iga_ops_info_get(ops).N
    b = torch.tensor(inputs.vectors(N, 1), dtype=torch.float32, device="cuda")
    y = torch.empty_like(b)
    for name, o in (("plain", ops), ("volume_preserving", vp)):
        info = iga.iga_ops_info_get(o)
        t_apply = _time_us(lambda: iga.iga_stencil_apply(o, iga.IGA_OP_M, iga.IGA_F32, b, y, 1, stream), stream)
        a = torch.zeros_like(b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, it, rel = iga.iga_mass_solve(o, iga.IGA_F32, b, a, 1, 1e-6, 2000, stream=stream,
                                        allow_not_converged=True)
        e1.record(stream)
        torch.cuda.synchronize()
        out["mass_" + name] = {"assembly_ms": info.t_total_ms, "apply_fp32_us": t_apply,
                               "apply_gbs": (info.nM * 4 + 8) * N / (t_apply * 1e-6) / 1e9,
                               "solve_fp32_iterations": int(it[0]), "solve_fp32_ms": e0.elapsed_time(e1),
                               "solve_fp32_relres": float(rel[0])}
    iga.iga_ops_destroy(vp)
    # (2) multi-patch quarter annulus, four sectors
    p, n_el, q, M = 3, 256, 3, 8
    e = np.linspace(0.0, 0.5 * np.pi, 5)
    sectors = [(1.0, 2.0, e[l], e[l + 1]) for l in range(4)]
    ifs = [(l, 3, l + 1, 2, 0) for l in range(3)]
    spaces = [iga.iga_space_create(2, p, n_el, iga.IGA_MAP_ANNULUS_SECTOR, 0.0, iga.IGA_COEF_CONST, 1.0, sector=sc)
              for sc in sectors]
    pops = [iga.iga_surrogate_assemble(sp, p, q, M, 0, stream) for sp in spaces]
    mp = iga.iga_multipatch_create(pops, ifs)
    G = iga.iga_multipatch_size(mp)
    n_loc = iga.iga_ops_info_get(pops[0]).N
    res = {"patches": 4, "p": p, "n_el_per_patch": n_el, "global_functions": G}
    for dtype, tdt, tag in ((iga.IGA_F32, torch.float32, "fp32"), (iga.IGA_F64, torch.float64, "fp64")):
        xg = torch.tensor(inputs.vectors(G, 1), dtype=tdt, device="cuda")
        yg = torch.empty_like(xg)
        xl = torch.tensor(inputs.vectors(n_loc, 1), dtype=tdt, device="cuda")
        yl = torch.empty_like(xl)
        for which, wn in ((iga.IGA_OP_K, "K"), (iga.IGA_OP_M, "M")):
            res["apply_%s_%s_us" % (wn, tag)] = _time_us(
                lambda: iga.iga_multipatch_apply(mp, which, dtype, xg, yg, 1, stream), stream)
            res["single_patch_apply_%s_%s_us" % (wn, tag)] = _time_us(
                lambda: iga.iga_stencil_apply(pops[0], which, dtype, xl, yl, 1, stream), stream)
    bg = torch.tensor(inputs.vectors(G, 1), dtype=torch.float32, device="cuda")
    ag = torch.zeros_like(bg)
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, it, rel = iga.iga_multipatch_mass_solve(mp, iga.IGA_F32, bg, ag, 1, 1e-6, 2000, stream=stream,
                                               allow_not_converged=True)
    torch.cuda.synchronize()
    res["mass_solve_fp32_iterations"] = int(it[0])
    res["mass_solve_fp32_ms"] = (time.perf_counter() - t) * 1e3
    res["mass_solve_fp32_relres"] = float(rel[0])
    iga.iga_multipatch_destroy(mp)
    for o in pops:
        iga.iga_ops_destroy(o)
    for sp in spaces:
        iga.iga_space_destroy(sp)
    out["multipatch"] = res
    return {"next_rows": out}


def fp64_forms_and_error(ctx, args):
    """Single-shot FP64 forms of the bench workload beside the FP32 persistent form.

    * FP64 with the plain CG schedule (a host round trip per CG iteration), with the
      graph schedule (phase launches in a CUDA graph, convergence on the device), by
      iterative refinement around the FP32 solver (IGA_SOLVE_REFINE: FP64 residual and
      stopping rule, FP32 corrections) and with the persistent schedule: shot-steps/s,
      the first three on `compare_steps` steps, the persistent one on all steps;
    * FP32 error: relative L2 distance of the FP32 state after all steps (the final state
      of the timed FP32 pass) from the FP64 persistent state after the same steps (CG
      rtol 1e-10).  The FP64 waves are pinned to the oracle by the wave parity tests.
    """
    import numpy as np
    import torch

    from paper_2004_05197_gb300 import iga
    space, ops, wave, w, nsteps, dt, src, rec = ctx
    N = iga.iga_ops_info_get(ops).N
    res = {}
    u64 = None
    for name, flags, P in (("plain", iga.IGA_SOLVE_PLAIN, min(args.compare_steps, nsteps)),
                           ("graph", iga.IGA_SOLVE_GRAPH, min(args.compare_steps, nsteps)),
                           ("refine", iga.IGA_SOLVE_REFINE, min(args.compare_steps, nsteps)),
                           ("persistent", 0, nsteps)):
        w64 = iga.iga_wave_create(ops, 1, iga.IGA_F64, dt, src_pos=src, f0=10.0, t0=0.1, cg_rtol=1e-10,
                                  cg_max_it=args.cg_max_it, solve_flags=flags, cg_guess=args.cg_guess)
        torch.cuda.synchronize()
        t = time.perf_counter()
        iga.iga_wave_step(w64, P)
        torch.cuda.synchronize()
        t = time.perf_counter() - t
        res["fp64_%s_shot_steps_per_s" % name] = P / t
        res["fp64_%s_steps" % name] = P
        if name == "persistent":
            u64 = torch.empty((1, N), dtype=torch.float64, device="cuda")
            iga.iga_wave_get_state(w64, u64)
        iga.iga_wave_destroy(w64)
    u32 = torch.empty((1, N), dtype=torch.float32, device="cuda")
    iga.iga_wave_get_state(wave, u32)
    torch.cuda.synchronize()
    a = u32.double().cpu().numpy()
    b = u64.cpu().numpy()
    res["fp32_vs_fp64_rel_l2_error"] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    res["fp32_vs_fp64_steps"] = nsteps
    fastest = max(res["fp64_plain_shot_steps_per_s"], res["fp64_graph_shot_steps_per_s"],
                  res["fp64_refine_shot_steps_per_s"], res["fp64_persistent_shot_steps_per_s"])
    res["fp64_fastest_single_shot_shot_steps_per_s"] = fastest
    return res


def config2_leg(args):
    """2-D p=3 annulus, 512^2 elements, c = 1 + 0.5 sin(2 pi x) cos(2 pi y), q = 3, M = 8,
    Ricker f0 = 10 at s = (0.5, 0.5), dt = 0.1 h, `config2_steps` steps: FP32 persistent
    (CG rtol as the bench) against FP64 persistent (CG rtol 1e-10), shot-steps/s of both
    (assembly not included) and the FP32 relative L2 error after all steps.  Its FP32
    operators (52 MB) are L2-resident, so its rates are L2-bound, not HBM-bound."""
    import numpy as np
    import torch

    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W
    w = W.scaled("annulus512_p3")
    P = args.config2_steps
    sp = W.make_space(w)
    ops = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
    N = iga.iga_ops_info_get(ops).N
    src = W.source_position(w)[None]
    res = {"config2_workload": "annulus512_p3, %d steps" % P}
    states = {}
    for name, dtype, rtol in (("fp32", iga.IGA_F32, args.cg_rtol), ("fp64", iga.IGA_F64, 1e-10)):
        wv = iga.iga_wave_create(ops, 1, dtype, W.dt_of(w), src_pos=src, f0=10.0, t0=0.1, cg_rtol=rtol,
                                 cg_max_it=args.cg_max_it, cg_guess=args.cg_guess)
        iga.iga_wave_step(wv, 5)                     # warm-up, then restart
        iga.iga_wave_reset(wv, ops)
        torch.cuda.synchronize()
        t = time.perf_counter()
        iga.iga_wave_step(wv, P)
        torch.cuda.synchronize()
        t = time.perf_counter() - t
        res["config2_%s_shot_steps_per_s" % name] = P / t
        st = iga.iga_wave_stats_get(wv)
        res["config2_%s_cg_iterations_per_step" % name] = st.cg_iterations / max(1, st.steps)
        u = torch.empty((1, N), dtype=torch.float64 if dtype == iga.IGA_F64 else torch.float32, device="cuda")
        iga.iga_wave_get_state(wv, u)
        torch.cuda.synchronize()
        states[name] = u.double().cpu().numpy()
        iga.iga_wave_destroy(wv)
    a, b = states["fp32"], states["fp64"]
    res["config2_fp32_vs_fp64_rel_l2_error"] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    res["config2_fp32_over_fp64"] = res["config2_fp32_shot_steps_per_s"] / res["config2_fp64_shot_steps_per_s"]
    res["config2_l2_resident"] = "FP32 fields 52 MB, FP64 fields 106 MB: both below the 129 MB L2"
    iga.iga_ops_destroy(ops)
    iga.iga_space_destroy(sp)
    return res


def msweep_leg(args):
    """Mesh-dependent sampling (Sec. 5.2, Eq. MeshDependentSamplingLength) against a fixed
    sampling length on the cube p = 2 family (sine-perturbed map, lognormal wave speed):
    for n_el in 32, 48, 64, 96, 128, surrogate assembly with q = 2, M = 6 (the bench's)
    and with q = 5, M = M(h) = max{1, floor(0.5 m^(1 - (p+1)/(q+1)))} (a = b = 1,
    C = 0.5, h = 1/m, vanishing eps: the form of the paper's 2-D experiment).  Reports
    rows/s of the assembly (device time of the second assembly on the space), samples per
    direction, the a2 / a3 / a4 / a5 split, and the consistency error
    max|A~ - A| / max|A| for K and M against the full-quadrature assembly of the same
    space (IGA_TRUE_ONLY, pinned to the oracle's true matrices by the parity tests)."""
    import torch

    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

    def fields64(ops, which):
        info = iga.iga_ops_info_get(ops)
        nf = info.nK if which == iga.IGA_OP_K else info.nM
        t = torch.empty((nf, info.N), dtype=torch.float64, device="cuda")
        iga.iga_ops_copy_fields(ops, which, iga.IGA_F64, t)
        return t

    rows = []
    for n in (32, 48, 64, 96, 128):
        w = W.scaled("cube96_p2", n_el=n)
        m = n + w["p"]
        sp = W.make_space(w)
        tru = iga.iga_surrogate_assemble(sp, w["p"], w["q"], 1, iga.IGA_TRUE_ONLY)
        Mh = iga.iga_sampling_length_for_mesh(1.0 / m, w["p"], 5, 1.0, 1.0, 0.5, 1e-9)
        for label, q, M in (("fixed", 2, 6), ("mesh_dependent", 5, Mh)):
            o = iga.iga_surrogate_assemble(sp, w["p"], q, M, 0)
            iga.iga_ops_destroy(o)
            o = iga.iga_surrogate_assemble(sp, w["p"], q, M, 0)
            info = iga.iga_ops_info_get(o)
            err = {}
            for name, which in (("K", iga.IGA_OP_K), ("M", iga.IGA_OP_M)):
                a, b = fields64(o, which), fields64(tru, which)
                err[name] = float((a - b).abs().max() / b.abs().max())
                del a, b
            rows.append({"n_el": n, "N": info.N, "sampling": label, "q": q, "M": M, "samples_per_dir": info.ns,
                         "sample_rows": info.n_sample_rows, "band_elements": info.n_band_elements,
                         "assembly_ms": info.t_total_ms, "rows_per_s": info.N / (info.t_total_ms / 1e3),
                         "split_ms": {"band": info.t_band_ms, "sample_rows": info.t_sample_ms,
                                      "interpolation": info.t_interp_ms, "evaluation": info.t_eval_ms},
                         "consistency_error_K": err["K"], "consistency_error_M": err["M"]})
            iga.iga_ops_destroy(o)
        iga.iga_ops_destroy(tru)
        iga.iga_space_destroy(sp)
        torch.cuda.empty_cache()
    return {"msweep": rows}


def run_e2e(args, ctx):
    """Same pass through the public API from host buffers: theta, source and receiver
    positions uploaded every step, traces and the final field read back every step."""
    import numpy as np
    import torch

    import inputs
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W
    _, _, _, w, nsteps, dt, src, rec = ctx
    theta = W.theta_for(w)
    h2d = (0 if theta is None else theta.size * 8) + src.size * 8 + rec.size * 8
    times = []
    d2h = 0
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        sp = W.make_space(w)                                   # theta: host -> device
        o = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
        wv = iga.iga_wave_create(o, args.nshot, iga.IGA_F32, dt, src_pos=np.repeat(src, args.nshot, 0),
                                 f0=10.0, t0=0.1, rec_pos=rec, nsteps_max=nsteps, cg_rtol=args.cg_rtol,
                                 cg_max_it=args.cg_max_it, cg_guess=args.cg_guess,
                                 solve_flags=iga.IGA_SOLVE_GRAPH if args.solve == "graph" else 0)
        iga.iga_wave_step(wv, nsteps)
        tr = iga.iga_wave_traces(wv, args.nshot, len(rec), nsteps)   # device -> host
        N = iga.iga_ops_info_get(o).N
        u = torch.empty((args.nshot, N), dtype=torch.float32, device="cuda")
        iga.iga_wave_get_state(wv, u)
        uh = u.cpu()                                                  # device -> host
        t = time.perf_counter() - t
        d2h = tr.nbytes + uh.numel() * 4
        iga.iga_wave_destroy(wv)
        iga.iga_ops_destroy(o)
        iga.iga_space_destroy(sp)
        if k > 0:                                                     # first pass warms up
            times.append(t)
    t = sorted(times)[len(times) // 2]
    return {"value": args.nshot * nsteps / t, "unit": "shot-steps/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "s_per_step": t}


def run_batched(args):
    """Batched FP32 form vs the plain FP64 single-shot form (the batched workload).

    Four 2-D p=3 quarter-annulus meshes, 128^2, 256^2, 384^2, 512^2 elements
    (c = 1 + 0.5 sin(2 pi x) cos(2 pi y), q = 3, M = 8, dt = 0.1 h), 16 Ricker shots
    each at seeded uniform positions in [0.1, 0.9]^2: 64 shots advanced together
    in one persistent cooperative launch replayed from a CUDA graph (16 shots per
    mesh as two right-hand-side groups of 8).  Against it, one shot at a time in
    FP64 with the plain (host round trip per CG iteration), graph and persistent
    CG schedules, and the error of the FP32 batch against the FP64 persistent
    shot after all steps.
    """
    import numpy as np
    import torch

    import inputs
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W
    sizes = (128, 256, 384, 512)
    nsteps = args.batched_steps
    meshes, waves = [], []
    for k, n in enumerate(sizes):
        w = W.scaled("annulus512_p3", n_el=n)
        sp = W.make_space(w)
        ops = iga.iga_surrogate_assemble(sp, w["p"], w["q"], w["M"])
        src = inputs.shot_positions(16, dim=2, seed=inputs.SEED_SHOTS_2D + 100 * k)
        meshes.append((w, sp, ops, src))
        for g in range(2):
            waves.append(iga.iga_wave_create(ops, 8, iga.IGA_F32, W.dt_of(w), src_pos=src[8 * g:8 * g + 8],
                                             f0=10.0, t0=0.1, rec_pos=np.array([[0.5, 0.5]]), nsteps_max=nsteps + 64,
                                             cg_rtol=args.batched_rtol, cg_max_it=args.cg_max_it, cfl_check=2,
                                             cg_guess=args.batched_cg_guess))
    b = iga.iga_batch_create(waves)
    iga.iga_batch_tune(b, trial_steps=5, rounds=3)
    part = iga.iga_batch_partition(b, len(waves))
    for wv, k in zip(waves, range(len(waves))):
        iga.iga_wave_reset(wv, meshes[k // 2][2])
    iga.iga_batch_step(b, min(nsteps, 50), use_graph=True)      # warm-up (a shorter captured launch)
    for wv, k in zip(waves, range(len(waves))):
        iga.iga_wave_reset(wv, meshes[k // 2][2])
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    iga.iga_batch_step(b, nsteps, use_graph=True)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    batched = 64 * nsteps / (ms / 1e3)
    # FP32 states of the first shot of each mesh after nsteps, for the error
    u32 = []
    for k, (w, sp, ops, src) in enumerate(meshes):
        N = iga.iga_ops_info_get(ops).N
        u = torch.empty((8, N), dtype=torch.float32, device="cuda")
        iga.iga_wave_get_state(waves[2 * k], u)
        u32.append(u[0].double().cpu().numpy())
    iga.iga_batch_destroy(b)
    for wv in waves:
        iga.iga_wave_destroy(wv)
    # FP64 single-shot forms (first shot of each mesh): the plain schedule and the graph
    # schedule timed on `plain_steps` steps, the persistent schedule on all steps; the
    # persistent FP64 wave (CG rtol 1e-10) is also the reference of the FP32 error
    t_form = {"plain": 0.0, "graph": 0.0, "persistent": 0.0}
    ss_form = {"plain": 0, "graph": 0, "persistent": 0}
    errs = []
    for k, (w, sp, ops, src) in enumerate(meshes):
        for name, flags, P in (("plain", iga.IGA_SOLVE_PLAIN, args.plain_steps),
                               ("graph", iga.IGA_SOLVE_GRAPH, args.plain_steps), ("persistent", 0, nsteps)):
            wv = iga.iga_wave_create(ops, 1, iga.IGA_F64, W.dt_of(w), src_pos=src[:1], f0=10.0, t0=0.1,
                                     cg_rtol=1e-10, cg_max_it=args.cg_max_it, solve_flags=flags,
                                     cfl_check=0, cg_guess=args.batched_cg_guess)
            torch.cuda.synchronize()
            t = time.perf_counter()
            iga.iga_wave_step(wv, P)
            torch.cuda.synchronize()
            t_form[name] += time.perf_counter() - t
            ss_form[name] += P
            if name == "persistent":
                N = iga.iga_ops_info_get(ops).N
                u = torch.empty((1, N), dtype=torch.float64, device="cuda")
                iga.iga_wave_get_state(wv, u)
                torch.cuda.synchronize()
                ref = u[0].cpu().numpy()
                errs.append(float(np.linalg.norm(u32[k] - ref) / max(np.linalg.norm(ref), 1e-300)))
            iga.iga_wave_destroy(wv)
    for (w, sp, ops, src) in meshes:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(sp)
    # a single-shot step costs the same whichever shot it is: rates over the four meshes
    rate = {k: ss_form[k] / t_form[k] for k in t_form}
    plain = rate["plain"]
    fastest = max(rate.values())
    return {"batched_workload": "annulus p=3 meshes 128^2,256^2,384^2,512^2 x 16 Ricker shots, %d steps" % nsteps,
            "batched_fp32_shot_steps_per_s": batched, "batched_ms": ms,
            "plain_fp64_single_shot_shot_steps_per_s": plain,
            "graph_fp64_single_shot_shot_steps_per_s": rate["graph"],
            "persistent_fp64_single_shot_shot_steps_per_s": rate["persistent"],
            "batched_over_plain": batched / plain,
            "batched_over_fastest_fp64_single_shot": batched / fastest,
            "batched_fp32_vs_fp64_rel_l2_error_max": max(errs),
            "batched_partition_blocks": part,
            "batched_cg_start": ("previous acceleration" if args.batched_cg_guess == 0 else
                                 "polynomial extrapolation in time, order %d" % args.batched_cg_guess)}


def run_adjoint(args):
    """Gradient of the receiver misfit on the adjoint workload, timed, with its
    central-difference check.

    3-D p=2, 64^3 elements, sine-perturbed cube (0.1), wave speed on 12^3 cubic
    B-spline coefficients (seeded smooth perturbation of 1), q=2, M=6, dt = 0.1 h,
    8 Ricker shots at seeded positions in [0.2, 0.8]^3, 32 receivers per face
    (192), `adjoint_steps` FP64 leapfrog steps with checkpoints every 50, CG rtol
    1e-13, CG start of order `cg_guess` in every sweep, FP64 solves by iterative
    refinement (FP64 residual, FP32 Jacobi-PCG corrections; --adjoint-cg: FP64
    Jacobi-PCG throughout).  Observed traces come from a
    second coefficient field through the same
    forward path.  Timed: J and its gradient through the torch.autograd.Function
    (assembly, forward with checkpoints, reverse sweep with recomputation).
    Check: central difference with eps = 1e-6 along one seeded direction against
    <grad, v>.
    """
    import numpy as np
    import torch

    import inputs
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300.autograd import misfit
    n_el, nsteps, nshot = 64, args.adjoint_steps, 8
    dt = 0.1 / n_el
    theta = inputs.theta_smooth(n=12, dim=3)
    theta_obs = inputs.theta_smooth(n=12, dim=3, seed=inputs.SEED_THETA_OBS)
    src = inputs.shot_positions(nshot, dim=3, lo=0.2, hi=0.8, seed=inputs.SEED_SHOTS_3D)
    rec = inputs.face_receivers(per_face=32)
    sp = iga.iga_space_create(3, 2, n_el, iga.IGA_MAP_CUBE_SINE, 0.1, iga.IGA_COEF_BSPLINE, 0.0,
                              theta=inputs.colex(theta_obs), n_theta=12, theta_degree=3)
    ops = iga.iga_surrogate_assemble(sp, 2, 2, 6)
    sflags = 0 if args.adjoint_cg else iga.IGA_SOLVE_REFINE
    wv = iga.iga_wave_create(ops, nshot, iga.IGA_F64, dt, src_pos=src, f0=10.0, t0=0.1, rec_pos=rec,
                             nsteps_max=nsteps, cg_rtol=1e-13, cg_max_it=5000, cfl_check=1,
                             cg_guess=args.cg_guess, solve_flags=sflags)
    iga.iga_wave_step(wv, nsteps)
    obs = iga.iga_wave_traces(wv, nshot, len(rec), nsteps)
    st = iga.iga_wave_stats_get(wv)
    lam_min, lam_max = st.lambda_min, st.lambda_max
    iga.iga_wave_destroy(wv)
    iga.iga_ops_destroy(ops)
    iga.iga_space_destroy(sp)
    problem = dict(dim=3, p=2, n_el=n_el, map_kind=iga.IGA_MAP_CUBE_SINE, map_param=0.1, q=2, M=6, dt=dt,
                   nsteps=nsteps, checkpoint_every=50, src_pos=src, rec_pos=rec, obs=obs, f0=10.0, t0=0.1,
                   cg_rtol=1e-13, cg_guess=args.cg_guess, solve_flags=sflags)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    J = misfit(th, problem)
    J.backward()
    J = J.detach()
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t
    g = th.grad.numpy().copy()
    v = np.random.default_rng(41).standard_normal(theta.shape)
    eps = 1e-6
    with torch.no_grad():
        Jp = float(misfit(torch.tensor(theta + eps * v), problem))
        Jm = float(misfit(torch.tensor(theta - eps * v), problem))
    fd = (Jp - Jm) / (2 * eps)
    gv = float(np.sum(g * v))
    return {"adjoint_workload": ("cube 64^3 p=2, 12^3 theta, 8 shots x %d FP64 steps, checkpoints every 50, "
                                 "192 receivers, CG start order %d, %s" %
                                 (nsteps, args.cg_guess, "FP64 Jacobi-PCG" if args.adjoint_cg else
                                  "FP64 solves by refinement with FP32 Jacobi-PCG corrections")),
            "adjoint_gradient_s": t_grad, "adjoint_shot_steps_per_s": nshot * nsteps / t_grad,
            "adjoint_J": float(J), "adjoint_grad_dot_v": gv, "adjoint_central_fd": fd,
            "adjoint_fd_rel_error": abs(gv - fd) / max(abs(gv), 1e-300),
            "adjoint_dt_sqrt_lambda_max": dt * float(np.sqrt(max(lam_max, 0.0))),
            "adjoint_lambda_min": lam_min}


# ------------------------------------------------------------------ oracle legs
def oracle_sample(args):
    """The FP64 oracle, as it stands, on a bounded sample of the workload.

    The oracle's assembly of the full workload is true quadrature of every sample
    row (Surrogate()) plus, for every row, true quadrature and surrogate
    evaluation (Surrogate.rows()).  Sampled here:
    (a) true_rows() of `oracle_rows` random sample rows and of `oracle_rows`
        random rows of the full workload -> seconds per quadrated row;
    (b) Surrogate() and Surrogate.rows() of the n_el = 24 version (same p, q, M,
        map, coefficient) on `oracle_rows` rows, minus their true_rows() time ->
        seconds of interpolation and evaluation per row;
    (c) leapfrog: oracle steps of the n_el = 12 version -> seconds per row per step.
    All per-row costs are scaled to the full workload's counts and combined into
    shot-steps/s of one full pass.
    """
    import numpy as np

    from oracle.assembly import true_rows
    from oracle.surrogate import Surrogate, sample_indices
    from oracle.wave import Leapfrog
    from paper_2004_05197_gb300 import workloads as W
    from tests.oracle_cases import oracle_space, oracle_surrogate
    w = W.scaled(args.workload)
    nsteps = args.nsteps or w["steps"]
    sp = oracle_space(w)
    N = sp.N
    rng = np.random.default_rng(0)
    k = args.oracle_rows
    samp = sample_indices(sp.m, sp.p, w["M"])
    n_sample_rows = len(samp) ** sp.dim
    srows = np.stack([rng.choice(samp, k) for _ in range(sp.dim)], axis=1)
    t = time.perf_counter()
    true_rows(sp, srows)
    t_srows = time.perf_counter() - t
    rows = sp.multi(rng.integers(0, N, size=k))
    t = time.perf_counter()
    true_rows(sp, rows)
    t_rows = time.perf_counter() - t
    wm = W.scaled(args.workload, n_el=24)
    spm = oracle_space(wm)
    rows_m = spm.multi(rng.integers(0, spm.N, size=k))
    t = time.perf_counter()
    Sm = Surrogate(spm, wm["q"], wm["M"])
    t_build_m = time.perf_counter() - t
    t = time.perf_counter()
    Sm.rows(rows_m)
    t_srow_m = time.perf_counter() - t
    t = time.perf_counter()
    true_rows(spm, rows_m)
    t_true_m = time.perf_counter() - t
    n_samp_m = len(Sm.samp) ** spm.dim
    ks = min(k, n_samp_m)
    srows_m = np.stack([rng.choice(Sm.samp, ks) for _ in range(spm.dim)], axis=1)
    t = time.perf_counter()
    true_rows(spm, srows_m)
    t_samp_m = (time.perf_counter() - t) * n_samp_m / ks           # sample quadrature inside Surrogate()
    eval_s = max(t_srow_m - t_true_m, 0.0) / k                     # evaluation per row
    interp_s = max(t_build_m - t_samp_m, 0.0)                       # interpolation (tiny)
    asm_s = n_sample_rows * t_srows / k + interp_s + N * (t_rows / k + eval_s)
    ws = W.scaled(args.workload, n_el=12, M=2)
    sps, Ss = oracle_surrogate(ws)
    SK, SM = Ss.rows(sps.all_rows())
    lf = Leapfrog(sps, SK, SM, W.dt_of(ws), rtol=1e-10, max_it=args.cg_max_it)
    u0 = np.zeros(sps.N)
    steps_small = args.oracle_steps
    t = time.perf_counter()
    lf.run(u0, steps_small, sources=[(W.source_position(ws), 10.0, 0.1, 1.0)])
    t_small = time.perf_counter() - t
    step_s = t_small / steps_small * N / sps.N
    total = asm_s + nsteps * step_s
    sample_s = t_srows + t_rows + t_build_m + t_srow_m + t_true_m + t_small
    return {"value": args.nshot * nsteps / total, "unit": "shot-steps/s", "cores": 1, "kind": "oracle",
            "sample": ("oracle true-row quadrature of %d random sample rows and %d random rows of the full "
                       "workload (%.1f s; scaled to %d sample rows and N=%d rows), surrogate interpolation "
                       "and evaluation of %d rows of the n_el=24 version (%.1f s; scaled by N), and %d "
                       "oracle leapfrog steps of the n_el=12 version (%.1f s; scaled by N); full pass "
                       "estimated at %.0f s" % (k, k, t_srows + t_rows, n_sample_rows, N, k,
                                               t_build_m + t_srow_m + t_true_m, steps_small, t_small, total)),
            "surrogate_rows_per_s": N / asm_s, "sample_seconds": sample_s,
            "_parts": {"N": N, "n_sample_rows": n_sample_rows, "interp_s": interp_s, "step_s": step_s,
                       "nsteps": nsteps, "k": k}}


def _oracle_rows_chunk(args):
    """Surrogate.rows() of a chunk of rows (a process-pool task)."""
    S, rows = args
    return S.rows(rows)


def oracle_sample_all_cores(args, single):
    """The oracle's row-parallel parts on all host cores: true-row quadrature and surrogate
    evaluation of `oracle_rows` x nproc random rows split over a process pool of nproc
    workers (spawn start, the same per-row arithmetic), scaled to the full workload as in
    the single-thread sample; the leapfrog part stays the single-thread measurement (one
    shot, sparse products on one core).  Returns the cpu_baseline object of that run."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np

    from oracle.surrogate import Surrogate, _true_rows_chunk
    from paper_2004_05197_gb300 import workloads as W
    from tests.oracle_cases import oracle_space
    nproc = os.cpu_count() or 1
    parts = single["_parts"]
    w = W.scaled(args.workload)
    sp = oracle_space(w)
    rng = np.random.default_rng(1)
    kk = parts["k"] * nproc
    rows = sp.multi(rng.integers(0, sp.N, size=kk))
    wm = W.scaled(args.workload, n_el=24)
    spm = oracle_space(wm)
    Sm = Surrogate(spm, wm["q"], wm["M"])
    rows_m = spm.multi(rng.integers(0, spm.N, size=kk))
    with cf.ProcessPoolExecutor(nproc, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_true_rows_chunk, [(sp, rows[:2])] * nproc))          # start-up of the workers
        t = time.perf_counter()
        list(ex.map(_true_rows_chunk, [(sp, c) for c in np.array_split(rows, nproc)]))
        t_rows = time.perf_counter() - t
        t = time.perf_counter()
        list(ex.map(_oracle_rows_chunk, [(Sm, c) for c in np.array_split(rows_m, nproc)]))
        t_srow = time.perf_counter() - t
        t = time.perf_counter()
        list(ex.map(_true_rows_chunk, [(spm, c) for c in np.array_split(rows_m, nproc)]))
        t_true = time.perf_counter() - t
    per_row = t_rows / kk
    eval_s = max(t_srow - t_true, 0.0) / kk
    N = parts["N"]
    asm_s = (parts["n_sample_rows"] + N) * per_row + parts["interp_s"] + N * eval_s
    total = asm_s + parts["nsteps"] * parts["step_s"]
    return {"value": args.nshot * parts["nsteps"] / total, "unit": "shot-steps/s", "cores": nproc, "kind": "oracle",
            "sample": ("the single-thread sample with its quadrature and evaluation parts re-run on %d cores "
                       "(%d random rows each, process pool; %.1f s + %.1f s); the leapfrog part single-core; "
                       "full pass estimated at %.0f s" % (nproc, kk, t_rows, t_srow + t_true, total)),
            "surrogate_rows_per_s": N / asm_s}


def workload_config(args, world=1):
    """The `config` object of both arms: the workload and the settings of the timed pass
    (host-side arithmetic only)."""
    from paper_2004_05197_gb300 import workloads as W
    w = W.scaled(args.workload)
    nsteps = args.nsteps or w["steps"]
    m = w["n_el"] + w["p"]
    N = m ** w["dim"]
    D = (2 * w["p"] + 1) ** w["dim"]
    pitch = (N + 63) // 64 * 64
    return {"workload": args.workload, "dim": w["dim"], "p": w["p"], "n_el": w["n_el"], "N": N,
            "q": w["q"], "M": w["M"], "nsteps": nsteps, "nshot": args.nshot, "cg_rtol": args.cg_rtol,
            "cg_schedule": args.solve,
            "cg_start": ("previous acceleration" if args.cg_guess == 0 else
                         "polynomial extrapolation in time, order %d" % args.cg_guess),
            "precision": "FP32 fields/vectors/apply, FP64 quadrature (band contractions in double-float FP32 pairs), residual in FP64 (row kernels) or as an FP32 pair (brick PCG), compensated dot products",
            "l2": "inputs larger than L2 (stencil fields %.2f GB)" % (D * pitch * 12 / 1e9),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, one bounded sample per step."""
    for _ in range(args.warmup):
        oracle_sample(args)
    vals, secs = [], []
    for _ in range(args.steps):
        t = time.perf_counter()
        r = oracle_sample(args)
        secs.append(time.perf_counter() - t)
        vals.append(r["value"])
    v = sorted(vals)[len(vals) // 2]
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "shot-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": "shot-steps/s", "cores": 1, "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": "shot-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube96_p2")
    ap.add_argument("--nsteps", type=int, default=0, help="time steps per pass (default: the workload's)")
    ap.add_argument("--nshot", type=int, default=1)
    ap.add_argument("--cg-rtol", type=float, default=1e-6)
    ap.add_argument("--cg-max-it", type=int, default=2000)
    ap.add_argument("--cg-guess", type=int, default=3, choices=range(7),
                    help="CG start of each step: polynomial extrapolation in time of this order (0: a^{n-1})")
    ap.add_argument("--solve", default="persistent", choices=["persistent", "graph"],
                    help="CG schedule of the FP32 waves")
    ap.add_argument("--compare-steps", type=int, default=50,
                    help="steps of the FP64 plain and graph single-shot rates (the persistent FP64 wave runs all steps)")
    ap.add_argument("--config2-steps", type=int, default=2000,
                    help="steps of the 2-D p=3 annulus 512^2 leg (0: skip it)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--oracle-rows", type=int, default=96)
    ap.add_argument("--oracle-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the oracle's row-parallel parts on all host cores")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched multi-mesh leg")
    ap.add_argument("--batched-steps", type=int, default=1000)
    ap.add_argument("--batched-rtol", type=float, default=3e-7,
                    help="CG tolerance of the batched FP32 shots (the CG term of the FP32 error is about 15 rtol after 1000 steps)")
    ap.add_argument("--batched-cg-guess", type=int, default=3, choices=range(7),
                    help="CG start order of the batched leg and of its plain FP64 comparison")
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--next-rows", action="store_true",
                    help="also measure the volume-preserving mass and the multi-patch operators")
    ap.add_argument("--msweep", action="store_true",
                    help="also run the sampling-length study: fixed M against M(h) over five cube meshes")
    ap.add_argument("--adjoint", action="store_true",
                    help="also run the adjoint-gradient leg (several minutes: FP64 forward / reverse sweeps)")
    ap.add_argument("--adjoint-steps", type=int, default=600)
    ap.add_argument("--adjoint-cg", action="store_true",
                    help="adjoint leg with FP64 Jacobi-PCG solves instead of refinement")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return 0

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=device)
    import __graft_entry__
    __graft_entry__.build()
    out, ctx = run_ours(args, rank, world, device)
    if rank == 0:
        out["components"].update(stencil_apply_leg(ctx, args))
        if args.next_rows:
            out["components"].update(next_rows_leg(ctx, args))
        if args.msweep:
            out["components"].update(msweep_leg(args))
        if not args.no_compare:
            out["components"].update(fp64_forms_and_error(ctx, args))
        if args.config2_steps > 0:
            out["components"].update(config2_leg(args))
        if args.e2e_steps > 0:
            out["e2e"] = run_e2e(args, ctx)
        if not args.no_batched:
            out["components"].update(run_batched(args))
        if args.adjoint:
            out["components"].update(run_adjoint(args))
        if not args.no_cpu_baseline:
            single = oracle_sample(args)
            if args.cpu_all_cores:
                out["cpu_baseline_all_cores"] = oracle_sample_all_cores(args, single)
            single.pop("_parts", None)
            out["cpu_baseline"] = single
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
