"""iga_mass_solve_noalloc (workspace in the library's fixed device array) against
iga_mass_solve (library-allocated workspace) on the same seeded inputs.

Both entry points run the same solver, so the tolerance is the one the other
GPU tests use for the CG paths: 1e-12 relative for FP64, 2e-5 for FP32.  Each
case calls the no-alloc entry twice in a row, so the second call runs on
scratch the first one left behind.  On an ops that never ran iga_mass_solve,
the no-alloc calls leave the library's CG workspace at zero bytes and, after a
first call, do not change the device's free memory.  The file sorts last so that
the suite also exercises the entry point after every other test has used the
device.
"""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

TOL = {"f64": 1e-12, "f32": 2e-5}


def _ops(name, **kw):
    w = W.scaled(name, **kw)
    space = W.make_space(w)
    return space, iga.iga_surrogate_assemble(space, w["p"], w["q"], w["M"], 0)


def _rhs(N, nrhs, tdt):
    b = inputs.vectors(N, nrhs).reshape(nrhs, N)
    return torch.tensor(b, dtype=tdt, device="cuda")


@pytest.mark.parametrize("dtype,nrhs", [("f64", 5), ("f64", 1), ("f32", 3)])
def test_noalloc_matches_allocating_solve_twice(dtype, nrhs):
    space, ops = _ops("annulus64_p2")
    try:
        N = iga.iga_ops_info_get(ops).N
        dt = iga.IGA_F64 if dtype == "f64" else iga.IGA_F32
        tdt = torch.float64 if dtype == "f64" else torch.float32
        rtol = 1e-12 if dtype == "f64" else 1e-6
        b = _rhs(N, nrhs, tdt)
        x_ref = torch.zeros_like(b)
        _, it_ref, rel_ref = iga.iga_mass_solve(ops, dt, b, x_ref, nrhs, rtol, 2000)
        torch.cuda.synchronize()
        scale = x_ref.abs().max().item()
        for call in range(2):
            x = torch.zeros_like(b)
            _, it, rel = iga.iga_mass_solve_noalloc(ops, dt, b, x, nrhs, rtol, 2000)
            torch.cuda.synchronize()
            err = (x - x_ref).abs().max().item() / scale
            assert err <= TOL[dtype], (call, err)
            assert np.array_equal(it, it_ref), (call, it, it_ref)
            assert np.all(rel <= rtol), (call, rel)
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(space)


def test_noalloc_rejects_workspace_beyond_the_fixed_array():
    # cube with n_el = 76, p = 2: N = 78^3 = 474552 rows; four FP64 right-hand sides
    # need about 160 N = 76 MB of CG workspace, more than the fixed 64 MiB.
    space, ops = _ops("cube96_p2", n_el=76)
    try:
        N = iga.iga_ops_info_get(ops).N
        assert 160 * N > iga.IGA_NOALLOC_SCRATCH_BYTES
        b = _rhs(N, 4, torch.float64)
        x = torch.full_like(b, 3.0)
        with pytest.raises(iga.IgaError) as ei:
            iga.iga_mass_solve_noalloc(ops, iga.IGA_F64, b, x, 4, 1e-8, 100)
        assert ei.value.code == iga.IGA_ERR_ARG
        assert "scratch" in iga.iga_last_error()
        torch.cuda.synchronize()
        assert bool((x == 3.0).all())
        # a single FP64 right-hand side of the same mesh fits (about 40 N bytes)
        x1 = torch.zeros_like(b[:1])
        x1_ref = torch.zeros_like(b[:1])
        iga.iga_mass_solve_noalloc(ops, iga.IGA_F64, b[:1], x1, 1, 1e-10, 2000)
        iga.iga_mass_solve(ops, iga.IGA_F64, b[:1], x1_ref, 1, 1e-10, 2000)
        torch.cuda.synchronize()
        err = (x1 - x1_ref).abs().max().item() / x1_ref.abs().max().item()
        assert err <= TOL["f64"], err
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(space)


@pytest.mark.parametrize("flags", [0, 1])   # default (persistent) and IGA_SOLVE_PLAIN schedules
def test_noalloc_allocates_nothing_on_a_fresh_ops(flags):
    space, ops = _ops("annulus64_p2")
    try:
        N = iga.iga_ops_info_get(ops).N
        b = _rhs(N, 1, torch.float64)
        # every tensor is allocated before free memory is read (torch's caching allocator
        # would otherwise show up in the reading)
        x0, x_ref = torch.zeros_like(b), torch.zeros_like(b)
        xs = [torch.zeros_like(b) for _ in range(2)]
        iga.iga_mass_solve_noalloc(ops, iga.IGA_F64, b, x0, 1, 1e-12, 2000, flags=flags)   # first call: set-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for x in xs:
            iga.iga_mass_solve_noalloc(ops, iga.IGA_F64, b, x, 1, 1e-12, 2000, flags=flags)
            torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert iga.iga_ops_info_get(ops).workspace_bytes == 0
        iga.iga_mass_solve(ops, iga.IGA_F64, b, x_ref, 1, 1e-12, 2000, flags=flags)
        torch.cuda.synchronize()
        assert iga.iga_ops_info_get(ops).workspace_bytes > 0
        scale = x_ref.abs().max().item()
        for x in xs:
            assert (x - x_ref).abs().max().item() <= TOL["f64"] * scale
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(space)


def test_noalloc_rejects_the_graph_schedule():
    space, ops = _ops("annulus64_p2")
    try:
        N = iga.iga_ops_info_get(ops).N
        b = _rhs(N, 1, torch.float64)
        x = torch.zeros_like(b)
        with pytest.raises(iga.IgaError) as ei:
            iga.iga_mass_solve_noalloc(ops, iga.IGA_F64, b, x, 1, 1e-12, 2000, flags=iga.IGA_SOLVE_GRAPH)
        assert ei.value.code == iga.IGA_ERR_ARG
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(space)


@pytest.mark.parametrize("entry", ["noalloc", "alloc"])
def test_missed_tolerance_is_returned_without_statistics(entry):
    """No statistics arrays (NULL iters_out / relres_out): the call still reports
    IGA_ERR_NOT_CONVERGED when max_it = 2 cannot reach rtol."""
    space, ops = _ops("annulus64_p2")
    try:
        N = iga.iga_ops_info_get(ops).N
        b = _rhs(N, 1, torch.float64)
        x = torch.zeros_like(b)
        fn = iga.iga_mass_solve_noalloc if entry == "noalloc" else iga.iga_mass_solve
        rc, _, _ = fn(ops, iga.IGA_F64, b, x, 1, 1e-12, 2, want_stats=False, allow_not_converged=True)
        assert rc == iga.IGA_ERR_NOT_CONVERGED
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(space)
