"""Thin ctypes binding of libiga (include/iga.h): argument marshalling only.

Every function keeps the C name.  Device buffers are torch CUDA tensors (their
data_ptr() is passed), host buffers are numpy arrays, streams default to
torch's current CUDA stream.  There is no fallback: if libiga.so is missing or
cannot be loaded, importing this module raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiga.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libiga.so not built: run `python -m paper_2004_05197_gb300.build` "
                      "(or __graft_entry__.build()) first")
_lib = C.CDLL(LIB_PATH)

# ---- constants (include/iga.h) -------------------------------------------------
IGA_OK = 0
IGA_ERR_ARG, IGA_ERR_OOM, IGA_ERR_CUDA = -1, -2, -3
IGA_ERR_NOT_CONVERGED, IGA_ERR_NONFINITE, IGA_ERR_TIMEOUT = -4, -5, -6
IGA_MAP_IDENTITY, IGA_MAP_ANNULUS_QUARTER, IGA_MAP_CUBE_SINE, IGA_MAP_ANNULUS_SECTOR, IGA_MAP_BOX = 0, 1, 2, 3, 4
IGA_COEF_CONST, IGA_COEF_SINCOS, IGA_COEF_BSPLINE = 0, 1, 2
IGA_F32, IGA_F64 = 0, 1
IGA_OP_K, IGA_OP_M = 0, 1
IGA_TRUE_ONLY, IGA_KEEP_SAMPLES, IGA_MASS_VOLUME_PRESERVING = 1, 2, 4
IGA_SOLVE_PLAIN, IGA_SOLVE_GRAPH, IGA_SOLVE_REFINE = 1, 2, 4
IGA_INIT_ZERO, IGA_INIT_GAUSS_PULSE = 0, 1
IGA_PATH_AUTO, IGA_PATH_ROWS, IGA_PATH_BRICK, IGA_PATH_ONTHEFLY = 0, 1, 2, 3

EXPORTED = [
    "iga_space_create", "iga_space_destroy", "iga_space_info_get", "iga_surrogate_assemble",
    "iga_ops_destroy", "iga_ops_info_get", "iga_ops_copy_fields", "iga_ops_copy_samples",
    "iga_ops_sample_indices", "iga_stencil_apply", "iga_mass_solve", "iga_wave_create",
    "iga_wave_destroy", "iga_wave_step", "iga_wave_get_state", "iga_wave_traces",
    "iga_wave_cg_iterations", "iga_last_error", "iga_launch_count", "iga_wave_reset",
    "iga_wave_set_timing", "iga_wave_stats_get", "iga_ops_spectrum", "iga_wave_adjoint",
    "iga_batch_create", "iga_batch_destroy", "iga_batch_step", "iga_batch_tune", "iga_batch_partition",
    "iga_mass_solve_noalloc", "iga_sampling_length_for_mesh",
    "iga_multipatch_create", "iga_multipatch_destroy", "iga_multipatch_size", "iga_multipatch_global_index",
    "iga_multipatch_apply", "iga_multipatch_mass_solve", "iga_multipatch_leapfrog", "iga_ops_set_path",
    "iga_ops_brick_info",
    "iga_barrier_selftest",
]


class IgaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libiga error %d: %s" % (code, msg))
        self.code = code


class iga_space_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("n_el", C.c_int), ("map_kind", C.c_int),
                ("map_param", C.c_double), ("coef_kind", C.c_int), ("coef_param", C.c_double),
                ("theta", C.POINTER(C.c_double)), ("n_theta", C.c_int), ("theta_degree", C.c_int),
                ("quad_pts", C.c_int), ("sector", C.c_double * 4), ("box", C.c_double * 6)]


class iga_space_info(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("n_el", C.c_int), ("m", C.c_int),
                ("N", C.c_longlong), ("D", C.c_int), ("nK", C.c_int), ("nM", C.c_int),
                ("interior_lo", C.c_int), ("interior_hi", C.c_int)]


class iga_ops_info(C.Structure):
    _fields_ = [("N", C.c_longlong), ("pitch", C.c_longlong), ("m", C.c_int), ("dim", C.c_int),
                ("p", C.c_int), ("q", C.c_int), ("M", C.c_int), ("nK", C.c_int), ("nM", C.c_int),
                ("D", C.c_int), ("ns", C.c_int), ("n_band_elements", C.c_int),
                ("n_sample_rows", C.c_int), ("t_sample_ms", C.c_double), ("t_band_ms", C.c_double),
                ("t_interp_ms", C.c_double), ("t_eval_ms", C.c_double), ("t_total_ms", C.c_double),
                ("workspace_bytes", C.c_longlong)]


class iga_interface(C.Structure):
    _fields_ = [("patch_a", C.c_int), ("side_a", C.c_int), ("patch_b", C.c_int), ("side_b", C.c_int),
                ("reversed", C.c_int)]


class iga_wave_desc(C.Structure):
    _fields_ = [("nshot", C.c_int), ("dtype", C.c_int), ("solve_flags", C.c_uint), ("dt", C.c_double),
                ("init_kind", C.c_int), ("pulse_centre", C.POINTER(C.c_double)),
                ("pulse_width", C.c_double), ("with_source", C.c_int),
                ("src_pos", C.POINTER(C.c_double)), ("f0", C.c_double), ("t0", C.c_double),
                ("src_amp", C.c_double), ("nrec", C.c_int), ("rec_pos", C.POINTER(C.c_double)),
                ("nsteps_max", C.c_int), ("cg_rtol", C.c_double), ("cg_max_it", C.c_int),
                ("cfl_check", C.c_int), ("cg_guess", C.c_int)]


class iga_wave_stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("cg_iterations", C.c_longlong), ("cg_solves", C.c_longlong),
                ("cg_ms", C.c_double), ("force_ms", C.c_double), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double)]


_vp, _i, _u, _d = C.c_void_p, C.c_int, C.c_uint, C.c_double
_sig = {
    "iga_space_create": [C.POINTER(iga_space_desc), C.POINTER(_vp)],
    "iga_space_destroy": [_vp],
    "iga_space_info_get": [_vp, C.POINTER(iga_space_info)],
    "iga_surrogate_assemble": [_vp, _i, _i, _i, _u, _vp, C.POINTER(_vp)],
    "iga_ops_destroy": [_vp],
    "iga_ops_info_get": [_vp, C.POINTER(iga_ops_info)],
    "iga_ops_copy_fields": [_vp, _i, _i, _vp, _vp],
    "iga_ops_copy_samples": [_vp, _i, _vp, _vp],
    "iga_ops_sample_indices": [_vp, C.POINTER(_i)],
    "iga_stencil_apply": [_vp, _i, _i, _vp, _vp, _i, _vp],
    "iga_ops_set_path": [_vp, _i],
    "iga_barrier_selftest": [_i, _i, _d, _vp],
    "iga_ops_brick_info": [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)],
    "iga_mass_solve": [_vp, _i, _vp, _vp, _i, _d, _i, _u, C.POINTER(_i), C.POINTER(_d), _vp],
    "iga_multipatch_create": [_i, C.POINTER(_vp), _i, C.POINTER(iga_interface), C.POINTER(_vp)],
    "iga_multipatch_destroy": [_vp],
    "iga_multipatch_size": [_vp, C.POINTER(C.c_longlong)],
    "iga_multipatch_global_index": [_vp, _i, C.POINTER(C.c_longlong)],
    "iga_multipatch_apply": [_vp, _i, _i, _vp, _vp, _i, _vp],
    "iga_multipatch_mass_solve": [_vp, _i, _vp, _vp, _i, _d, _i, C.POINTER(_i), C.POINTER(_d), _vp],
    "iga_multipatch_leapfrog": [_vp, _i, _d, _i, _vp, _i, C.POINTER(_d), _d, _d, _d, _i, C.POINTER(_i),
                                C.POINTER(_d), C.POINTER(_d), _d, _i, C.POINTER(C.c_longlong), _vp],
    "iga_sampling_length_for_mesh": [_d, _i, _i, _d, _d, _d, _d, C.POINTER(_i)],
    "iga_mass_solve_noalloc": [_vp, _i, _vp, _vp, _i, _d, _i, _u, C.POINTER(_i), C.POINTER(_d), _vp],
    "iga_wave_create": [_vp, C.POINTER(iga_wave_desc), C.POINTER(_vp)],
    "iga_wave_destroy": [_vp],
    "iga_wave_step": [_vp, _i, _vp],
    "iga_wave_get_state": [_vp, _vp, _vp, _vp],
    "iga_wave_traces": [_vp, C.POINTER(_d), C.POINTER(_i)],
    "iga_wave_cg_iterations": [_vp, C.POINTER(C.c_longlong)],
    "iga_wave_reset": [_vp, _vp, _vp],
    "iga_wave_set_timing": [_vp, _i],
    "iga_wave_stats_get": [_vp, C.POINTER(iga_wave_stats)],
    "iga_ops_spectrum": [_vp, _i, _i, C.POINTER(_d), C.POINTER(_d), _vp],
    "iga_wave_adjoint": [_vp, _i, _i, C.POINTER(_d), C.POINTER(_d), C.POINTER(_d), _vp],
    "iga_batch_create": [_i, C.POINTER(_vp), C.POINTER(_vp)],
    "iga_batch_destroy": [_vp],
    "iga_batch_step": [_vp, _i, _i, _vp],
    "iga_batch_tune": [_vp, _i, _i, _vp],
    "iga_batch_partition": [_vp, C.POINTER(_i)],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.iga_last_error.argtypes = []
_lib.iga_last_error.restype = C.c_char_p
_lib.iga_launch_count.argtypes = []
_lib.iga_launch_count.restype = C.c_longlong


def iga_last_error():
    return _lib.iga_last_error().decode()


def iga_launch_count():
    return int(_lib.iga_launch_count())


def _check(rc, ok=(IGA_OK,)):
    if rc not in ok:
        raise IgaError(rc, iga_last_error())
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _host_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


# ---- space ---------------------------------------------------------------------
def iga_space_create(dim, p, n_el, map_kind, map_param=0.0, coef_kind=IGA_COEF_CONST, coef_param=1.0,
                     theta=None, n_theta=0, theta_degree=3, quad_pts=0, sector=(0.0, 0.0, 0.0, 0.0),
                     box=(0.0, 0.0, 0.0, 1.0, 1.0, 1.0)):
    """theta: host array, colex flat (first parametric direction fastest);
    sector: (r0, r1, a0, a1) of IGA_MAP_ANNULUS_SECTOR; box: (o1, o2, o3, e1, e2, e3) of
    IGA_MAP_BOX."""
    keep = None
    tptr = C.POINTER(C.c_double)()
    if theta is not None:
        keep, tptr = _host_f64(np.asarray(theta).ravel())
    desc = iga_space_desc(dim, p, n_el, map_kind, map_param, coef_kind, coef_param, tptr, n_theta,
                          theta_degree, quad_pts, (C.c_double * 4)(*sector), (C.c_double * 6)(*box))
    out = C.c_void_p()
    _check(_lib.iga_space_create(C.byref(desc), C.byref(out)))
    del keep
    return out


def iga_space_destroy(space):
    _check(_lib.iga_space_destroy(space))


def iga_space_info_get(space):
    info = iga_space_info()
    _check(_lib.iga_space_info_get(space, C.byref(info)))
    return info


# ---- assembly ------------------------------------------------------------------
def iga_surrogate_assemble(space, p, q, M, flags=0, stream=None):
    out = C.c_void_p()
    _check(_lib.iga_surrogate_assemble(space, p, q, M, flags, _stream(stream), C.byref(out)))
    return out


def iga_ops_destroy(ops):
    _check(_lib.iga_ops_destroy(ops))


def iga_ops_info_get(ops):
    info = iga_ops_info()
    _check(_lib.iga_ops_info_get(ops, C.byref(info)))
    return info


def iga_ops_copy_fields(ops, which, dtype, dst, stream=None):
    _check(_lib.iga_ops_copy_fields(ops, which, dtype, _dptr(dst), _stream(stream)))


def iga_ops_copy_samples(ops, which, dst, stream=None):
    _check(_lib.iga_ops_copy_samples(ops, which, _dptr(dst), _stream(stream)))


def iga_ops_sample_indices(ops):
    ns = iga_ops_info_get(ops).ns
    buf = (C.c_int * max(ns, 1))()
    _check(_lib.iga_ops_sample_indices(ops, buf))
    return np.array(buf[:ns], dtype=np.int64)


def iga_sampling_length_for_mesh(h, p, q, a=0.0, b=0.0, C_=1.0, eps=0.1):
    out = C.c_int()
    _check(_lib.iga_sampling_length_for_mesh(h, p, q, a, b, C_, eps, C.byref(out)))
    return out.value


# ---- operators -----------------------------------------------------------------
def iga_stencil_apply(ops, which, dtype, x, y, nrhs, stream=None):
    _check(_lib.iga_stencil_apply(ops, which, dtype, _dptr(x), _dptr(y), nrhs, _stream(stream)))


def iga_ops_set_path(ops, path):
    _check(_lib.iga_ops_set_path(ops, path))


def iga_ops_brick_info(ops, with_paths=False):
    """(bricks, threads per CTA, ring stages, shared-memory bytes per CTA[, brick_paths]);
    zeros without a brick form.  brick_paths: bit 0 K~ apply, bit 1 M~ apply and mass solve."""
    v = [C.c_int() for _ in range(5)]
    _check(_lib.iga_ops_brick_info(ops, *[C.byref(t) for t in v]))
    out = tuple(t.value for t in v)
    return out if with_paths else out[:4]


def iga_barrier_selftest(blocks, expected, limit_ms, stream=None):
    """Status code of the bounded grid-barrier self-test (IGA_OK or IGA_ERR_TIMEOUT)."""
    return _check(_lib.iga_barrier_selftest(blocks, expected, limit_ms, _stream(stream)),
                  (IGA_OK, IGA_ERR_TIMEOUT))


def iga_mass_solve(ops, dtype, b, x, nrhs, rtol, max_it, flags=0, want_stats=True, stream=None,
                   allow_not_converged=False):
    iters = (C.c_int * nrhs)() if want_stats else None
    rel = (C.c_double * nrhs)() if want_stats else None
    ok = (IGA_OK, IGA_ERR_NOT_CONVERGED) if allow_not_converged else (IGA_OK,)
    rc = _check(_lib.iga_mass_solve(ops, dtype, _dptr(b), _dptr(x), nrhs, rtol, max_it, flags,
                                    iters, rel, _stream(stream)), ok)
    if want_stats:
        return rc, np.array(iters[:]), np.array(rel[:])
    return rc, None, None


IGA_NOALLOC_SCRATCH_BYTES = 64 << 20


def iga_mass_solve_noalloc(ops, dtype, b, x, nrhs, rtol, max_it, flags=0, want_stats=True, stream=None,
                           allow_not_converged=False):
    """iga_mass_solve with the CG workspace in the library's fixed device array (no allocation)."""
    iters = (C.c_int * nrhs)() if want_stats else None
    rel = (C.c_double * nrhs)() if want_stats else None
    ok = (IGA_OK, IGA_ERR_NOT_CONVERGED) if allow_not_converged else (IGA_OK,)
    rc = _check(_lib.iga_mass_solve_noalloc(ops, dtype, _dptr(b), _dptr(x), nrhs, rtol, max_it, flags,
                                            iters, rel, _stream(stream)), ok)
    if want_stats:
        return rc, np.array(iters[:]), np.array(rel[:])
    return rc, None, None


# ---- multi-patch -----------------------------------------------------------------
def iga_multipatch_create(patch_ops, interfaces):
    """patch_ops: list of iga_ops handles; interfaces: (patch_a, side_a, patch_b, side_b, reversed)."""
    arr = (C.c_void_p * len(patch_ops))(*[o.value if isinstance(o, C.c_void_p) else o for o in patch_ops])
    ifs = (iga_interface * max(1, len(interfaces)))(*[iga_interface(*t) for t in interfaces])
    out = C.c_void_p()
    _check(_lib.iga_multipatch_create(len(patch_ops), arr, len(interfaces), ifs, C.byref(out)))
    return out


def iga_multipatch_destroy(mp):
    _check(_lib.iga_multipatch_destroy(mp))


def iga_multipatch_size(mp):
    n = C.c_longlong()
    _check(_lib.iga_multipatch_size(mp, C.byref(n)))
    return int(n.value)


def iga_multipatch_global_index(mp, patch, n_local):
    out = np.zeros(n_local, dtype=np.int64)
    _check(_lib.iga_multipatch_global_index(mp, patch, out.ctypes.data_as(C.POINTER(C.c_longlong))))
    return out


def iga_multipatch_apply(mp, which, dtype, x, y, nrhs, stream=None):
    _check(_lib.iga_multipatch_apply(mp, which, dtype, _dptr(x), _dptr(y), nrhs, _stream(stream)))


def iga_multipatch_mass_solve(mp, dtype, b, x, nrhs, rtol, max_it, stream=None, allow_not_converged=False):
    iters = (C.c_int * nrhs)()
    rel = (C.c_double * nrhs)()
    ok = (IGA_OK, IGA_ERR_NOT_CONVERGED) if allow_not_converged else (IGA_OK,)
    rc = _check(_lib.iga_multipatch_mass_solve(mp, dtype, _dptr(b), _dptr(x), nrhs, rtol, max_it, iters, rel,
                                               _stream(stream)), ok)
    return rc, np.array(iters[:]), np.array(rel[:])


def iga_multipatch_leapfrog(mp, dtype, dt, nsteps, u, src_patch=-1, src_s=None, f0=10.0, t0=0.1, amp=1.0,
                            rec_patch=(), rec_s=None, cg_rtol=1e-10, cg_max_it=1000, stream=None):
    """u: device [n_global] (u^0 in, u^nsteps out); src_s: [dim]; rec_patch: [nrec];
    rec_s: [nrec][dim].  Returns (traces [nrec][nsteps], CG iterations summed over steps)."""
    nrec = len(rec_patch)
    keep = []
    sp = C.POINTER(C.c_double)()
    if src_s is not None:
        a, sp = _host_f64(np.asarray(src_s, dtype=np.float64).ravel())
        keep.append(a)
    rp = (C.c_int * max(1, nrec))(*[int(r) for r in rec_patch])
    rs = C.POINTER(C.c_double)()
    if nrec:
        a, rs = _host_f64(np.asarray(rec_s, dtype=np.float64).ravel())
        keep.append(a)
    tr = np.zeros((nrec, nsteps), dtype=np.float64)
    it = C.c_longlong(0)
    _check(_lib.iga_multipatch_leapfrog(mp, dtype, dt, nsteps, _dptr(u), src_patch, sp, f0, t0, amp, nrec, rp, rs,
                                        tr.ctypes.data_as(C.POINTER(C.c_double)), cg_rtol, cg_max_it, C.byref(it),
                                        _stream(stream)))
    del keep
    return tr, it.value


# ---- waves ---------------------------------------------------------------------
def iga_wave_create(ops, nshot, dtype, dt, init_kind=IGA_INIT_ZERO, pulse_centre=None, pulse_width=0.05,
                    src_pos=None, f0=10.0, t0=0.1, src_amp=1.0, rec_pos=None, nsteps_max=0,
                    cg_rtol=1e-10, cg_max_it=1000, solve_flags=0, cfl_check=1, cg_guess=0):
    keep = []

    def hp(a):
        if a is None:
            return C.POINTER(C.c_double)()
        arr, ptr = _host_f64(a)
        keep.append(arr)
        return ptr

    nrec = 0 if rec_pos is None else int(np.asarray(rec_pos).shape[0])
    desc = iga_wave_desc(nshot, dtype, solve_flags, dt, init_kind, hp(pulse_centre), pulse_width,
                         1 if src_pos is not None else 0, hp(src_pos), f0, t0, src_amp, nrec,
                         hp(rec_pos), nsteps_max, cg_rtol, cg_max_it, cfl_check, cg_guess)
    out = C.c_void_p()
    _check(_lib.iga_wave_create(ops, C.byref(desc), C.byref(out)))
    return out


def iga_wave_destroy(wave):
    _check(_lib.iga_wave_destroy(wave))


def iga_wave_step(wave, nsteps, stream=None):
    return _check(_lib.iga_wave_step(wave, nsteps, _stream(stream)))


def iga_wave_get_state(wave, u, u_prev=None, stream=None):
    _check(_lib.iga_wave_get_state(wave, _dptr(u), _dptr(u_prev), _stream(stream)))


def iga_wave_traces(wave, nshot, nrec, nsteps):
    out = np.zeros((nshot, nrec, nsteps), dtype=np.float64)
    done = C.c_int()
    _check(_lib.iga_wave_traces(wave, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(done)))
    return out[:, :, :done.value]


def iga_wave_cg_iterations(wave):
    tot = C.c_longlong()
    _check(_lib.iga_wave_cg_iterations(wave, C.byref(tot)))
    return int(tot.value)


def iga_wave_reset(wave, ops, stream=None):
    _check(_lib.iga_wave_reset(wave, ops, _stream(stream)))


def iga_wave_set_timing(wave, on=True):
    _check(_lib.iga_wave_set_timing(wave, 1 if on else 0))


def iga_wave_stats_get(wave):
    st = iga_wave_stats()
    _check(_lib.iga_wave_stats_get(wave, C.byref(st)))
    return st


def iga_ops_spectrum(ops, dtype=IGA_F64, k=40, stream=None):
    """(lambda_min, lambda_max) of the pencil (K~, M~) by k Lanczos steps."""
    lo, hi = C.c_double(), C.c_double()
    _check(_lib.iga_ops_spectrum(ops, dtype, k, C.byref(lo), C.byref(hi), _stream(stream)))
    return lo.value, hi.value


def iga_wave_adjoint(wave, nsteps, checkpoint_every, obs, n_theta_total=0, stream=None):
    """(J, grad_theta or None); obs host [nshot][nrec][nsteps]."""
    obs_a, obs_p = _host_f64(obs)
    J = C.c_double()
    grad = np.zeros(n_theta_total) if n_theta_total else None
    gp = grad.ctypes.data_as(C.POINTER(C.c_double)) if grad is not None else C.POINTER(C.c_double)()
    _check(_lib.iga_wave_adjoint(wave, nsteps, checkpoint_every, obs_p, C.byref(J), gp, _stream(stream)))
    del obs_a
    return J.value, grad


def iga_batch_create(waves):
    arr = (C.c_void_p * len(waves))(*[w.value if isinstance(w, C.c_void_p) else w for w in waves])
    out = C.c_void_p()
    _check(_lib.iga_batch_create(len(waves), arr, C.byref(out)))
    return out


def iga_batch_destroy(batch):
    _check(_lib.iga_batch_destroy(batch))


def iga_batch_step(batch, nsteps, use_graph=True, stream=None):
    _check(_lib.iga_batch_step(batch, nsteps, 1 if use_graph else 0, _stream(stream)))


def iga_batch_tune(batch, trial_steps=5, rounds=3, stream=None):
    _check(_lib.iga_batch_tune(batch, trial_steps, rounds, _stream(stream)))


def iga_batch_partition(batch, nprob):
    buf = (C.c_int * nprob)()
    _check(_lib.iga_batch_partition(batch, buf))
    return list(buf)
