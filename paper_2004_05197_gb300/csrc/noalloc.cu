// iga_mass_solve_noalloc: the Jacobi-PCG mass solve of iga_mass_solve with its
// CG workspace in a fixed device array compiled into the library, so that a
// call allocates no device memory.  The solver itself (kernels, schedule,
// convergence test, results) is the one iga_mass_solve runs; only where the
// workspace comes from differs.
//
// The array lives in this translation unit alone.  With lazy module loading (the
// CUDA default since 12.2, CUDA_MODULE_LOADING=LAZY) its module, and the
// IGA_NOALLOC_SCRATCH_BYTES it occupies, is loaded on a device only when this
// entry point first runs there; with CUDA_MODULE_LOADING=EAGER every context that
// loads libiga reserves the array on its device whether or not it calls here.
#include <vector>

#include "iga_internal.cuh"

namespace iga {
size_t mass_solve_work_bytes_nrhs(const iga_ops* ops, int dtype, int nrhs);
}

using namespace iga;

static __device__ __align__(256) unsigned char g_noalloc_scratch[IGA_NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side handle, so the address is looked up with the
// device current.  The lookup runs on every call (cheap once the module is
// loaded; the first call on a device may load it): a cached address would go
// stale after a device reset reloads the module.
int scratch_address(void** out) {
    void* p = nullptr;
    IGA_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) return fail(IGA_ERR_CUDA, "cudaGetSymbolAddress returned a null scratch address");
    *out = p;
    return IGA_OK;
}
}  // namespace

extern "C" int iga_mass_solve_noalloc(const iga_ops* ops, int dtype, const void* b, void* x, int nrhs, double rtol,
                                      int max_it, unsigned flags, int* iters_out, double* relres_out, void* stream) {
    if (!ops || !b || !x) return fail(IGA_ERR_ARG, "null argument");
    if (dtype != IGA_F32 && dtype != IGA_F64) return fail(IGA_ERR_ARG, "dtype must be IGA_F32 or IGA_F64");
    if (nrhs < 0 || max_it < 0 || !(rtol >= 0.0)) return fail(IGA_ERR_ARG, "bad nrhs / max_it / rtol");
    if (nrhs == 0) return IGA_OK;
    if (b == x) return fail(IGA_ERR_ARG, "x must not alias b");
    // the graph schedule builds and instantiates a CUDA graph per call, which may
    // reserve device resources: not offered here
    if (flags & IGA_SOLVE_GRAPH) return fail(IGA_ERR_ARG, "mass_solve_noalloc does not take IGA_SOLVE_GRAPH");
    // the fixed array is sized for the plain solves, not for a refinement chunk
    if (flags & IGA_SOLVE_REFINE) return fail(IGA_ERR_ARG, "mass_solve_noalloc does not take IGA_SOLVE_REFINE");
    const size_t need = mass_solve_work_bytes_nrhs(ops, dtype, nrhs);
    if (need > (size_t)IGA_NOALLOC_SCRATCH_BYTES)
        return fail(IGA_ERR_ARG, "mass_solve_noalloc: CG workspace of " + std::to_string(need) +
                                     " bytes exceeds the fixed scratch of " +
                                     std::to_string((size_t)IGA_NOALLOC_SCRATCH_BYTES) +
                                     " bytes (use iga_mass_solve for this size)");
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    // Whatever must start at zero (CG direction buffers, the grid-barrier
    // counter and error word) is cleared on the stream by the solver itself at
    // the start of every right-hand-side chunk; the rest of the workspace is
    // written before it is read.
    // statistics are always read back (host vectors, not device memory), so that
    // errors are returned also when the caller passes no statistics arrays
    std::vector<int> it_local(iters_out ? 0 : nrhs);
    std::vector<double> rr_local(relres_out ? 0 : nrhs);
    return mass_solve_impl(ops, dtype, b, x, ops->N, nrhs, rtol, max_it, flags,
                           iters_out ? iters_out : it_local.data(), relres_out ? relres_out : rr_local.data(),
                           (cudaStream_t)stream, scratch, (size_t)IGA_NOALLOC_SCRATCH_BYTES, nullptr, nullptr);
}
