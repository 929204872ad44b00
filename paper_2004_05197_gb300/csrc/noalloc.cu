// iga_mass_solve_noalloc: the Jacobi-PCG mass solve of iga_mass_solve with its
// CG workspace in a fixed device array compiled into the library, so that a
// call allocates no device memory.  The solver itself (kernels, schedule,
// convergence test, results) is the one iga_mass_solve runs; only where the
// workspace comes from differs.
//
// The array lives in this translation unit alone, so its module (and the
// IGA_NOALLOC_SCRATCH_BYTES it occupies) is loaded only by programs that call
// this entry point.
#include <mutex>

#include "iga_internal.cuh"

namespace iga {
size_t mass_solve_work_bytes_nrhs(const iga_ops* ops, int dtype, int nrhs);
}

using namespace iga;

static __device__ __align__(256) unsigned char g_noalloc_scratch[IGA_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the lookup may load this module; later calls only read the cache).
int scratch_address(void** out) {
    int dev = 0;
    IGA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(IGA_ERR_ARG, "device ordinal beyond the scratch table");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        IGA_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        if (!p) return fail(IGA_ERR_CUDA, "cudaGetSymbolAddress returned a null scratch address");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
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
    return mass_solve_impl(ops, dtype, b, x, ops->N, nrhs, rtol, max_it, flags, iters_out, relres_out,
                           (cudaStream_t)stream, scratch, (size_t)IGA_NOALLOC_SCRATCH_BYTES, nullptr, nullptr);
}
