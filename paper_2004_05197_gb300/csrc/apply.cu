// stencil_apply: y = K~ x or y = M~ x, matrix-free, for nrhs vectors.
// One thread per output row (grid-stride), rows of a warp contiguous so every
// field read is a coalesced 128-byte (FP32) line; all right-hand sides of a
// chunk reuse the field values held in registers.
#include <algorithm>
#include <cstdint>

#include "iga_internal.cuh"
#include "stencil.cuh"

namespace iga {

template <int DIM, int P, typename T, bool MASS, int R>
__global__ void __launch_bounds__(256) apply_kernel(const T* __restrict__ F, long long pitch,
                                                     const T* __restrict__ x, T* __restrict__ y, int N,
                                                     int m) {
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    fill_delta_table<DIM, P>(sdl, m);
    const int dmax = max_delta<DIM, P>(m);
    const LdgLoad<T> ld{x, N};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        T acc[R], own[R];
        if (i >= dmax && i < N - dmax)
            stencil_row_interior<DIM, P, T, MASS, R, (R >= 4 ? 2 : 16), LdgLoad<T>, true>(F, pitch, ld, i, sdl, acc,
                                                                                     own);
        else
            stencil_row<DIM, P, T, MASS, R, (R >= 4 ? 2 : 4), LdgLoad<T>, true>(F, pitch, ld, i, N, m, acc, own);
#pragma unroll
        for (int r = 0; r < R; ++r) y[(size_t)r * N + i] = acc[r];
    }
}

// The four-rows-per-thread FP32 variant measured slower than one row per thread
// with the interior fast path (fewer resident warps, serialised unaligned
// loads); it is kept selectable for comparison.
constexpr bool kUseFourRowPath = false;

// FP32, four rows per thread; interior groups vectorised, the rest per row.
template <int DIM, int P, bool MASS, int R>
__global__ void __launch_bounds__(256) apply4_kernel(const float* __restrict__ F, long long pitch,
                                                      const float* __restrict__ x, float* __restrict__ y,
                                                      long long ld, int N, int m) {
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    fill_delta_table<DIM, P>(sdl, m);
    const int dmax = max_delta<DIM, P>(m);
    const int ngroups = (N + 3) / 4;
    const LdgLoad4 ld4{x, ld};
    const LdgLoad<float> ld1{x, ld};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
        const int i0 = 4 * g;
        if (i0 >= dmax && i0 + 7 + dmax <= N - 1) {
            float4 acc[R], own[R];
            stencil_row4<DIM, P, MASS, R, 2>(F, pitch, ld4, i0, sdl, acc, own);
#pragma unroll
            for (int r = 0; r < R; ++r) *reinterpret_cast<float4*>(y + r * ld + i0) = acc[r];
        } else {
            for (int k = 0; k < 4 && i0 + k < N; ++k) {
                float acc[R], own[R];
                stencil_row<DIM, P, float, MASS, R, 4>(F, pitch, ld1, i0 + k, N, m, acc, own);
#pragma unroll
                for (int r = 0; r < R; ++r) y[r * ld + i0 + k] = acc[r];
            }
        }
    }
}

static int apply_grid(long long N) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    const long long want = (N + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * 16));
}

template <int DIM, int P>
static bool apply4_launch(const iga_ops* ops, int which, const float* F, const float* x, float* y, int R,
                          cudaStream_t st) {
    const int N = (int)ops->N;
    if (((uintptr_t)x | (uintptr_t)y) % 16 != 0 || (R > 1 && N % 4 != 0)) return false;
    const int grid = apply_grid((N + 3) / 4);
    if (R == 4) {
        if (which == IGA_OP_M) apply4_kernel<DIM, P, true, 4><<<grid, 256, 0, st>>>(F, ops->pitch, x, y, N, N, ops->m);
        else apply4_kernel<DIM, P, false, 4><<<grid, 256, 0, st>>>(F, ops->pitch, x, y, N, N, ops->m);
    } else {
        if (which == IGA_OP_M) apply4_kernel<DIM, P, true, 1><<<grid, 256, 0, st>>>(F, ops->pitch, x, y, N, N, ops->m);
        else apply4_kernel<DIM, P, false, 1><<<grid, 256, 0, st>>>(F, ops->pitch, x, y, N, N, ops->m);
    }
    return true;
}

template <int DIM, int P, typename T>
static int apply_typed(const iga_ops* ops, int which, const T* F, const T* x, T* y, int nrhs, cudaStream_t st) {
    const int N = (int)ops->N;
    const int grid = apply_grid(N);
    int r0 = 0;
    while (r0 < nrhs) {
        const int left = nrhs - r0;
        const T* xr = x + (size_t)r0 * N;
        T* yr = y + (size_t)r0 * N;
        if constexpr (sizeof(T) == 4) {
            const int R = left >= 4 ? 4 : 1;
            if (kUseFourRowPath && apply4_launch<DIM, P>(ops, which, (const float*)F, (const float*)xr, (float*)yr, R, st)) {
                IGA_LAUNCH_CHECK("apply4_kernel");
                r0 += R;
                continue;
            }
        }
        if (left >= 4) {
            if (which == IGA_OP_M)
                apply_kernel<DIM, P, T, true, 4><<<grid, 256, 0, st>>>(F, ops->pitch, xr, yr, N, ops->m);
            else
                apply_kernel<DIM, P, T, false, 4><<<grid, 256, 0, st>>>(F, ops->pitch, xr, yr, N, ops->m);
            r0 += 4;
        } else {
            if (which == IGA_OP_M)
                apply_kernel<DIM, P, T, true, 1><<<grid, 256, 0, st>>>(F, ops->pitch, xr, yr, N, ops->m);
            else
                apply_kernel<DIM, P, T, false, 1><<<grid, 256, 0, st>>>(F, ops->pitch, xr, yr, N, ops->m);
            r0 += 1;
        }
        IGA_LAUNCH_CHECK("apply_kernel");
    }
    return IGA_OK;
}

template <typename T>
static int apply_dispatch(const iga_ops* ops, int which, const T* F, const T* x, T* y, int nrhs,
                          cudaStream_t st) {
    const int d = ops->dim, p = ops->p;
    if (d == 2 && p == 1) return apply_typed<2, 1, T>(ops, which, F, x, y, nrhs, st);
    if (d == 2 && p == 2) return apply_typed<2, 2, T>(ops, which, F, x, y, nrhs, st);
    if (d == 2 && p == 3) return apply_typed<2, 3, T>(ops, which, F, x, y, nrhs, st);
    if (d == 3 && p == 1) return apply_typed<3, 1, T>(ops, which, F, x, y, nrhs, st);
    if (d == 3 && p == 2) return apply_typed<3, 2, T>(ops, which, F, x, y, nrhs, st);
    return fail(IGA_ERR_ARG, "unsupported (dim, p) for stencil_apply");
}

int launch_apply(const iga_ops* ops, int which, int dtype, const void* x, void* y, int nrhs, cudaStream_t st) {
    if (ops->path == IGA_PATH_ONTHEFLY) return onthefly_apply(ops, which, dtype, x, y, nrhs, st);
    if (dtype == IGA_F64) {
        const double* F = which == IGA_OP_K ? ops->fK64.as<double>() : ops->fM64.as<double>();
        return apply_dispatch<double>(ops, which, F, (const double*)x, (double*)y, nrhs, st);
    }
    if (brick_usable(ops, which)) {
        // brick kernels: one launch per right-hand side
        const long long N = ops->N;
        for (int r = 0; r < nrhs; ++r) {
            const int rc = brick_apply(ops, which, (const float*)x + (size_t)r * N, (float*)y + (size_t)r * N, st);
            if (rc) return rc;
        }
        return IGA_OK;
    }
    const float* F = which == IGA_OP_K ? ops->fK32.as<float>() : ops->fM32.as<float>();
    return apply_dispatch<float>(ops, which, F, (const float*)x, (float*)y, nrhs, st);
}

}  // namespace iga

using namespace iga;

extern "C" int iga_stencil_apply(const iga_ops* ops, int which, int dtype, const void* x, void* y, int nrhs,
                                 void* stream) {
    if (!ops || !x || !y) return fail(IGA_ERR_ARG, "null argument");
    if (which != IGA_OP_K && which != IGA_OP_M) return fail(IGA_ERR_ARG, "which must be IGA_OP_K or IGA_OP_M");
    if (dtype != IGA_F32 && dtype != IGA_F64) return fail(IGA_ERR_ARG, "dtype must be IGA_F32 or IGA_F64");
    if (nrhs < 0) return fail(IGA_ERR_ARG, "nrhs must be >= 0");
    if (x == y) return fail(IGA_ERR_ARG, "y must not alias x");
    if (nrhs == 0) return IGA_OK;
    return launch_apply(ops, which, dtype, x, y, nrhs, (cudaStream_t)stream);
}
