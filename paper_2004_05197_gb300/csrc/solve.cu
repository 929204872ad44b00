// Jacobi-PCG on the surrogate mass M~ (mass_solve) and leapfrog time stepping
// (wave_*).
//
// PCG recurrence (standard preconditioned CG, diagonal preconditioner D^-1):
//   r = b - M~x, z = D^-1 r, p = z, rz = (r, z)
//   repeat while ||r|| > rtol ||b|| and it < max_it:
//     q = M~p, alpha = rz / (p, q), x += alpha p, r -= alpha q, z = D^-1 r,
//     beta = (r, z)_new / rz, p = z + beta p
// The update p = z + beta p is folded into the next mass apply: the apply reads
// z and the previous p at the neighbours and forms z + beta p on the fly, while
// the row's own new p is written to the other half of a double buffer.  One
// iteration is thus two grid-wide phases:
//   A: p_new = z + beta p_old, q = M~ p_new, partial (p_new, q)
//   B: x += alpha p_new, r -= alpha q, z = D^-1 r, partial (r, z), (r, r)
// FP32 dtype: fields, x, z, p, q in FP32; the residual r and every dot product
// in FP64.  Dot products are reduced deterministically: per-block partials,
// then a fixed-order warp reduction that every block performs identically.
//
// Default schedule: one cooperative (persistent) launch runs all iterations,
// phases separated by a bounded grid barrier; convergence is decided on the
// device.  IGA_SOLVE_PLAIN: the same phases as separate launches with the
// scalars read back to the host every phase (the plain reference schedule).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "geom.cuh"
#include "host_bspline.h"
#include "iga_internal.cuh"
#include "stencil.cuh"

namespace iga {

// Optional self-checking build (-DIGA_BOUNDS_CHECK): every global access of the
// CG path is checked against the extent of its buffer; the first violation is
// recorded (site, index, extent) and the access is skipped instead of faulting.
__device__ long long g_bounds_record[4];
#ifdef IGA_BOUNDS_CHECK
__device__ __noinline__ void bounds_record(long long idx, long long ext, int site) {
    if (atomicCAS((unsigned long long*)&g_bounds_record[0], 0ull, (unsigned long long)site) == 0ull) {
        g_bounds_record[1] = idx;
        g_bounds_record[2] = ext;
    }
}
#define IGA_IN(idx, ext, site) \
    (((long long)(idx) >= 0 && (long long)(idx) < (long long)(ext)) ? true : (bounds_record((idx), (ext), (site)), false))
#else
#define IGA_IN(idx, ext, site) true
#endif

constexpr int kCgThreads = 256;
constexpr int kCgMaxBlocksPerSM = 8;
constexpr bool kCgFourRow = false;   // four-rows-per-thread phase A (measured slower; kept selectable)
template <int R>
constexpr int kCgUnroll = R >= 4 ? 2 : 4;   // fields in flight per thread in the mass apply
constexpr int kCgWarps = kCgThreads / 32;
constexpr long long kBarrierSpinCycles = 4000000000LL;   // ~2 s at 2 GHz

// ---------------------------------------------------------------- loaders
// Vectors written inside the persistent kernel are read with ordinary
// (coherent) loads, never through the read-only path: the grid barrier's
// fences make writes of other blocks visible to ordinary loads only.
template <typename T>
struct PlainLoad {
    const T* x;
    long long xs;
    long long ext;
    __device__ __forceinline__ T operator()(int r, int idx) const {
        const long long o = r * xs + idx;
        return IGA_IN(o, ext, 1) ? x[o] : T(0);
    }
};
template <typename T, int R>
struct CombLoad {   // z + beta p_old, formed on the fly
    const T* z;
    const T* p;
    long long xs;
    long long ext;
    T beta[R];
    __device__ __forceinline__ T operator()(int r, int idx) const {
        const long long o = r * xs + idx;
        return IGA_IN(o, ext, 2) ? fma(beta[r], p[o], z[o]) : T(0);
    }
};

// ---------------------------------------------------------------- reductions
// Block sum of K doubles per thread (v[K]) into red[K] (shared), fixed order.
template <int K>
__device__ __forceinline__ void block_sum(double* v, double* wsum /*[kCgWarps][K]*/, double* red /*[K]*/) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = v[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) wsum[w * K + k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double s = 0.0;
        for (int ww = 0; ww < kCgWarps; ++ww) s += wsum[ww * K + k];
        red[k] = s;
    }
    __syncthreads();
}

// Sum over blocks of partials[b * stride + off + k] (k < K) into out[k]
// (shared), fixed order; every block computes the identical result.
template <int K>
__device__ __forceinline__ void grid_sum(const double* partials, int nblocks, int stride, int off, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < K; k += kCgWarps) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32)
            s += IGA_IN((long long)b * stride + off + k, (long long)nblocks * stride, 14)
                     ? __ldcg(partials + (size_t)b * stride + off + k)
                     : 0.0;
#pragma unroll
        for (int off2 = 16; off2 > 0; off2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, off2);
        if (lane == 0) out[k] = s;
    }
    __syncthreads();
}

// Bounded grid barrier (cooperative launch guarantees co-residency).  On time-out
// it sets bit 4 of *err and returns false; every caller then leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == gen) {
                __nanosleep(32);
                if (clock64() - t0 > kBarrierSpinCycles) {
                    atomicOr(err, 4);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int*)err) == 0;
}

// ---------------------------------------------------------------- CG phases
// Internal vectors (r, z, p0, p1, q) are [R][ldw] with ldw a multiple of 4;
// the caller's b and x are [R][ldu].
template <typename T>
struct CgVecs {
    const T* F;          // M~ fields (field 0 = diagonal)
    long long pitch;
    const T* dinv;
    const T* b;
    T* x;
    double* r;
    T* z;
    T* p0;
    T* p1;
    T* q;
    int N, m;
    long long ldw, ldu;
    long long ext_vec;   // R * ldw: extent of every internal vector
    long long ext_user;  // R * ldu: extent of b and x
    long long ext_diag;  // extent of dinv
};

// z + beta p_old for four consecutive rows (coherent 16-byte loads)
__device__ __forceinline__ float4 ld4c(const float* p) { return *reinterpret_cast<const float4*>(p); }
template <int R>
struct CombLoad4 {
    const float* z;
    const float* p;
    long long ld;
    float beta[R];
    __device__ __forceinline__ float4 load4(int r, int idx) const {
        const float b = beta[r];
        return f4_fma(make_float4(b, b, b, b), ld4c(p + r * ld + idx), ld4c(z + r * ld + idx));
    }
    __device__ __forceinline__ float4 load4u(int r, int j) const {
        const int off = j & 3;
        const long long a = r * ld + (j - off);
        const float b = beta[r];
        const float4 bb = make_float4(b, b, b, b);
        const float4 v0 = f4_fma(bb, ld4c(p + a), ld4c(z + a));
        if (off == 0) return v0;
        const float4 v1 = f4_fma(bb, ld4c(p + a + 4), ld4c(z + a + 4));
        return f4_window(v0, v1, off);
    }
};

// init: r = b - M~x, z = D^-1 r; partials (r,z), (r,r), (b,b)
template <int DIM, int P, typename T, int R>
__device__ __forceinline__ void cg_init_rows(const CgVecs<T>& v, double* part) {
    for (int k = 0; k < 3 * R; ++k) part[k] = 0.0;
    PlainLoad<T> ld{v.x, v.ldu, v.ext_user};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x) {
        T acc[R], own[R];
        stencil_row<DIM, P, T, true, R, kCgUnroll<R>>(v.F, v.pitch, ld, i, v.N, v.m, acc, own);
        const double di = IGA_IN(i, v.ext_diag, 6) ? (double)v.dinv[i] : 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long ou = (long long)r * v.ldu + i, ow = (long long)r * v.ldw + i;
            const bool ok = IGA_IN(ou, v.ext_user, 7) && IGA_IN(ow, v.ext_vec, 16);
            const double bi = ok ? (double)v.b[ou] : 0.0;
            const double ri = bi - (double)acc[r];
            const T zi = (T)(di * ri);
            if (ok) {
                v.r[ow] = ri;
                v.z[ow] = zi;
            }
            part[3 * r + 0] += ri * (double)zi;
            part[3 * r + 1] += ri * ri;
            part[3 * r + 2] += bi * bi;
        }
    }
}

// phase A: p_new = z + beta p_old, q = M~ p_new; partial (p_new, q)
template <int DIM, int P, typename T, int R>
__device__ __forceinline__ void cg_phase_a(const CgVecs<T>& v, const T* pold, T* pnew, const double* beta,
                                           const int* active, double* part, const int* sdl) {
    for (int k = 0; k < R; ++k) part[k] = 0.0;
    CombLoad<T, R> ld;
    ld.z = v.z;
    ld.p = pold;
    ld.xs = v.ldw;
    ld.ext = v.ext_vec;
#pragma unroll
    for (int r = 0; r < R; ++r) ld.beta[r] = (T)beta[r];
    if constexpr (kCgFourRow && sizeof(T) == 4) {
        // four rows per thread; interior groups vectorised (see stencil_row4)
        CombLoad4<R> ld4;
        ld4.z = v.z;
        ld4.p = pold;
        ld4.ld = v.ldw;
#pragma unroll
        for (int r = 0; r < R; ++r) ld4.beta[r] = (float)beta[r];
        const int dmax = max_delta<DIM, P>(v.m);
        const int ngroups = (v.N + 3) / 4;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
            const int i0 = 4 * g;
            if (i0 >= dmax && i0 + 7 + dmax <= v.N - 1) {
                float4 acc[R], own[R];
                stencil_row4<DIM, P, true, R, kCgUnroll<R>>(v.F, v.pitch, ld4, i0, sdl, acc, own);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (!active[r]) continue;
                    const long long o = (long long)r * v.ldw + i0;
                    *reinterpret_cast<float4*>(pnew + o) = own[r];
                    *reinterpret_cast<float4*>(v.q + o) = acc[r];
                    part[r] += (double)own[r].x * acc[r].x + (double)own[r].y * acc[r].y +
                               (double)own[r].z * acc[r].z + (double)own[r].w * acc[r].w;
                }
            } else {
                for (int k = 0; k < 4 && i0 + k < v.N; ++k) {
                    T acc[R], own[R];
                    stencil_row<DIM, P, T, true, R, kCgUnroll<R>>(v.F, v.pitch, ld, i0 + k, v.N, v.m, acc, own);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!active[r]) continue;
                        const long long o = (long long)r * v.ldw + i0 + k;
                        if (IGA_IN(o, v.ext_vec, 8)) {
                            pnew[o] = own[r];
                            v.q[o] = acc[r];
                        }
                        part[r] += (double)own[r] * (double)acc[r];
                    }
                }
            }
        }
    } else {
        const int dmax = max_delta<DIM, P>(v.m);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x) {
            T acc[R], own[R];
            if (i >= dmax && i < v.N - dmax)
                stencil_row_interior<DIM, P, T, true, R, kCgUnroll<R>>(v.F, v.pitch, ld, i, sdl, acc, own);
            else
                stencil_row<DIM, P, T, true, R, kCgUnroll<R>>(v.F, v.pitch, ld, i, v.N, v.m, acc, own);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                const long long o = (long long)r * v.ldw + i;
                if (IGA_IN(o, v.ext_vec, 8)) {
                    pnew[o] = own[r];
                    v.q[o] = acc[r];
                }
                part[r] += (double)own[r] * (double)acc[r];
            }
        }
    }
}

// phase B: x += alpha p, r -= alpha q, z = D^-1 r; partials (r,z), (r,r)
template <typename T, int R>
__device__ __forceinline__ void cg_phase_b(const CgVecs<T>& v, const T* pnew, const double* alpha,
                                           const int* active, double* part) {
    for (int k = 0; k < 2 * R; ++k) part[k] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x) {
        const double di = IGA_IN(i, v.ext_diag, 9) ? (double)v.dinv[i] : 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!active[r]) continue;
            const size_t o = (size_t)r * v.ldw + i;
            const size_t ou = (size_t)r * v.ldu + i;
            if (!IGA_IN(o, v.ext_vec, 10) || !IGA_IN(ou, v.ext_user, 17)) continue;
            const T pi = pnew[o];
            v.x[ou] = v.x[ou] + (T)alpha[r] * pi;
            const double ri = v.r[o] - alpha[r] * (double)v.q[o];
            const T zi = (T)(di * ri);
            v.r[o] = ri;
            v.z[o] = zi;
            part[2 * r + 0] += ri * (double)zi;
            part[2 * r + 1] += ri * ri;
        }
    }
}

struct CgCtl {
    double rtol;
    int max_it;
    int nblocks;
    double* partials;    // [nblocks][3R]
    unsigned* bar;       // [2]
    int* err;
    int* iters_out;      // [R]
    double* relres_out;  // [R]
    long long* iter_acc; // nullable: iterations are added here (device counter)
    int* status_acc;     // nullable: bit 8 set when an RHS misses rtol
};

// Partials of block b live at partials[b * 6R + ...]: phase A (p, q) at [0, R),
// phase B (r, z), (r, r) at [R, 3R), initial (r, z), (r, r), (b, b) at [3R, 6R).
// Separate regions make one barrier per phase sufficient: a block can only
// overwrite a region after every block has passed the next barrier, i.e. after
// every block has read that region.
template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(kCgThreads) pcg_persistent_kernel(CgVecs<T> v, CgCtl c) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R];
    __shared__ double rz[R], rr[R], bnorm[R], alpha[R], beta[R];
    __shared__ int active[R], iters[R];
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    double part[3 * R];
    const int S = 6 * R;
    fill_delta_table<DIM, P>(sdl, v.m);

    cg_init_rows<DIM, P, T, R>(v, part);
    block_sum<3 * R>(part, wsum, red);
    if (threadIdx.x < 3 * R && IGA_IN((long long)blockIdx.x * S + 3 * R + threadIdx.x, (long long)c.nblocks * S, 11))
        c.partials[(size_t)blockIdx.x * S + 3 * R + threadIdx.x] = red[threadIdx.x];
    if (!grid_barrier(c.bar, c.err)) return;
    grid_sum<3 * R>(c.partials, gridDim.x, S, 3 * R, red);
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        rz[r] = red[3 * r];
        rr[r] = red[3 * r + 1];
        bnorm[r] = sqrt(red[3 * r + 2]);
        beta[r] = 0.0;
        alpha[r] = 0.0;
        iters[r] = 0;
        active[r] = bnorm[r] > 0.0 && !(c.rtol > 0.0 && sqrt(rr[r]) <= c.rtol * bnorm[r]);
    }
    __syncthreads();
    // a zero right-hand side has the solution 0
    for (int r = 0; r < R; ++r)
        if (!(bnorm[r] > 0.0))
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x)
                if (IGA_IN((long long)r * v.ldu + i, v.ext_user, 15)) v.x[(size_t)r * v.ldu + i] = T(0);
    // p_old starts at 0 (cleared by the host) so that p = z on the first iteration
    for (int it = 0; it < c.max_it; ++it) {
        bool any = false;
        for (int r = 0; r < R; ++r) any = any || active[r];
        if (!any) break;
        T* pold = (it & 1) ? v.p1 : v.p0;
        T* pnew = (it & 1) ? v.p0 : v.p1;
        cg_phase_a<DIM, P, T, R>(v, pold, pnew, beta, active, part, sdl);
        block_sum<R>(part, wsum, red);
        if (threadIdx.x < R && IGA_IN((long long)blockIdx.x * S + threadIdx.x, (long long)c.nblocks * S, 12))
            c.partials[(size_t)blockIdx.x * S + threadIdx.x] = red[threadIdx.x];
        if (!grid_barrier(c.bar, c.err)) return;
        grid_sum<R>(c.partials, gridDim.x, S, 0, red);
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            if (active[r]) {
                const double pq = red[r];
                if (!(pq > 0.0) || !isfinite(pq)) {
                    active[r] = 0;
                    if (blockIdx.x == 0) atomicOr(c.err, 1);
                }
                alpha[r] = active[r] ? rz[r] / pq : 0.0;
            }
        }
        __syncthreads();
        cg_phase_b<T, R>(v, pnew, alpha, active, part);
        block_sum<2 * R>(part, wsum, red);
        if (threadIdx.x < 2 * R && IGA_IN((long long)blockIdx.x * S + R + threadIdx.x, (long long)c.nblocks * S, 13))
            c.partials[(size_t)blockIdx.x * S + R + threadIdx.x] = red[threadIdx.x];
        if (!grid_barrier(c.bar, c.err)) return;
        grid_sum<2 * R>(c.partials, gridDim.x, S, R, red);
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            if (active[r]) {
                const double rz_new = red[2 * r];
                rr[r] = red[2 * r + 1];
                beta[r] = rz_new / rz[r];
                rz[r] = rz_new;
                iters[r] += 1;
                if (c.rtol > 0.0 && sqrt(rr[r]) <= c.rtol * bnorm[r]) active[r] = 0;
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x < R) {
        const int r = threadIdx.x;
        const double rel = bnorm[r] > 0.0 ? sqrt(rr[r]) / bnorm[r] : 0.0;
        c.iters_out[r] = iters[r];
        c.relres_out[r] = rel;
        if (c.iter_acc) atomicAdd((unsigned long long*)c.iter_acc, (unsigned long long)iters[r]);
        if (c.status_acc && c.rtol > 0.0 && rel > c.rtol) atomicOr(c.status_acc, 8);
    }
}

// ---------------------------------------------------------------- plain schedule kernels
template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(kCgThreads) cg_init_kernel(CgVecs<T> v, double* partials) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R];
    double part[3 * R];
    cg_init_rows<DIM, P, T, R>(v, part);
    block_sum<3 * R>(part, wsum, red);
    if (threadIdx.x < 3 * R) partials[(size_t)blockIdx.x * 6 * R + 3 * R + threadIdx.x] = red[threadIdx.x];
}

template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(kCgThreads) cg_a_kernel(CgVecs<T> v, const T* pold, T* pnew, const double* sc,
                                                          double* partials) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R];
    __shared__ double beta[R];
    __shared__ int active[R];
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    if (threadIdx.x < R) {
        beta[threadIdx.x] = sc[threadIdx.x];
        active[threadIdx.x] = (int)sc[2 * R + threadIdx.x];
    }
    fill_delta_table<DIM, P>(sdl, v.m);
    double part[3 * R];
    cg_phase_a<DIM, P, T, R>(v, pold, pnew, beta, active, part, sdl);
    block_sum<R>(part, wsum, red);
    if (threadIdx.x < R) partials[(size_t)blockIdx.x * 6 * R + threadIdx.x] = red[threadIdx.x];
}

template <typename T, int R>
__global__ void __launch_bounds__(kCgThreads) cg_b_kernel(CgVecs<T> v, const T* pnew, const double* sc,
                                                          double* partials) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R];
    __shared__ double alpha[R];
    __shared__ int active[R];
    if (threadIdx.x < R) {
        alpha[threadIdx.x] = sc[R + threadIdx.x];
        active[threadIdx.x] = (int)sc[2 * R + threadIdx.x];
    }
    __syncthreads();
    double part[3 * R];
    cg_phase_b<T, R>(v, pnew, alpha, active, part);
    block_sum<2 * R>(part, wsum, red);
    if (threadIdx.x < 2 * R) partials[(size_t)blockIdx.x * 6 * R + R + threadIdx.x] = red[threadIdx.x];
}

template <int K>
__global__ void grid_sum_kernel(const double* partials, int nblocks, int stride, int off, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < K; k += kCgWarps) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) s += partials[(size_t)b * stride + off + k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) out[k] = s;
    }
}

// ---------------------------------------------------------------- host driver
struct CgWork {
    double* r;
    void* z;
    void* p0;
    void* p1;
    void* q;
    double* partials;
    unsigned* bar;
    int* err;
    int* iters;
    double* relres;
    double* sc;   // plain schedule scalars [3R]
    double* red;  // plain schedule reduced values [3R]
};

template <typename T>
static CgWork carve(void* base, long long N /* leading dimension of the internal vectors */, int R, int nblocks) {
    char* p = (char*)base;
    auto take = [&](size_t bytes) {
        void* out = p;
        p += (bytes + 255) / 256 * 256;
        return out;
    };
    CgWork w;
    w.r = (double*)take(sizeof(double) * (size_t)R * N);
    w.z = take(sizeof(T) * (size_t)R * N);
    w.p0 = take(sizeof(T) * (size_t)R * N);
    w.p1 = take(sizeof(T) * (size_t)R * N);
    w.q = take(sizeof(T) * (size_t)R * N);
    w.partials = (double*)take(sizeof(double) * (size_t)nblocks * 6 * R);
    w.bar = (unsigned*)take(64);
    w.err = (int*)take(64);
    w.iters = (int*)take(sizeof(int) * R);
    w.relres = (double*)take(sizeof(double) * R);
    w.sc = (double*)take(sizeof(double) * 3 * R);
    w.red = (double*)take(sizeof(double) * 3 * R);
    return w;
}

static size_t carve_bytes(size_t es, long long N, int R, int nblocks) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return up(sizeof(double) * (size_t)R * N) + 4 * up(es * (size_t)R * N) + up(sizeof(double) * (size_t)nblocks * 6 * R) +
           2 * up(64) + up(sizeof(int) * R) + 3 * up(sizeof(double) * 3 * R) + 256;
}

template <int DIM, int P, typename T, int R>
static int cg_blocks() {
    static int nb = 0;
    if (!nb) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_persistent_kernel<DIM, P, T, R>, kCgThreads, 0);
        nb = std::max(1, sms * std::max(1, std::min(per, kCgMaxBlocksPerSM)));
    }
    return nb;
}

template <int DIM, int P, typename T, int R>
static int pcg_chunk(const iga_ops* ops, const T* b, T* x, long long ldu, double rtol, int max_it, unsigned flags,
                     int* iters_h, double* relres_h, cudaStream_t st, void* work, size_t work_bytes, bool* not_conv,
                     long long* iter_acc, int* status_acc) {
    const long long N = ops->N;
    const long long ldw = (N + 3) / 4 * 4;
    const int nblocks = cg_blocks<DIM, P, T, R>();
    if (carve_bytes(sizeof(T), ldw, R, nblocks) > work_bytes) return fail(IGA_ERR_ARG, "CG workspace too small");
    CgWork w = carve<T>(work, ldw, R, nblocks);
    CgVecs<T> v;
    v.F = (sizeof(T) == 8) ? (const T*)ops->fM64.ptr : (const T*)ops->fM32.ptr;
    v.pitch = ops->pitch;
    v.dinv = (sizeof(T) == 8) ? (const T*)ops->dinv64.ptr : (const T*)ops->dinv32.ptr;
    v.b = b;
    v.x = x;
    v.r = w.r;
    v.z = (T*)w.z;
    v.p0 = (T*)w.p0;
    v.p1 = (T*)w.p1;
    v.q = (T*)w.q;
    v.N = (int)N;
    v.m = ops->m;
    v.ldw = ldw;
    v.ldu = ldu;
    v.ext_vec = (long long)R * ldw;
    v.ext_user = (long long)(R - 1) * ldu + N;
    v.ext_diag = ops->pitch;
    IGA_CUDA(cudaMemsetAsync(w.p0, 0, sizeof(T) * R * ldw, st));
    IGA_CUDA(cudaMemsetAsync(w.bar, 0, 64, st));
    IGA_CUDA(cudaMemsetAsync(w.err, 0, 64, st));
    int iters[R];
    double relres[R];
    if (!(flags & IGA_SOLVE_PLAIN)) {
        CgCtl c;
        c.rtol = rtol;
        c.max_it = max_it;
        c.nblocks = nblocks;
        c.partials = w.partials;
        c.bar = w.bar;
        c.err = w.err;
        c.iters_out = w.iters;
        c.relres_out = w.relres;
        c.iter_acc = iter_acc;
        c.status_acc = status_acc;
        void* args[] = {&v, &c};
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_persistent_kernel<DIM, P, T, R>, nblocks,
                                                    kCgThreads, args, 0, st);
        count_launch();
        if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(pcg)");
#ifdef IGA_BOUNDS_CHECK
        {
            long long rec[4] = {0, 0, 0, 0};
            IGA_CUDA(cudaStreamSynchronize(st));
            IGA_CUDA(cudaMemcpyFromSymbol(rec, g_bounds_record, sizeof(rec)));
            if (rec[0] != 0) {
                char msg[160];
                snprintf(msg, sizeof(msg), "bounds check: site %lld index %lld extent %lld", rec[0], rec[1], rec[2]);
                return fail(IGA_ERR_ARG, msg);
            }
        }
#endif
        if (iters_h || relres_h || not_conv) {
            int err = 0;
            IGA_CUDA(cudaMemcpyAsync(iters, w.iters, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
            IGA_CUDA(cudaMemcpyAsync(relres, w.relres, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
            IGA_CUDA(cudaMemcpyAsync(&err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
            IGA_CUDA(cudaStreamSynchronize(st));
            if (err & 4) return fail(IGA_ERR_TIMEOUT, "grid barrier timed out in pcg");
            if (err & 1) return fail(IGA_ERR_NONFINITE, "CG breakdown: (p, M p) <= 0 or non-finite");
        }
    } else {
        // plain schedule: host-side scalars, two read-backs per iteration
        const int grid = nblocks;
        cg_init_kernel<DIM, P, T, R><<<grid, kCgThreads, 0, st>>>(v, w.partials);
        IGA_LAUNCH_CHECK("cg_init_kernel");
        grid_sum_kernel<3 * R><<<1, kCgThreads, 0, st>>>(w.partials, grid, 6 * R, 3 * R, w.red);
        IGA_LAUNCH_CHECK("grid_sum_kernel");
        double red[3 * R], sc[3 * R];
        IGA_CUDA(cudaMemcpyAsync(red, w.red, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, st));
        IGA_CUDA(cudaStreamSynchronize(st));
        double rz[R], rr[R], bn[R];
        int active[R];
        for (int r = 0; r < R; ++r) {
            rz[r] = red[3 * r];
            rr[r] = red[3 * r + 1];
            bn[r] = std::sqrt(red[3 * r + 2]);
            iters[r] = 0;
            active[r] = bn[r] > 0.0 && !(rtol > 0.0 && std::sqrt(rr[r]) <= rtol * bn[r]);
            sc[r] = 0.0;                // beta
            sc[R + r] = 0.0;            // alpha
            if (!(bn[r] > 0.0)) IGA_CUDA(cudaMemsetAsync(x + (size_t)r * ldu, 0, sizeof(T) * N, st));
        }
        for (int it = 0; it < max_it; ++it) {
            bool any = false;
            for (int r = 0; r < R; ++r) any = any || active[r];
            if (!any) break;
            for (int r = 0; r < R; ++r) sc[2 * R + r] = active[r];
            T* pold = (T*)((it & 1) ? w.p1 : w.p0);
            T* pnew = (T*)((it & 1) ? w.p0 : w.p1);
            IGA_CUDA(cudaMemcpyAsync(w.sc, sc, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, st));
            cg_a_kernel<DIM, P, T, R><<<grid, kCgThreads, 0, st>>>(v, pold, pnew, w.sc, w.partials);
            IGA_LAUNCH_CHECK("cg_a_kernel");
            grid_sum_kernel<R><<<1, kCgThreads, 0, st>>>(w.partials, grid, 6 * R, 0, w.red);
            IGA_LAUNCH_CHECK("grid_sum_kernel");
            IGA_CUDA(cudaMemcpyAsync(red, w.red, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
            IGA_CUDA(cudaStreamSynchronize(st));
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                if (!(red[r] > 0.0) || !std::isfinite(red[r]))
                    return fail(IGA_ERR_NONFINITE, "CG breakdown: (p, M p) <= 0 or non-finite");
                sc[R + r] = rz[r] / red[r];
            }
            IGA_CUDA(cudaMemcpyAsync(w.sc, sc, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, st));
            cg_b_kernel<T, R><<<grid, kCgThreads, 0, st>>>(v, pnew, w.sc, w.partials);
            IGA_LAUNCH_CHECK("cg_b_kernel");
            grid_sum_kernel<2 * R><<<1, kCgThreads, 0, st>>>(w.partials, grid, 6 * R, R, w.red);
            IGA_LAUNCH_CHECK("grid_sum_kernel");
            IGA_CUDA(cudaMemcpyAsync(red, w.red, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, st));
            IGA_CUDA(cudaStreamSynchronize(st));
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                const double rz_new = red[2 * r];
                rr[r] = red[2 * r + 1];
                sc[r] = rz_new / rz[r];
                rz[r] = rz_new;
                iters[r] += 1;
                if (rtol > 0.0 && std::sqrt(rr[r]) <= rtol * bn[r]) active[r] = 0;
            }
        }
        long long tot = 0;
        int nc_flag = 0;
        for (int r = 0; r < R; ++r) {
            relres[r] = bn[r] > 0.0 ? std::sqrt(rr[r]) / bn[r] : 0.0;
            tot += iters[r];
            if (rtol > 0.0 && relres[r] > rtol) nc_flag = 8;
        }
        if (iter_acc || status_acc) {
            // fold the host-side counts into the device accumulators (plain schedule)
            long long acc_h = 0;
            int st_h = 0;
            if (iter_acc) IGA_CUDA(cudaMemcpy(&acc_h, iter_acc, sizeof(acc_h), cudaMemcpyDeviceToHost));
            if (status_acc) IGA_CUDA(cudaMemcpy(&st_h, status_acc, sizeof(st_h), cudaMemcpyDeviceToHost));
            acc_h += tot;
            st_h |= nc_flag;
            if (iter_acc) IGA_CUDA(cudaMemcpy(iter_acc, &acc_h, sizeof(acc_h), cudaMemcpyHostToDevice));
            if (status_acc) IGA_CUDA(cudaMemcpy(status_acc, &st_h, sizeof(st_h), cudaMemcpyHostToDevice));
        }
    }
    if (iters_h || relres_h || not_conv) {
        for (int r = 0; r < R; ++r) {
            if (iters_h) iters_h[r] = iters[r];
            if (relres_h) relres_h[r] = relres[r];
            if (not_conv && rtol > 0.0 && relres[r] > rtol) *not_conv = true;
        }
    }
    return IGA_OK;
}

template <int DIM, int P, typename T>
static int pcg_typed(const iga_ops* ops, const T* b, T* x, long long ldu, int nrhs, double rtol, int max_it,
                     unsigned flags, int* iters_h, double* relres_h, cudaStream_t st, void* work, size_t work_bytes,
                     bool* nc, long long* iter_acc, int* status_acc) {
    const long long N = ldu;
    int r0 = 0;
    while (r0 < nrhs) {
        const int left = nrhs - r0;
        int rc;
        if (left >= 4) {
            rc = pcg_chunk<DIM, P, T, 4>(ops, b + (size_t)r0 * N, x + (size_t)r0 * N, ldu, rtol, max_it, flags,
                                         iters_h ? iters_h + r0 : nullptr, relres_h ? relres_h + r0 : nullptr, st,
                                         work, work_bytes, nc, iter_acc, status_acc);
            r0 += 4;
        } else {
            rc = pcg_chunk<DIM, P, T, 1>(ops, b + (size_t)r0 * N, x + (size_t)r0 * N, ldu, rtol, max_it, flags,
                                         iters_h ? iters_h + r0 : nullptr, relres_h ? relres_h + r0 : nullptr, st,
                                         work, work_bytes, nc, iter_acc, status_acc);
            r0 += 1;
        }
        if (rc) return rc;
    }
    return IGA_OK;
}

size_t mass_solve_work_bytes(const iga_ops* ops, int dtype, int nrhs) {
    (void)nrhs;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = std::max(1, sms) * kCgMaxBlocksPerSM;
    return carve_bytes(dtype == IGA_F64 ? 8 : 4, (ops->N + 3) / 4 * 4, 4, nb);
}

int mass_solve_impl(const iga_ops* ops, int dtype, const void* b, void* x, long long ld, int nrhs, double rtol,
                    int max_it, unsigned flags, int* iters_out, double* relres_out, cudaStream_t st, void* work,
                    size_t work_bytes, long long* iter_acc, int* status_acc) {
    bool nc = false;
    const bool want = iters_out || relres_out;
    std::vector<int> it_h(nrhs);
    std::vector<double> rr_h(nrhs);
    const int d = ops->dim, p = ops->p;
    int rc;
#define IGA_PCG_CASE(DD, PP)                                                                                   \
    if (d == DD && p == PP)                                                                                    \
        rc = dtype == IGA_F64                                                                                  \
                 ? pcg_typed<DD, PP, double>(ops, (const double*)b, (double*)x, ld, nrhs, rtol, max_it, flags,\
                                             want ? it_h.data() : nullptr, want ? rr_h.data() : nullptr, st,  \
                                             work, work_bytes, want ? &nc : nullptr, iter_acc, status_acc)    \
                 : pcg_typed<DD, PP, float>(ops, (const float*)b, (float*)x, ld, nrhs, rtol, max_it, flags,   \
                                            want ? it_h.data() : nullptr, want ? rr_h.data() : nullptr, st,   \
                                            work, work_bytes, want ? &nc : nullptr, iter_acc, status_acc);    \
    else
    IGA_PCG_CASE(2, 1) IGA_PCG_CASE(2, 2) IGA_PCG_CASE(2, 3) IGA_PCG_CASE(3, 1) IGA_PCG_CASE(3, 2)
    return fail(IGA_ERR_ARG, "unsupported (dim, p) for mass_solve");
#undef IGA_PCG_CASE
    if (rc) return rc;
    if (want) {
        for (int r = 0; r < nrhs; ++r) {
            if (iters_out) iters_out[r] = it_h[r];
            if (relres_out) relres_out[r] = rr_h[r];
        }
    }
    if (nc) return fail(IGA_ERR_NOT_CONVERGED, "CG reached max_it before rtol");
    return IGA_OK;
}

}  // namespace iga

using namespace iga;

extern "C" int iga_mass_solve(const iga_ops* ops, int dtype, const void* b, void* x, int nrhs, double rtol,
                              int max_it, unsigned flags, int* iters_out, double* relres_out, void* stream) {
    if (!ops || !b || !x) return fail(IGA_ERR_ARG, "null argument");
    if (dtype != IGA_F32 && dtype != IGA_F64) return fail(IGA_ERR_ARG, "dtype must be IGA_F32 or IGA_F64");
    if (nrhs < 0 || max_it < 0 || !(rtol >= 0.0)) return fail(IGA_ERR_ARG, "bad nrhs / max_it / rtol");
    if (nrhs == 0) return IGA_OK;
    if (b == x) return fail(IGA_ERR_ARG, "x must not alias b");
    iga_ops* mops = const_cast<iga_ops*>(ops);
    const size_t need = mass_solve_work_bytes(ops, dtype, nrhs);
    if (mops->work.bytes < need) {
        int rc = mops->work.alloc(need);
        if (rc) return rc;
    }
    return mass_solve_impl(ops, dtype, b, x, ops->N, nrhs, rtol, max_it, flags, iters_out, relres_out,
                           (cudaStream_t)stream, mops->work.ptr, mops->work.bytes, nullptr, nullptr);
}
