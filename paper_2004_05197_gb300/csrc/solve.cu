// Jacobi-PCG on the surrogate mass M~ (mass_solve).
//
// Preconditioned CG with the diagonal (Jacobi) preconditioner D^-1 of M~, in
// the Chronopoulos-Gear arrangement (recurrence below, at the CG phases): one
// mass apply of a single gathered vector and one joint reduction per iteration,
// the same iterates as the textbook recurrence in exact arithmetic.  Each
// iteration is two grid-wide phases: a vector update (phase 1) and the mass
// apply with its dot product (phase 2).
// FP32 dtype: fields and the vectors u, w, p, s, x in FP32; the residual r in
// FP64 (one FP64 FMA per row and iteration).  Dot products: exact FP32 products
// summed per thread in a compensated FP32 pair (DotAcc, about 48 significant
// bits), then in FP64 across threads and blocks; u = D^-1 r is formed in FP32
// from r rounded to FP32.  Dot products are reduced deterministically:
// per-block partials, then a fixed-order warp reduction that every block
// performs identically.
//
// Default schedule: one cooperative (persistent) launch runs all iterations,
// phases separated by a bounded grid barrier; convergence is decided on the
// device.  IGA_SOLVE_PLAIN: the same phases as separate launches with the
// scalars read back to the host every iteration (the plain reference schedule).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "geom.cuh"
#include "host_bspline.h"
#include "iga_internal.cuh"
#include "stencil.cuh"
#include "cg.cuh"

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

constexpr int kCgThreads = 768;
constexpr int kCgMaxBlocksPerSM = 2;
template <int R>
constexpr int kCgUnroll = R >= 4 ? 2 : 4;   // fields in flight per thread in the mass apply
constexpr int kCgWarps = kCgThreads / 32;

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

// Sum over blocks of partials[b * stride + off + k] (k < K) into out[k]
// (shared), fixed order; every block computes the identical result.
template <int K>
__device__ __forceinline__ void grid_sum(const double* partials, int nblocks, int stride, int off, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < K; k += kCgWarps) {
        double s = IGA_IN((long long)(nblocks - 1) * stride + off + k, (long long)nblocks * stride, 14)
                       ? lane_partial_sum(partials, nblocks, stride, off + k, lane)
                       : 0.0;
#pragma unroll
        for (int off2 = 16; off2 > 0; off2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, off2);
        if (lane == 0) out[k] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- CG phases
// Chronopoulos-Gear form of Jacobi-PCG (one reduction per iteration; same
// iterates as the standard recurrence in exact arithmetic):
//   r = b - M~x, u = D^-1 r, w = M~u, gamma = (r,u), delta = (w,u), alpha = gamma/delta, beta = 0
//   repeat:  p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r,
//            w = M~u, gamma' = (r,u), delta = (w,u), stop if ||r|| <= rtol ||b||,
//            beta = gamma'/gamma, alpha = gamma' / (delta - beta gamma'/alpha)
// The mass apply gathers a single vector (u).  Internal vectors (r FP64; u, w,
// p, s in the dtype) are [R][ldw] with ldw a multiple of 4; the caller's b and
// x are [R][ldu].
template <typename T>
struct CgVecs {
    const T* F;          // M~ fields (field 0 = diagonal)
    long long pitch;
    const T* dinv;
    const T* b;
    T* x;
    double* r;
    T* u;
    T* w;
    T* p;
    T* s;
    int N, m;
    long long ldw, ldu;
    long long ext_vec;   // R * ldw: extent of every internal vector
    long long ext_user;  // extent of b and x
    long long ext_diag;  // extent of dinv
};

// Rows are distributed grid-stride: in each round all blocks cover one
// contiguous window, so the mirrored field reads F_u[i - Delta] hit L2 (a
// contiguous range per block was measured to raise DRAM reads by 27 %).
// mass apply y = M~ vec for R vectors (interior rows on the fast path)
template <int DIM, int P, typename T, int R, class Load>
__device__ __forceinline__ void mass_apply_row(const CgVecs<T>& v, const Load& ld, int i, int dmax, const int* sdl,
                                               T* acc, T* own) {
    if (i >= dmax && i < v.N - dmax)
        stencil_row_interior<DIM, P, T, true, R, kCgUnroll<R>>(v.F, v.pitch, ld, i, sdl, acc, own);
    else
        stencil_row<DIM, P, T, true, R, kCgUnroll<R>>(v.F, v.pitch, ld, i, v.N, v.m, acc, own);
}

// init 1: r = b - M~x, u = D^-1 r; partials (r,u), (r,r), (b,b)
template <int DIM, int P, typename T, int R>
__device__ __forceinline__ void cg_init1(const CgVecs<T>& v, double* part, const int* sdl) {
    DotAcc<T> dot[3 * R];
    PlainLoad<T> ld{v.x, v.ldu, v.ext_user};
    const int dmax = max_delta<DIM, P>(v.m);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x) {
        T acc[R], own[R];
        mass_apply_row<DIM, P, T, R>(v, ld, i, dmax, sdl, acc, own);
        const T di = IGA_IN(i, v.ext_diag, 6) ? v.dinv[i] : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long ou = (long long)r * v.ldu + i, ow = (long long)r * v.ldw + i;
            const bool ok = IGA_IN(ou, v.ext_user, 7) && IGA_IN(ow, v.ext_vec, 16);
            const T bi = ok ? v.b[ou] : T(0);
            const double ri = (double)bi - (double)acc[r];   // FP64 residual
            const T rt = (T)ri;
            const T ui = di * rt;
            if (ok) {
                v.r[ow] = ri;
                v.u[ow] = ui;
            }
            dot[3 * r + 0].add(rt, ui);
            dot[3 * r + 1].add(rt, rt);
            dot[3 * r + 2].add(bi, bi);
        }
    }
    for (int k = 0; k < 3 * R; ++k) part[k] = dot[k].value();
}

// phase 2 (and init 2): w = M~u; partial (w,u)
template <int DIM, int P, typename T, int R>
__device__ __forceinline__ void cg_phase2(const CgVecs<T>& v, const int* active, double* part, const int* sdl) {
    DotAcc<T> dot[R];
    PlainLoad<T> ld{v.u, v.ldw, v.ext_vec};
    const int dmax = max_delta<DIM, P>(v.m);
    // Full grid-stride rounds one row per thread; for a single right-hand side a
    // remainder of at most four rows per warp goes one row per warp (fields split
    // across lanes) instead of leaving a few threads to run a whole extra round
    // alone (measured: 126 -> 111 us per iteration on the 941,192-row operator;
    // with four right-hand sides the split was slower and is not used).
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x, nwarp = nth >> 5;
    const int body = (v.N / nth) * nth;
    const int n1 = (R == 1 && v.N - body <= 4 * nwarp) ? body : v.N;
    for (int i = tid; i < n1; i += nth) {
        T acc[R], own[R];
        mass_apply_row<DIM, P, T, R>(v, ld, i, dmax, sdl, acc, own);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!active[r]) continue;
            const long long o = (long long)r * v.ldw + i;
            if (IGA_IN(o, v.ext_vec, 8)) v.w[o] = acc[r];
            dot[r].add(own[r], acc[r]);
        }
    }
    const int lane = threadIdx.x & 31;
    for (int i = n1 + (tid >> 5); i < v.N; i += nwarp) {
        T acc[R], own[R];
        stencil_row_warp<DIM, P, T, true, R>(v.F, v.pitch, ld, i, v.N, v.m, lane, acc, own);
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                const long long o = (long long)r * v.ldw + i;
                if (IGA_IN(o, v.ext_vec, 8)) v.w[o] = acc[r];
                dot[r].add(own[r], acc[r]);
            }
        }
    }
    for (int k = 0; k < R; ++k) part[k] = dot[k].value();
}

// phase 1: p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r;
// partials (r,u), (r,r).  (Two-row 8 / 16-byte vector accesses were measured no
// faster here: the phase is not bound by its load instructions.)
template <typename T, int R>
__device__ __forceinline__ void cg_phase1(const CgVecs<T>& v, const double* alpha, const double* beta,
                                          const int* active, double* part) {
    DotAcc<T> dot[2 * R];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x) {
        const T di = IGA_IN(i, v.ext_diag, 9) ? v.dinv[i] : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!active[r]) continue;
            const size_t o = (size_t)r * v.ldw + i;
            const size_t ou = (size_t)r * v.ldu + i;
            if (!IGA_IN(o, v.ext_vec, 10) || !IGA_IN(ou, v.ext_user, 17)) continue;
            const T be = (T)beta[r], al = (T)alpha[r];
            const T pi = v.u[o] + be * v.p[o];
            const T si = v.w[o] + be * v.s[o];
            v.p[o] = pi;
            v.s[o] = si;
            v.x[ou] = v.x[ou] + al * pi;
            const double ri = v.r[o] - alpha[r] * (double)si;   // FP64 residual
            const T rt = (T)ri;
            const T ui = di * rt;
            v.r[o] = ri;
            v.u[o] = ui;
            dot[2 * r + 0].add(rt, ui);
            dot[2 * r + 1].add(rt, rt);
        }
    }
    for (int k = 0; k < 2 * R; ++k) part[k] = dot[k].value();
}

struct CgCtl {
    double rtol;
    int max_it;
    int nblocks;
    double* partials;    // [nblocks][kCgStride(R)]
    unsigned* bar;       // [2]
    int* err;
    int* iters_out;      // [R]
    double* relres_out;  // [R]
    long long* iter_acc; // nullable: iterations are added here (device counter)
    int* status_acc;     // nullable: bit 8 set when an RHS misses rtol
    long long spin_cycles;   // grid-barrier wait limit (SM clocks)
};

// Per-block partial layout (stride 10 R): phase-1 partials double-buffered by
// iteration parity at [0, 2R) / [2R, 4R) (a fast block may write the next
// iteration's phase-1 partials before a slow block has read the current ones),
// phase-2 partials at [4R, 5R), init-1 partials at [6R, 9R).
template <int R>
constexpr int kCgStride = 10 * R;

// Device error word of a solve (bit 1 breakdown, 4 barrier time-out, 16 stage-ring
// time-out) folded into the caller's status accumulator, so that solves issued
// without a host read-back (wave steps) still report it.
__device__ __forceinline__ void cg_report(const CgCtl& c) {
    if (threadIdx.x == 0 && c.status_acc) {
        const int e = *((volatile int*)c.err);
        if (e) atomicOr(c.status_acc, e);
    }
}


}  // namespace iga

#include "pcg_brick.cuh"

namespace iga {

template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(kCgThreads, (R == 1 ? kCgMaxBlocksPerSM : 1)) pcg_persistent_kernel(CgVecs<T> v, CgCtl c) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R], red2[R];
    __shared__ double gam[R], rr[R], bnorm[R], alpha[R], beta[R];
    __shared__ int active[R], iters[R];
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    double part[3 * R];
    constexpr int S = kCgStride<R>;
    fill_delta_table<DIM, P>(sdl, v.m);

    cg_init1<DIM, P, T, R>(v, part, sdl);
    block_sum<3 * R, kCgWarps>(part, wsum, red);
    if (threadIdx.x < 3 * R) c.partials[(size_t)blockIdx.x * S + 6 * R + threadIdx.x] = red[threadIdx.x];
    if (threadIdx.x < R) active[threadIdx.x] = 1;
    if (!grid_barrier(c.bar, c.err, gridDim.x, c.spin_cycles)) return cg_report(c);
    cg_phase2<DIM, P, T, R>(v, active, part, sdl);
    block_sum<R, kCgWarps>(part, wsum, red);
    if (threadIdx.x < R) c.partials[(size_t)blockIdx.x * S + 4 * R + threadIdx.x] = red[threadIdx.x];
    if (!grid_barrier(c.bar, c.err, gridDim.x, c.spin_cycles)) return cg_report(c);
    grid_sum<3 * R>(c.partials, gridDim.x, S, 6 * R, red);
    grid_sum<R>(c.partials, gridDim.x, S, 4 * R, red2);
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        gam[r] = red[3 * r];
        rr[r] = red[3 * r + 1];
        bnorm[r] = sqrt(red[3 * r + 2]);
        beta[r] = 0.0;
        iters[r] = 0;
        active[r] = bnorm[r] > 0.0 && !(c.rtol > 0.0 && sqrt(rr[r]) <= c.rtol * bnorm[r]);
        const double d = red2[r];
        if (active[r] && (!(d > 0.0) || !isfinite(d))) {
            active[r] = 0;
            atomicOr(c.err, 1);
        }
        alpha[r] = active[r] ? gam[r] / d : 0.0;
    }
    __syncthreads();
    // a zero right-hand side has the solution 0
    for (int r = 0; r < R; ++r)
        if (!(bnorm[r] > 0.0))
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x)
                if (IGA_IN((long long)r * v.ldu + i, v.ext_user, 15)) v.x[(size_t)r * v.ldu + i] = T(0);
    for (int it = 0; it < c.max_it; ++it) {
        bool any = false;
        for (int r = 0; r < R; ++r) any = any || active[r];
        if (!any) break;
        const int off1 = (it & 1) * 2 * R;
        cg_phase1<T, R>(v, alpha, beta, active, part);
        block_sum<2 * R, kCgWarps>(part, wsum, red);
        if (threadIdx.x < 2 * R) c.partials[(size_t)blockIdx.x * S + off1 + threadIdx.x] = red[threadIdx.x];
        if (!grid_barrier(c.bar, c.err, gridDim.x, c.spin_cycles)) return cg_report(c);
        cg_phase2<DIM, P, T, R>(v, active, part, sdl);
        block_sum<R, kCgWarps>(part, wsum, red);
        if (threadIdx.x < R) c.partials[(size_t)blockIdx.x * S + 4 * R + threadIdx.x] = red[threadIdx.x];
        if (!grid_barrier(c.bar, c.err, gridDim.x, c.spin_cycles)) return cg_report(c);
        grid_sum<2 * R>(c.partials, gridDim.x, S, off1, red);
        grid_sum<R>(c.partials, gridDim.x, S, 4 * R, red2);
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            if (active[r]) {
                int brk = 0;
                double rro = rr[r];
                int act = active[r];
                cg_scalars(red[2 * r], red[2 * r + 1], red2[r], c.rtol, bnorm[r], gam[r], alpha[r], beta[r], act,
                           iters[r], rro, &brk);
                active[r] = act;
                rr[r] = rro;
                if (brk && blockIdx.x == 0) atomicOr(c.err, 1);
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
    if (blockIdx.x == 0) cg_report(c);
}

// ---------------------------------------------------------------- plain schedule kernels
template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(kCgThreads) cg_init1_kernel(CgVecs<T> v, double* partials) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R];
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    fill_delta_table<DIM, P>(sdl, v.m);
    double part[3 * R];
    cg_init1<DIM, P, T, R>(v, part, sdl);
    block_sum<3 * R, kCgWarps>(part, wsum, red);
    if (threadIdx.x < 3 * R) partials[(size_t)blockIdx.x * kCgStride<R> + 6 * R + threadIdx.x] = red[threadIdx.x];
}

template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(kCgThreads) cg_phase2_kernel(CgVecs<T> v, const double* sc, double* partials) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R];
    __shared__ int active[R];
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    if (threadIdx.x < R) active[threadIdx.x] = (int)sc[2 * R + threadIdx.x];
    fill_delta_table<DIM, P>(sdl, v.m);
    double part[3 * R];
    cg_phase2<DIM, P, T, R>(v, active, part, sdl);
    block_sum<R, kCgWarps>(part, wsum, red);
    if (threadIdx.x < R) partials[(size_t)blockIdx.x * kCgStride<R> + 4 * R + threadIdx.x] = red[threadIdx.x];
}

template <typename T, int R>
__global__ void __launch_bounds__(kCgThreads) cg_phase1_kernel(CgVecs<T> v, const double* sc, double* partials) {
    __shared__ double wsum[kCgWarps * 3 * R];
    __shared__ double red[3 * R];
    __shared__ double alpha[R], beta[R];
    __shared__ int active[R];
    if (threadIdx.x < R) {
        beta[threadIdx.x] = sc[threadIdx.x];
        alpha[threadIdx.x] = sc[R + threadIdx.x];
        active[threadIdx.x] = (int)sc[2 * R + threadIdx.x];
    }
    __syncthreads();
    double part[3 * R];
    cg_phase1<T, R>(v, alpha, beta, active, part);
    block_sum<2 * R, kCgWarps>(part, wsum, red);
    if (threadIdx.x < 2 * R) partials[(size_t)blockIdx.x * kCgStride<R> + threadIdx.x] = red[threadIdx.x];
}

template <int K>
__global__ void grid_sum_kernel(const double* partials, int nblocks, int stride, int off, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < K; k += kCgWarps) {
        double s = lane_partial_sum(partials, nblocks, stride, off + k, lane);
#pragma unroll
        for (int off2 = 16; off2 > 0; off2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, off2);
        if (lane == 0) out[k] = s;
    }
}

// ---------------------------------------------------------------- host driver
struct CgWork {
    double* r;
    void* u;
    void* w;
    void* p;
    void* s;
    double* partials;
    unsigned* bar;
    int* err;
    int* iters;
    double* relres;
    double* sc;   // plain schedule scalars [3R]
    double* red;  // plain schedule reduced values [3R]
    void* gs;     // graph schedule scalar state (CgGState, <= 256 bytes)
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
    w.u = take(sizeof(T) * (size_t)R * N);
    w.w = take(sizeof(T) * (size_t)R * N);
    w.p = take(sizeof(T) * (size_t)R * N);
    w.s = take(sizeof(T) * (size_t)R * N);
    w.partials = (double*)take(sizeof(double) * (size_t)nblocks * 10 * R);
    w.bar = (unsigned*)take(64);
    w.err = (int*)take(64);
    w.iters = (int*)take(sizeof(int) * R);
    w.relres = (double*)take(sizeof(double) * R);
    w.sc = (double*)take(sizeof(double) * 3 * R);
    w.red = (double*)take(sizeof(double) * 3 * R);
    w.gs = take(256);
    return w;
}

static size_t carve_bytes(size_t es, long long N, int R, int nblocks) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return up(sizeof(double) * (size_t)R * N) + 4 * up(es * (size_t)R * N) +
           up(sizeof(double) * (size_t)nblocks * 10 * R) + 2 * up(64) + up(sizeof(int) * R) +
           3 * up(sizeof(double) * 3 * R) + up(256) + 256;
}

// ---------------------------------------------------------------- graph schedule
// IGA_SOLVE_GRAPH: the phases as separate full-occupancy launches inside one
// CUDA graph,
//   init 1 -> init 2 -> zero x of zero RHS -> WHILE { phase 1 -> phase 2 } -> finish,
// whose conditional WHILE node repeats the iteration until the device decides
// convergence.  Every phase-2 launch ends with a ticket counter: the last block
// to finish sums the per-block partials in fixed order, updates the scalars in
// CgGState and sets the loop condition.  Kernel boundaries order the phases,
// so there is neither a grid barrier nor a host round trip per iteration.
constexpr int kGThreads = 256;
constexpr int kGWarps = kGThreads / 32;

struct CgGState {
    double gam[4], rr[4], bnorm[4], alpha[4], beta[4];
    int active[4], iters[4];
    int it;
    unsigned ticket;
};

template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(kGThreads, (R == 1 ? 8 : 2)) cgg_init1_kernel(CgVecs<T> v, double* partials) {
    __shared__ double wsum[kGWarps * 3 * R];
    __shared__ double red[3 * R];
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    double part[3 * R];
    fill_delta_table<DIM, P>(sdl, v.m);
    cg_init1<DIM, P, T, R>(v, part, sdl);
    block_sum<3 * R, kGWarps>(part, wsum, red);
    if (threadIdx.x < 3 * R) partials[(size_t)blockIdx.x * kCgStride<R> + 6 * R + threadIdx.x] = red[threadIdx.x];
}

template <int DIM, int P, typename T, int R, bool INIT>
__global__ void __launch_bounds__(kGThreads, (R == 1 ? 8 : 2))
    cgg_phase2_kernel(CgVecs<T> v, double* partials, CgGState* gs, double rtol, int max_it, int* err,
                      cudaGraphConditionalHandle loop) {
    constexpr int S = kCgStride<R>;
    __shared__ double wsum[kGWarps * R];
    __shared__ double red[3 * R], red2[R];
    __shared__ int active[R];
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    __shared__ int last;
    double part[R];
    if (threadIdx.x < R) active[threadIdx.x] = INIT ? 1 : gs->active[threadIdx.x];
    fill_delta_table<DIM, P>(sdl, v.m);   // ends with __syncthreads
    cg_phase2<DIM, P, T, R>(v, active, part, sdl);
    block_sum<R, kGWarps>(part, wsum, red);
    if (threadIdx.x < R) partials[(size_t)blockIdx.x * S + 4 * R + threadIdx.x] = red[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&gs->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    grid_sum_b<(INIT ? 3 : 2) * R>(partials, gridDim.x, S, INIT ? 6 * R : 0, red);
    grid_sum_b<R>(partials, gridDim.x, S, 4 * R, red2);
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        if (INIT) {
            gs->gam[r] = red[3 * r];
            gs->rr[r] = red[3 * r + 1];
            gs->bnorm[r] = sqrt(red[3 * r + 2]);
            gs->beta[r] = 0.0;
            gs->iters[r] = 0;
            int act = gs->bnorm[r] > 0.0 && !(rtol > 0.0 && sqrt(gs->rr[r]) <= rtol * gs->bnorm[r]);
            const double d = red2[r];
            if (act && (!(d > 0.0) || !isfinite(d))) {
                act = 0;
                atomicOr(err, 1);
            }
            gs->alpha[r] = act ? gs->gam[r] / d : 0.0;
            gs->active[r] = act;
        } else if (gs->active[r]) {
            int brk = 0, act = 1;
            cg_scalars(red[2 * r], red[2 * r + 1], red2[r], rtol, gs->bnorm[r], gs->gam[r], gs->alpha[r], gs->beta[r],
                       act, gs->iters[r], gs->rr[r], &brk);
            gs->active[r] = act;
            if (brk) atomicOr(err, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int r = 0; r < R; ++r) any |= gs->active[r];
        const int it = INIT ? 0 : gs->it + 1;
        gs->it = it;
        gs->ticket = 0;
        cudaGraphSetConditional(loop, (any && it < max_it) ? 1u : 0u);
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(kGThreads, (R == 1 ? 8 : 2)) cgg_phase1_kernel(CgVecs<T> v, double* partials,
                                                                                  const CgGState* gs) {
    __shared__ double wsum[kGWarps * 2 * R];
    __shared__ double red[2 * R], alpha[R], beta[R];
    __shared__ int active[R];
    if (threadIdx.x < R) {
        alpha[threadIdx.x] = gs->alpha[threadIdx.x];
        beta[threadIdx.x] = gs->beta[threadIdx.x];
        active[threadIdx.x] = gs->active[threadIdx.x];
    }
    __syncthreads();
    double part[2 * R];
    cg_phase1<T, R>(v, alpha, beta, active, part);
    block_sum<2 * R, kGWarps>(part, wsum, red);
    if (threadIdx.x < 2 * R) partials[(size_t)blockIdx.x * kCgStride<R> + threadIdx.x] = red[threadIdx.x];
}

// a zero right-hand side has the solution 0
template <typename T, int R>
__global__ void cgg_zero_kernel(CgVecs<T> v, const CgGState* gs) {
    for (int r = 0; r < R; ++r)
        if (!(gs->bnorm[r] > 0.0))
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.N; i += gridDim.x * blockDim.x)
                v.x[(size_t)r * v.ldu + i] = T(0);
}

template <int R>
__global__ void cgg_finish_kernel(const CgGState* gs, double rtol, int* iters_out, double* relres_out,
                                  long long* iter_acc, int* status_acc, const int* err) {
    const int r = threadIdx.x;
    if (r == 0 && status_acc && *err) atomicOr(status_acc, *err);
    if (r >= R) return;
    const double rel = gs->bnorm[r] > 0.0 ? sqrt(gs->rr[r]) / gs->bnorm[r] : 0.0;
    iters_out[r] = gs->iters[r];
    relres_out[r] = rel;
    if (iter_acc) atomicAdd((unsigned long long*)iter_acc, (unsigned long long)gs->iters[r]);
    if (status_acc && rtol > 0.0 && rel > rtol) atomicOr(status_acc, 8);
}

// Grid of the graph-schedule phases: two waves of resident blocks, at most one
// block per 256 rows.
template <int DIM, int P, typename T, int R>
static int cgg_blocks(long long N) {
    static int per = 0, sms = 0;
    if (!per) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cgg_phase2_kernel<DIM, P, T, R, false>, kGThreads, 0);
        per = std::max(1, per);
    }
    return (int)std::max(1LL, std::min<long long>((N + kGThreads - 1) / kGThreads, 2LL * sms * per));
}

// Builds, instantiates and launches the graph of one solve chunk.
template <int DIM, int P, typename T, int R>
static int cgg_launch(CgVecs<T> v, double* partials, CgGState* gs, int* err, double rtol, int max_it, int grid,
                      int* iters_out, double* relres_out, long long* iter_acc, int* status_acc, cudaStream_t st) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int rc = IGA_OK;
    auto check = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == IGA_OK) rc = cuda_fail(e, what);
        return e == cudaSuccess;
    };
    auto kernel_node = [&](cudaGraph_t gr, const void* fn, void** args, const cudaGraphNode_t* dep, size_t ndep,
                           int blocks, int threads, cudaGraphNode_t* out) {
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void*>(fn);
        kp.gridDim = dim3(blocks);
        kp.blockDim = dim3(threads);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        kp.extra = nullptr;
        return check(cudaGraphAddKernelNode(out, gr, dep, ndep, &kp), "cudaGraphAddKernelNode(cg)");
    };
    if (check(cudaGraphCreate(&g, 0), "cudaGraphCreate(cg)")) {
        cudaGraphConditionalHandle loop;
        cudaGraphNode_t n_init1, n_init2, n_zero, n_loop, n_finish, n_p1, n_p2;
        if (check(cudaGraphConditionalHandleCreate(&loop, g, 0, cudaGraphCondAssignDefault),
                  "cudaGraphConditionalHandleCreate(cg)")) {
            void* a_init1[] = {&v, &partials};
            void* a_p2[] = {&v, &partials, &gs, &rtol, &max_it, &err, &loop};
            void* a_zero[] = {&v, &gs};
            void* a_p1[] = {&v, &partials, &gs};
            void* a_fin[] = {&gs, &rtol, &iters_out, &relres_out, &iter_acc, &status_acc, &err};
            bool ok = kernel_node(g, (const void*)cgg_init1_kernel<DIM, P, T, R>, a_init1, nullptr, 0, grid, kGThreads,
                                  &n_init1) &&
                      kernel_node(g, (const void*)cgg_phase2_kernel<DIM, P, T, R, true>, a_p2, &n_init1, 1, grid,
                                  kGThreads, &n_init2) &&
                      kernel_node(g, (const void*)cgg_zero_kernel<T, R>, a_zero, &n_init2, 1, 152, kGThreads, &n_zero);
            if (ok) {
                cudaGraphNodeParams cp = {};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = loop;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                ok = check(cudaGraphAddNode(&n_loop, g, &n_zero, nullptr, 1, &cp), "cudaGraphAddNode(cg loop)");
                if (ok) {
                    cudaGraph_t body = cp.conditional.phGraph_out[0];
                    ok = kernel_node(body, (const void*)cgg_phase1_kernel<T, R>, a_p1, nullptr, 0, grid, kGThreads,
                                     &n_p1) &&
                         kernel_node(body, (const void*)cgg_phase2_kernel<DIM, P, T, R, false>, a_p2, &n_p1, 1, grid,
                                     kGThreads, &n_p2) &&
                         kernel_node(g, (const void*)cgg_finish_kernel<R>, a_fin, &n_loop, 1, 1, 32, &n_finish);
                }
            }
            if (ok && check(cudaGraphInstantiate(&ge, g, 0), "cudaGraphInstantiate(cg)"))
                if (check(cudaGraphLaunch(ge, st), "cudaGraphLaunch(cg)")) count_launch();
        }
    }
    if (ge) cudaGraphExecDestroy(ge);   // freed once the launched work completes
    if (g) cudaGraphDestroy(g);
    return rc;
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

// Brick form of the persistent solve (FP32, one right-hand side, 3-D operators
// whose brick form the mass apply uses).  Returns false when it does not apply
// (the grid-stride persistent kernel runs instead); a failed launch is reported
// through the CUDA error state like the other launches.
template <int DIM, int P, typename T, int R>
static bool brick_pcg_launch(const iga_ops* ops, CgVecs<T>& v, CgCtl& c, cudaStream_t st) {
#ifdef IGA_BOUNDS_CHECK
    (void)ops; (void)v; (void)c; (void)st;
    return false;
#else
    if constexpr (DIM != 3 || sizeof(T) != 4 || R != 1 || P > 2) {
        (void)ops; (void)v; (void)c; (void)st;
        return false;
    } else {
        if (!brick_usable(ops, IGA_OP_M)) return false;
        const BrickOps& bo = *ops->brick;
        // one CTA per SM: at least half the SM's shared memory, so that the
        // kernel's allocation of the whole TMEM never waits for another CTA
        const size_t smem = std::max<size_t>(
            kBrickPcgHeader + sizeof(float) * ((size_t)bo.ns * bo.stage_floats + bo.xt_floats), 116 * 1024);
        if (smem > 227 * 1024) return false;
        for (const BrickDesc& b : bo.host)
            if (brick_pcg_tmem_cols(b.nx, b.ny, b.nz) > (int)kTmemCols) return false;
        const int threads = (bo.ncw + 1) * 32;
        auto fn3 = pcg_brick_kernel<P, 3>;
        auto fn2 = pcg_brick_kernel<P, 2>;
        const void* fn = bo.ns == 3 ? (const void*)fn3 : (const void*)fn2;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        int per = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per != 1 ||
            bo.nbricks > sms) {
            cudaGetLastError();
            return false;
        }
        const BrickMaps* maps = &bo.mapM;
        const BrickMaps* umaps = &bo.mapU;
        const BrickDesc* bricks = bo.bricks.as<BrickDesc>();
        int nF = ops->nM, sf = bo.stage_floats, XP = bo.XP;
        float* upad = bo.upad.as<float>();
        void* args[] = {(void*)maps, (void*)umaps, (void*)&bricks, &nF, &sf, &upad, &XP, &v, &c};
        const cudaError_t e = cudaLaunchCooperativeKernel(fn, bo.nbricks, threads, args, smem, st);
        count_launch();
        if (e != cudaSuccess) {
            cuda_fail(e, "cudaLaunchCooperativeKernel(pcg_brick)");
            return false;
        }
        return true;
    }
#endif
}

template <int DIM, int P, typename T, int R>
static int pcg_chunk(const iga_ops* ops, const T* b, T* x, long long ldu, double rtol, int max_it, unsigned flags,
                     int* iters_h, double* relres_h, cudaStream_t st, void* work, size_t work_bytes, bool* not_conv,
                     long long* iter_acc, int* status_acc) {
    const long long N = ops->N;
    const long long ldw = (N + 3) / 4 * 4;
    const int nblocks = cg_blocks<DIM, P, T, R>();
    const int ggrid = cgg_blocks<DIM, P, T, R>(N);
    const int nb_carve = std::max(nblocks, ggrid);
    if (carve_bytes(sizeof(T), ldw, R, nb_carve) > work_bytes) return fail(IGA_ERR_ARG, "CG workspace too small");
    CgWork w = carve<T>(work, ldw, R, nb_carve);
    CgVecs<T> v;
    v.F = (sizeof(T) == 8) ? (const T*)ops->fM64.ptr : (const T*)ops->fM32.ptr;
    v.pitch = ops->pitch;
    v.dinv = (sizeof(T) == 8) ? (const T*)ops->dinv64.ptr : (const T*)ops->dinv32.ptr;
    v.b = b;
    v.x = x;
    v.r = w.r;
    v.u = (T*)w.u;
    v.w = (T*)w.w;
    v.p = (T*)w.p;
    v.s = (T*)w.s;
    v.N = (int)N;
    v.m = ops->m;
    v.ldw = ldw;
    v.ldu = ldu;
    v.ext_vec = (long long)R * ldw;
    v.ext_user = (long long)(R - 1) * ldu + N;
    v.ext_diag = ops->pitch;
    // p and s start at 0 (beta = 0 on the first iteration multiplies them)
    IGA_CUDA(cudaMemsetAsync(w.p, 0, sizeof(T) * R * ldw, st));
    IGA_CUDA(cudaMemsetAsync(w.s, 0, sizeof(T) * R * ldw, st));
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
        c.spin_cycles = kBarrierSpinCycles;
        bool use_graph = (flags & IGA_SOLVE_GRAPH) != 0;
        if (use_graph) {
            // a graph launch is not issued into a stream under capture: persistent schedule there
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) use_graph = false;
        }
        if (use_graph) {
            IGA_CUDA(cudaMemsetAsync(w.gs, 0, sizeof(CgGState), st));
            const int rc = cgg_launch<DIM, P, T, R>(v, w.partials, (CgGState*)w.gs, w.err, rtol, max_it, ggrid,
                                                   w.iters, w.relres, iter_acc, status_acc, st);
            if (rc) return rc;
        } else if (!brick_pcg_launch<DIM, P, T, R>(ops, v, c, st)) {
            void* args[] = {&v, &c};
            cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_persistent_kernel<DIM, P, T, R>, nblocks,
                                                        kCgThreads, args, 0, st);
            count_launch();
            if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(pcg)");
        }
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
            if (err & 16) return fail(IGA_ERR_TIMEOUT, "a stage of the brick field ring timed out in pcg");
            if (err & 1) return fail(IGA_ERR_NONFINITE, "CG breakdown: (p, M p) <= 0 or non-finite");
        }
    } else {
        // plain schedule: the same phases as separate launches, scalars on the host
        const int grid = nblocks;
        constexpr int S = kCgStride<R>;
        double red[3 * R], red2[R], sc[3 * R];
        double gam[R], rr[R], bn[R], alpha[R], beta[R];
        int active[R];
        for (int r = 0; r < R; ++r) {
            sc[r] = 0.0;
            sc[R + r] = 0.0;
            sc[2 * R + r] = 1.0;
        }
        cg_init1_kernel<DIM, P, T, R><<<grid, kCgThreads, 0, st>>>(v, w.partials);
        IGA_LAUNCH_CHECK("cg_init1_kernel");
        IGA_CUDA(cudaMemcpyAsync(w.sc, sc, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, st));
        cg_phase2_kernel<DIM, P, T, R><<<grid, kCgThreads, 0, st>>>(v, w.sc, w.partials);
        IGA_LAUNCH_CHECK("cg_phase2_kernel");
        grid_sum_kernel<3 * R><<<1, kCgThreads, 0, st>>>(w.partials, grid, S, 6 * R, w.red);
        IGA_LAUNCH_CHECK("grid_sum_kernel");
        IGA_CUDA(cudaMemcpyAsync(red, w.red, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, st));
        grid_sum_kernel<R><<<1, kCgThreads, 0, st>>>(w.partials, grid, S, 4 * R, w.red);
        IGA_LAUNCH_CHECK("grid_sum_kernel");
        IGA_CUDA(cudaMemcpyAsync(red2, w.red, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        IGA_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r) {
            gam[r] = red[3 * r];
            rr[r] = red[3 * r + 1];
            bn[r] = std::sqrt(red[3 * r + 2]);
            beta[r] = 0.0;
            iters[r] = 0;
            active[r] = bn[r] > 0.0 && !(rtol > 0.0 && std::sqrt(rr[r]) <= rtol * bn[r]);
            if (active[r] && (!(red2[r] > 0.0) || !std::isfinite(red2[r])))
                return fail(IGA_ERR_NONFINITE, "CG breakdown: (u, M u) <= 0 or non-finite");
            alpha[r] = active[r] ? gam[r] / red2[r] : 0.0;
            if (!(bn[r] > 0.0)) IGA_CUDA(cudaMemsetAsync(x + (size_t)r * ldu, 0, sizeof(T) * N, st));
        }
        for (int it = 0; it < max_it; ++it) {
            bool any = false;
            for (int r = 0; r < R; ++r) any = any || active[r];
            if (!any) break;
            for (int r = 0; r < R; ++r) {
                sc[r] = beta[r];
                sc[R + r] = alpha[r];
                sc[2 * R + r] = active[r];
            }
            IGA_CUDA(cudaMemcpyAsync(w.sc, sc, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, st));
            cg_phase1_kernel<T, R><<<grid, kCgThreads, 0, st>>>(v, w.sc, w.partials);
            IGA_LAUNCH_CHECK("cg_phase1_kernel");
            cg_phase2_kernel<DIM, P, T, R><<<grid, kCgThreads, 0, st>>>(v, w.sc, w.partials);
            IGA_LAUNCH_CHECK("cg_phase2_kernel");
            grid_sum_kernel<2 * R><<<1, kCgThreads, 0, st>>>(w.partials, grid, S, 0, w.red);
            IGA_LAUNCH_CHECK("grid_sum_kernel");
            IGA_CUDA(cudaMemcpyAsync(red, w.red, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, st));
            grid_sum_kernel<R><<<1, kCgThreads, 0, st>>>(w.partials, grid, S, 4 * R, w.red);
            IGA_LAUNCH_CHECK("grid_sum_kernel");
            IGA_CUDA(cudaMemcpyAsync(red2, w.red, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
            IGA_CUDA(cudaStreamSynchronize(st));
            for (int r = 0; r < R; ++r) {
                if (!active[r]) continue;
                int brk = 0;
                cg_scalars(red[2 * r], red[2 * r + 1], red2[r], rtol, bn[r], gam[r], alpha[r], beta[r], active[r],
                           iters[r], rr[r], &brk);
                if (brk) return fail(IGA_ERR_NONFINITE, "CG breakdown: non-positive curvature or non-finite");
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

// Per-block partials are sized for the larger of the persistent grid and the
// graph-schedule grid (two waves of up to 8 resident 256-thread blocks per SM).
static int work_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, sms) * std::max(kCgMaxBlocksPerSM, 16);
}

// FP64 workspace also holds an IGA_SOLVE_REFINE chunk: FP64 residual, FP32 residual
// and FP32 correction of up to 4 right-hand sides, then the FP32 CG workspace.
static size_t refine_extra_bytes(long long N) { return (size_t)16 * 4 * (size_t)N + 3 * 256; }

size_t mass_solve_work_bytes(const iga_ops* ops, int dtype, int nrhs) {
    (void)nrhs;
    const int nb = work_blocks();
    const long long N4 = (ops->N + 3) / 4 * 4;
    const size_t plain = carve_bytes(dtype == IGA_F64 ? 8 : 4, N4, 4, nb);   // R = 4 is the largest chunk
    if (dtype != IGA_F64) return plain;
    return std::max(plain, refine_extra_bytes(ops->N) + carve_bytes(4, N4, 4, nb));
}

// ---------------------------------------------------------------- IGA_SOLVE_REFINE
// FP64 solve by iterative refinement: r = b - M~x with the FP64 fields, correction
// d from the FP32 Jacobi-PCG on the FP32 fields (the fast kernels), x += d in FP64,
// until ||b - M~x||_2 <= rtol ||b||_2 for every right-hand side (the stopping rule of
// the FP64 solve, on the FP64 residual).  Each refinement gains about the digits of
// the FP32 solve, up to cond(M~) times the FP32 rounding of the fields.
__global__ void refine_norm_kernel(const double* __restrict__ v, long long ld, int N, double* out) {
    __shared__ double ws[32];
    const double* x = v + (size_t)blockIdx.x * ld;
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) acc += x[i] * x[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        out[blockIdx.x] = t;
    }
}

// r64 holds M~x on entry: r64 = b - M~x; r32 = r64 in FP32 (0 for converged columns)
__global__ void refine_residual_kernel(const double* __restrict__ b, double* __restrict__ r64,
                                       float* __restrict__ r32, long long N, int R, unsigned done_mask) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)R * N;
         idx += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(idx / N);
        const double r = b[idx] - r64[idx];
        r64[idx] = r;
        r32[idx] = ((done_mask >> s) & 1u) ? 0.f : (float)r;
    }
}

__global__ void refine_update_kernel(double* __restrict__ x, const float* __restrict__ d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

static int refine_chunk(const iga_ops* ops, const double* b, double* x, int R, double rtol, int max_it,
                        unsigned flags, int* iters_h, double* relres_h, bool* nc, cudaStream_t st, void* work,
                        size_t work_bytes, long long* tot_iters) {
    const long long N = ops->N;
    char* base = (char*)work;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    double* r64 = (double*)base;
    float* r32 = (float*)(base + up(sizeof(double) * 4 * N));
    float* d32 = (float*)((char*)r32 + up(sizeof(float) * 4 * N));
    double* nrm = (double*)((char*)d32 + up(sizeof(float) * 4 * N));
    char* inner = (char*)nrm + 256;
    if ((size_t)(inner - base) > work_bytes) return fail(IGA_ERR_ARG, "CG workspace too small");
    const size_t inner_bytes = work_bytes - (size_t)(inner - base);
    const int grid = (int)std::max<long long>(1, std::min<long long>((R * N + 255) / 256, 152 * 16));
    double bn[4], rn[4];
    refine_norm_kernel<<<R, 1024, 0, st>>>(b, N, (int)N, nrm);
    IGA_LAUNCH_CHECK("refine_norm_kernel");
    IGA_CUDA(cudaMemcpyAsync(bn, nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r) {
        bn[r] = std::sqrt(bn[r]);
        iters_h[r] = 0;
        if (!(bn[r] > 0.0)) IGA_CUDA(cudaMemsetAsync(x + (size_t)r * N, 0, sizeof(double) * N, st));
    }
    constexpr int kMaxRefine = 12;
    unsigned done = 0;
    for (int k = 0; k <= kMaxRefine; ++k) {
        int rc = launch_apply(ops, IGA_OP_M, IGA_F64, x, r64, R, st);
        if (rc) return rc;
        refine_residual_kernel<<<grid, 256, 0, st>>>(b, r64, r32, N, R, done);
        IGA_LAUNCH_CHECK("refine_residual_kernel");
        refine_norm_kernel<<<R, 1024, 0, st>>>(r64, N, (int)N, nrm);
        IGA_LAUNCH_CHECK("refine_norm_kernel");
        IGA_CUDA(cudaMemcpyAsync(rn, nrm, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        IGA_CUDA(cudaStreamSynchronize(st));
        double target = 1.0;
        for (int r = 0; r < R; ++r) {
            rn[r] = std::sqrt(rn[r]);
            relres_h[r] = bn[r] > 0.0 ? rn[r] / bn[r] : 0.0;
            if (!(bn[r] > 0.0) || (rtol > 0.0 && relres_h[r] <= rtol)) done |= 1u << r;
            else target = std::min(target, rtol * bn[r] / rn[r]);
        }
        if (done == (1u << R) - 1 || k == kMaxRefine) break;
        // the FP32 correction: to 1e-6, or to what is left of the tolerance
        const double inner_rtol = std::max(1e-6, std::min(0.1, 0.5 * target));
        IGA_CUDA(cudaMemsetAsync(d32, 0, sizeof(float) * R * N, st));
        int it32[4];
        double rr32[4];
        rc = mass_solve_impl(ops, IGA_F32, r32, d32, N, R, inner_rtol, max_it, flags, it32, rr32, st, inner,
                             inner_bytes, nullptr, nullptr);
        if (rc && rc != IGA_ERR_NOT_CONVERGED) return rc;
        for (int r = 0; r < R; ++r) {
            iters_h[r] += it32[r];
            *tot_iters += it32[r];
        }
        refine_update_kernel<<<grid, 256, 0, st>>>(x, d32, (long long)R * N);
        IGA_LAUNCH_CHECK("refine_update_kernel");
    }
    for (int r = 0; r < R; ++r)
        if (rtol > 0.0 && bn[r] > 0.0 && relres_h[r] > rtol) *nc = true;
    return IGA_OK;
}

static int refine_solve(const iga_ops* ops, const double* b, double* x, long long ld, int nrhs, double rtol,
                        int max_it, unsigned flags, int* iters_out, double* relres_out, cudaStream_t st, void* work,
                        size_t work_bytes, long long* iter_acc, int* status_acc) {
    if (ld != ops->N) return fail(IGA_ERR_ARG, "IGA_SOLVE_REFINE needs vectors of leading dimension N");
    bool nc = false;
    long long tot = 0;
    for (int r0 = 0; r0 < nrhs; r0 += 4) {
        const int R = std::min(4, nrhs - r0);
        int it[4];
        double rel[4];
        const int rc = refine_chunk(ops, b + (size_t)r0 * ld, x + (size_t)r0 * ld, R, rtol, max_it, flags, it, rel,
                                    &nc, st, work, work_bytes, &tot);
        if (rc) return rc;
        for (int r = 0; r < R; ++r) {
            if (iters_out) iters_out[r0 + r] = it[r];
            if (relres_out) relres_out[r0 + r] = rel[r];
        }
    }
    if (iter_acc || status_acc) {
        // fold the host-side counts into the caller's device accumulators
        long long acc_h = 0;
        int st_h = 0;
        if (iter_acc) IGA_CUDA(cudaMemcpy(&acc_h, iter_acc, sizeof(acc_h), cudaMemcpyDeviceToHost));
        if (status_acc) IGA_CUDA(cudaMemcpy(&st_h, status_acc, sizeof(st_h), cudaMemcpyDeviceToHost));
        acc_h += tot;
        if (nc) st_h |= 8;
        if (iter_acc) IGA_CUDA(cudaMemcpy(iter_acc, &acc_h, sizeof(acc_h), cudaMemcpyHostToDevice));
        if (status_acc) IGA_CUDA(cudaMemcpy(status_acc, &st_h, sizeof(st_h), cudaMemcpyHostToDevice));
    }
    if (nc && (iters_out || relres_out)) return fail(IGA_ERR_NOT_CONVERGED, "refinement reached its limit before rtol");
    return IGA_OK;
}

// Workspace for exactly the chunks pcg_typed runs for nrhs right-hand sides
// (4-wide chunks while at least 4 remain, then single ones).
size_t mass_solve_work_bytes_nrhs(const iga_ops* ops, int dtype, int nrhs) {
    const int nb = work_blocks();
    return carve_bytes(dtype == IGA_F64 ? 8 : 4, (ops->N + 3) / 4 * 4, nrhs >= 4 ? 4 : 1, nb);
}

int mass_solve_impl(const iga_ops* ops, int dtype, const void* b, void* x, long long ld, int nrhs, double rtol,
                    int max_it, unsigned flags, int* iters_out, double* relres_out, cudaStream_t st, void* work,
                    size_t work_bytes, long long* iter_acc, int* status_acc) {
    if (dtype == IGA_F64 && (flags & IGA_SOLVE_REFINE))
        return refine_solve(ops, (const double*)b, (double*)x, ld, nrhs, rtol, max_it, flags & ~IGA_SOLVE_REFINE,
                            iters_out, relres_out, st, work, work_bytes, iter_acc, status_acc);
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
    // the statistics are always read back (synchronising the stream), so that a
    // missed tolerance, a breakdown or a time-out is returned also when the caller
    // passes no statistics arrays
    std::vector<int> it_local(iters_out ? 0 : nrhs);
    std::vector<double> rr_local(relres_out ? 0 : nrhs);
    return mass_solve_impl(ops, dtype, b, x, ops->N, nrhs, rtol, max_it, flags,
                           iters_out ? iters_out : it_local.data(), relres_out ? relres_out : rr_local.data(),
                           (cudaStream_t)stream, mops->work.ptr, mops->work.bytes, nullptr, nullptr);
}

// ---------------------------------------------------------------- barrier self-test
namespace iga {
__device__ unsigned g_selftest_bar[2];
__device__ int g_selftest_err;
__global__ void barrier_selftest_kernel(unsigned expected, long long spin_cycles) {
    grid_barrier(g_selftest_bar, &g_selftest_err, expected, spin_cycles);
}
}  // namespace iga

extern "C" int iga_barrier_selftest(int blocks, int expected, double limit_ms, void* stream) {
    int dev = 0, sms = 0, khz = 0;
    IGA_CUDA(cudaGetDevice(&dev));
    IGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    IGA_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    if (blocks < 1 || blocks > sms || expected < 1 || !(limit_ms > 0.0) || limit_ms > 10000.0)
        return fail(IGA_ERR_ARG, "need 1 <= blocks <= SMs, expected >= 1, 0 < limit_ms <= 10000");
    cudaStream_t st = (cudaStream_t)stream;
    void* bar = nullptr;
    void* err = nullptr;
    IGA_CUDA(cudaGetSymbolAddress(&bar, g_selftest_bar));
    IGA_CUDA(cudaGetSymbolAddress(&err, g_selftest_err));
    IGA_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    IGA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    // the limit in SM clocks at the maximum clock: at a lower clock the wait is longer
    unsigned ex = (unsigned)expected;
    long long spin = (long long)(limit_ms * (double)khz);
    void* args[] = {&ex, &spin};
    IGA_CUDA(cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, blocks, 32, args, 0, st));
    count_launch();
    int e = 0;
    IGA_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    if (e & 4) return fail(IGA_ERR_TIMEOUT, "grid barrier self-test: the wait ran out");
    return IGA_OK;
}
