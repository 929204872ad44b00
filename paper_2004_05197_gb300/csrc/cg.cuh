// Device helpers of the persistent Jacobi-PCG kernels (single problem and
// batched): deterministic block reductions, the bounded grid / partition
// barrier, and the Chronopoulos-Gear scalar recurrence.
#pragma once

#include "iga_internal.cuh"

namespace iga {

constexpr long long kBarrierSpinCycles = 4000000000LL;   // ~2 s at 2 GHz

// Block sum of K doubles per thread (v[K]) into red[K] (shared), fixed order.
template <int K, int kWarps>
__device__ __forceinline__ void block_sum(double* v, double* wsum /*[kWarps][K]*/, double* red /*[K]*/) {
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
        for (int ww = 0; ww < kWarps; ++ww) s += wsum[ww * K + k];
        red[k] = s;
    }
    __syncthreads();
}

// Bounded barrier over `nblocks` co-resident blocks (a whole cooperative grid or
// one partition of it).  A block that waits longer than spin_cycles SM clocks
// sets bit 4 of *err and returns false; every caller then leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned nblocks,
                                             long long spin_cycles = kBarrierSpinCycles) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == gen) {
                __nanosleep(32);
                if (clock64() - t0 > spin_cycles) {
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

// Scalar update shared by the persistent and plain schedules (thread r of a block).
__device__ __host__ inline void cg_scalars(double gamma_new, double rr, double delta, double rtol, double bnorm,
                                           double& gamma, double& alpha, double& beta, int& active, int& iters,
                                           double& rr_out, int* breakdown) {
    iters += 1;
    rr_out = rr;
    if (rtol > 0.0 && sqrt(rr) <= rtol * bnorm) {
        active = 0;
        return;
    }
    const double b = gamma_new / gamma;
    const double den = delta - b * gamma_new / alpha;
    if (!(den > 0.0) || !isfinite(den)) {
        active = 0;
        *breakdown = 1;
        return;
    }
    beta = b;
    alpha = gamma_new / den;
    gamma = gamma_new;
}

// Per-thread dot-product accumulator.  FP64 path: plain FP64 products and sums.
// FP32 path: each product of two FP32 numbers is split exactly into p + e
// (TwoProd through fmaf) and added to an unevaluated pair hi + lo with Knuth's
// TwoSum, so a thread's partial sum carries about 48 significant bits while
// using FP32 instructions only; the pair is widened to FP64 for the block and
// grid reductions.  (On this part the FP64 pipe issues about 1.6 DFMA per clock
// and SM against about 117 FFMA: per-row FP64 products cost more time than the
// row's memory traffic.)  The explicit _rn intrinsics keep the compiler from
// contracting the TwoSum steps into FMAs.
template <typename T>
struct DotAcc {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s += a * b; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Coherent loads of vectors written inside the same persistent launch.
template <typename T>
struct PlainLoadB {
    const T* x;
    long long xs;
    __device__ __forceinline__ T operator()(int r, int idx) const { return x[r * xs + idx]; }
};

// One lane's share of a fixed-order sum over blocks: partials[b * stride + idx]
// for b = lane, lane + 32, ... in increasing b.  The loads of sixteen consecutive
// terms are issued before they are added (same order, so the same result), so a
// sum over up to 512 blocks waits for L2 latency once (eight terms per batch
// measured 1 us per CG iteration slower with 304 blocks: two round trips).
__device__ __forceinline__ double lane_partial_sum(const double* partials, int nblocks, int stride, int idx,
                                                   int lane) {
    double s = 0.0;
    for (int b0 = lane; b0 < nblocks; b0 += 32 * 16) {
        double v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int b = b0 + 32 * j;
            v[j] = b < nblocks ? __ldcg(partials + (size_t)b * stride + idx) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (b0 + 32 * j < nblocks) s += v[j];
    }
    return s;
}

// Sum over the blocks of a partition of partials[b * stride + off + k] (k < K)
// into out[k] (shared); fixed order, so every block gets the identical value.
template <int K>
__device__ __forceinline__ void grid_sum_b(const double* partials, int nblocks, int stride, int off, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = w; k < K; k += nw) {
        double s = lane_partial_sum(partials, nblocks, stride, off + k, lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[k] = s;
    }
    __syncthreads();
}

}  // namespace iga
