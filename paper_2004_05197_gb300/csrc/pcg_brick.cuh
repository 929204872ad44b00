// Brick form of the persistent Jacobi-PCG (FP32 dtype, one right-hand side, 3-D
// operators with a brick form).  Same recurrence, precision and stopping rule as
// pcg_persistent_kernel (Chronopoulos-Gear form; FP64 residual, compensated FP32
// dot products widened to FP64, fixed-order reductions), with the rows owned by
// bricks instead of a grid-stride loop:
//   * one CTA per brick for the whole solve (cooperative launch, one wave);
//   * phase 1 updates the brick's own rows (p, s, x, r, u and the partials of
//     (r,u), (r,r));
//   * phase 2 loads the u tile of the brick grown by p (coherent loads: u was
//     written by the neighbouring CTAs in phase 1), applies M~ with the brick
//     kernels of brick.cuh, writes w and the partial of (w,u);
//   * the phases are separated by a bounded grid barrier among the compute
//     warps; the producer warp streams the M~ fields through the stage ring
//     without waiting for the vectors (the fields are the same every pass), so
//     the ring refills during phase 1 and the barriers.
#pragma once

#include "brick.cuh"

namespace iga {

// Grid barrier among the compute warps (named barrier 2); the producer warp does
// not take part.  The counter only grows: barrier number e of a launch (epoch,
// counted by every CTA) is passed once it reaches e * nblocks, so an arrival is a
// single atomic and nothing is reset in between.  The counter is zero at launch.
// Bounded: on time-out bit 4 of *err is set and every caller leaves.
__device__ __forceinline__ bool compute_grid_barrier(unsigned* bar, int* err, unsigned nblocks, int ncw,
                                                     long long spin_cycles, unsigned long long& epoch) {
    named_bar_sync(2, ncw * 32);
    epoch += 1;
    if (threadIdx.x == 0) {
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(bar);
        const unsigned long long target = epoch * nblocks;
        __threadfence();
        const unsigned long long old = atomicAdd(cnt, 1ull);
        if (old + 1 < target) {
            const long long t0 = clock64();
            for (;;) {
                unsigned long long v;
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(cnt) : "memory");
                if (v >= target) break;
                if (clock64() - t0 > spin_cycles) {
                    atomicOr(err, 4);
                    break;
                }
            }
        }
        __threadfence();
    }
    named_bar_sync(2, ncw * 32);
    return *((volatile int*)err) == 0;
}

// Fixed-order block sum over the compute warps of K doubles per thread; the
// result is in red[0..K) for every compute thread.  wsum: [ncw][K] doubles.
template <int K>
__device__ __forceinline__ void compute_block_sum(const double* v, double* wsum, double* red, int ncw) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = v[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) wsum[w * K + k] = s;
    }
    named_bar_sync(1, ncw * 32);
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int ww = 0; ww < ncw; ++ww) s += wsum[ww * K + threadIdx.x];
        red[threadIdx.x] = s;
    }
    named_bar_sync(1, ncw * 32);
}

// Fixed-order sum over blocks of partials[b * stride + off + k], k < K, into
// out[k] (shared), computed by the compute warps (warp k sums term k).
template <int K>
__device__ __forceinline__ void compute_grid_sum(const double* partials, int nblocks, int stride, int off,
                                                 double* out, int ncw) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < K; k += ncw) {
        double s = lane_partial_sum(partials, nblocks, stride, off + k, lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[k] = s;
    }
    named_bar_sync(1, ncw * 32);
}

// Fixed-order sums over blocks of three terms at offsets o0, o1, o2 into out[0..2]
// (term k summed by compute warp k mod ncw; with three or more compute warps one
// L2 round trip for all three).
__device__ __forceinline__ void compute_grid_sum3(const double* partials, int nblocks, int stride, int o0, int o1,
                                                  int o2, double* out, int ncw) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < 3; k += ncw) {
        const int off = k == 0 ? o0 : (k == 1 ? o1 : o2);
        double s = lane_partial_sum(partials, nblocks, stride, off, lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[k] = s;
    }
    named_bar_sync(1, ncw * 32);
}

// CG vector accesses with an L2 evict-last policy: the vectors of a solve (about
// 32 B per row) stay in L2 while the fields stream through it evict-first.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float ldv(const float* p, uint64_t pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ldv(const double* p, uint64_t pol) {
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void stv(float* p, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void stv(double* p, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}

// Shared scratch of the brick PCG, placed in the first kBrickPcgHeader bytes of
// the dynamic shared memory (the stage ring starts after it).
struct BrickPcgShared {
    uint64_t full[4], empty[4];
    int done;              // set when the compute warps leave: the producer stops
    int active, iters;
    double gam, rr, bnorm, alpha, beta;
    double red[4], red2[4];
    double wsum[32 * 3];
};
constexpr int kBrickPcgHeader = 2048;
static_assert(sizeof(BrickPcgShared) <= kBrickPcgHeader, "brick PCG header");

// Producer with a stop flag: streams the nF field boxes pass after pass until
// *done is set (the waits for a free stage give up when it is); then waits for
// the boxes still in flight.
template <int P, int NS>
__device__ __forceinline__ void brick_produce_until_done(const BrickMaps& maps, const BrickGeo& g, float* stages,
                                                         int stage_floats, uint64_t* full, uint64_t* empty, int nF,
                                                         volatile int* done, int* err) {
    const CUtensorMap* tm = &maps.tm[g.cls];
    const unsigned bytes = (unsigned)(g.bxb * g.byb * g.bzb) * 4u;
    const uint64_t policy = l2_evict_first_policy();
    unsigned long long k = 0;
    bool ok = true;
    for (;; ++k) {
        const int s = (int)(k % NS);
        const unsigned long long use = k / NS;
        if (use > 0) {
            const unsigned par = (unsigned)((use - 1) & 1);
            bool got = mbar_try_wait(&empty[s], par);
            const unsigned long long t0 = got ? 0ull : global_ns();
            while (!got && !*done) {
                got = mbar_try_wait(&empty[s], par);
                if (!got && global_ns() - t0 > kBrickWaitNs) {
                    ok = false;
                    break;
                }
            }
            if (!got) break;
        }
        if (*done) break;
        mbar_arrive_expect_tx(&full[s], bytes);
        tma_load_4d(stages + (size_t)s * stage_floats, tm, g.x0, g.y0 - P, g.z0 - P, (int)(k % nF), &full[s], policy);
    }
    if (!ok) atomicOr(err, 16);
    brick_drain<NS>(full, k);
}

template <int P, int NS>
__global__ void __launch_bounds__(1024, 1)
    pcg_brick_kernel(const __grid_constant__ BrickMaps maps, const BrickDesc* __restrict__ bricks, int nF,
                     int stage_floats, CgVecs<float> v, CgCtl c) {
    constexpr int BZM = 12;
    constexpr int S = kCgStride<1>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BrickPcgShared& sh = *reinterpret_cast<BrickPcgShared*>(smem_raw);
    float* stages = (float*)(smem_raw + kBrickPcgHeader);
    float* xt = stages + (size_t)NS * stage_floats;
    const int ncw = (int)(blockDim.x >> 5) - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], ncw);
        }
        sh.done = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const BrickDesc bd = bricks[blockIdx.x];
    if (warp == ncw) {
        if (lane == 0) {
            const BrickGeo g = brick_geo(maps, bd, 0, 0);
            brick_produce_until_done<P, NS>(maps, g, stages, stage_floats, sh.full, sh.empty, nF, &sh.done, c.err);
        }
        return;
    }
    const BrickGeo g = brick_geo(maps, bd, warp, lane);
    const int m = v.m;
    const long long mm = (long long)m * m;
    const long long colbase = (long long)g.z0 * mm + (long long)(g.y0 + g.cy) * m + g.x0 + g.cx;
    unsigned long long fc = 0, epoch = 0;
    float acc[BZM], xo[BZM];
    double part[3];
    bool ok = true;
    auto stop = [&]() {
        if (threadIdx.x == 0) {
            sh.done = 1;
            __threadfence_block();
        }
        cg_report(c);
    };

    // ---- init 1: r = b - M~x, u = D^-1 r; partials (r,u), (r,r), (b,b)
    {
        brick_load_tile<P, true>(xt, v.x, g, m, warp, ncw, lane);
        ok = brick_pass<P, true, true, BZM, NS>(g, stages, stage_floats, xt, sh.full, sh.empty, fc, lane, acc, xo);
        fc += nF;
        DotAcc<float> d0, d1, d2;
        if (g.lane_ok) {
#pragma unroll
            for (int zl = 0; zl < BZM; ++zl) {
                if (zl >= g.nz) break;
                const long long j = colbase + zl * mm;
                const float bi = v.b[j];
                const double ri = (double)bi - (double)acc[zl];   // FP64 residual
                const float rt = (float)ri;
                const float ui = v.dinv[j] * rt;
                v.r[j] = ri;
                v.u[j] = ui;
                d0.add(rt, ui);
                d1.add(rt, rt);
                d2.add(bi, bi);
            }
        }
        part[0] = d0.value();
        part[1] = d1.value();
        part[2] = d2.value();
        compute_block_sum<3>(part, sh.wsum, sh.red, ncw);
        if (threadIdx.x < 3) c.partials[(size_t)blockIdx.x * S + 6 + threadIdx.x] = sh.red[threadIdx.x];
    }
    if (!ok) atomicOr(c.err, 16);
    if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch)) return stop();
    // ---- init 2: w = M~u; partial (w,u)
    {
        brick_load_tile<P, true>(xt, v.u, g, m, warp, ncw, lane);
        ok = brick_pass<P, true, true, BZM, NS>(g, stages, stage_floats, xt, sh.full, sh.empty, fc, lane, acc, xo);
        fc += nF;
        DotAcc<float> d0;
        if (g.lane_ok) {
#pragma unroll
            for (int zl = 0; zl < BZM; ++zl) {
                if (zl >= g.nz) break;
                v.w[colbase + zl * mm] = acc[zl];
                d0.add(xo[zl], acc[zl]);
            }
        }
        part[0] = d0.value();
        compute_block_sum<1>(part, sh.wsum, sh.red, ncw);
        if (threadIdx.x == 0) c.partials[(size_t)blockIdx.x * S + 4] = sh.red[0];
    }
    if (!ok) atomicOr(c.err, 16);
    if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch)) return stop();
    compute_grid_sum<3>(c.partials, gridDim.x, S, 6, sh.red, ncw);
    compute_grid_sum<1>(c.partials, gridDim.x, S, 4, sh.red2, ncw);
    if (threadIdx.x == 0) {
        sh.gam = sh.red[0];
        sh.rr = sh.red[1];
        sh.bnorm = sqrt(sh.red[2]);
        sh.beta = 0.0;
        sh.iters = 0;
        int act = sh.bnorm > 0.0 && !(c.rtol > 0.0 && sqrt(sh.rr) <= c.rtol * sh.bnorm);
        const double d = sh.red2[0];
        if (act && (!(d > 0.0) || !isfinite(d))) {
            act = 0;
            atomicOr(c.err, 1);
        }
        sh.alpha = act ? sh.gam / d : 0.0;
        sh.active = act;
    }
    named_bar_sync(1, ncw * 32);
    // a zero right-hand side has the solution 0
    if (!(sh.bnorm > 0.0) && g.lane_ok)
        for (int zl = 0; zl < g.nz; ++zl) v.x[colbase + zl * mm] = 0.f;

    for (int it = 0; it < c.max_it && sh.active; ++it) {
        const int off1 = (it & 1) * 2;
        // ---- phase 1 (own rows), x-runs of the brick for coalesced access
        {
            const float be = (float)sh.beta, al = (float)sh.alpha;
            const double ald = sh.alpha;
            const uint64_t pol = l2_evict_last_policy();
            DotAcc<float> d0, d1;
            const int nch = (g.nx + 31) / 32;   // 32-column chunks of an x-run
            const int nitems = g.ny * g.nz * nch;
            for (int item = warp; item < nitems; item += ncw) {
                const int line = item / nch, xl = (item - line * nch) * 32 + lane;
                if (xl >= g.nx) continue;
                const int yl = line % g.ny, zl = line / g.ny;
                const long long o = (long long)(g.z0 + zl) * mm + (long long)(g.y0 + yl) * m + g.x0 + xl;
                const float di = ldv(v.dinv + o, pol);
                const float pi = ldv(v.u + o, pol) + be * ldv(v.p + o, pol);
                const float si = ldv(v.w + o, pol) + be * ldv(v.s + o, pol);
                const float xi = ldv(v.x + o, pol);
                const double rv = ldv(v.r + o, pol);
                stv(v.p + o, pi, pol);
                stv(v.s + o, si, pol);
                stv(v.x + o, xi + al * pi, pol);
                const double ri = rv - ald * (double)si;   // FP64 residual
                const float rt = (float)ri;
                const float ui = di * rt;
                stv(v.r + o, ri, pol);
                stv(v.u + o, ui, pol);
                d0.add(rt, ui);
                d1.add(rt, rt);
            }
            part[0] = d0.value();
            part[1] = d1.value();
        }
        compute_block_sum<2>(part, sh.wsum, sh.red, ncw);
        if (threadIdx.x < 2) c.partials[(size_t)blockIdx.x * S + off1 + threadIdx.x] = sh.red[threadIdx.x];
        if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch)) return stop();
        // ---- phase 2: w = M~u; partial (w,u)
        {
            brick_load_tile<P, true>(xt, v.u, g, m, warp, ncw, lane);
            ok = brick_pass<P, true, true, BZM, NS>(g, stages, stage_floats, xt, sh.full, sh.empty, fc, lane, acc,
                                                    xo);
            fc += nF;
            DotAcc<float> d0;
            if (g.lane_ok) {
                const uint64_t pol = l2_evict_last_policy();
#pragma unroll
                for (int zl = 0; zl < BZM; ++zl) {
                    if (zl >= g.nz) break;
                    stv(v.w + colbase + zl * mm, acc[zl], pol);
                    d0.add(xo[zl], acc[zl]);
                }
            }
            part[0] = d0.value();
            compute_block_sum<1>(part, sh.wsum, sh.red, ncw);
            if (threadIdx.x == 0) c.partials[(size_t)blockIdx.x * S + 4] = sh.red[0];
        }
        if (!ok) {
            atomicOr(c.err, 16);
            return stop();
        }
        if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch)) return stop();
        compute_grid_sum3(c.partials, gridDim.x, S, off1, off1 + 1, 4, sh.red, ncw);
        if (threadIdx.x == 0) {
            int brk = 0, act = 1, iters = sh.iters;
            double rro = sh.rr, gam = sh.gam, alpha = sh.alpha, beta = sh.beta;
            cg_scalars(sh.red[0], sh.red[1], sh.red[2], c.rtol, sh.bnorm, gam, alpha, beta, act, iters, rro, &brk);
            sh.gam = gam;
            sh.alpha = alpha;
            sh.beta = beta;
            sh.iters = iters;
            sh.rr = rro;
            sh.active = act;
            if (brk && blockIdx.x == 0) atomicOr(c.err, 1);
        }
        named_bar_sync(1, ncw * 32);
    }
    stop();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rel = sh.bnorm > 0.0 ? sqrt(sh.rr) / sh.bnorm : 0.0;
        c.iters_out[0] = sh.iters;
        c.relres_out[0] = rel;
        if (c.iter_acc) atomicAdd((unsigned long long*)c.iter_acc, (unsigned long long)sh.iters);
        if (c.status_acc && c.rtol > 0.0 && rel > c.rtol) atomicOr(c.status_acc, 8);
    }
}

}  // namespace iga
