// Brick form of the persistent Jacobi-PCG (FP32 dtype, one right-hand side, 3-D
// operators with a brick form).  Same recurrence, precision and stopping rule as
// pcg_persistent_kernel (Chronopoulos-Gear form; compensated FP32 dot products
// widened to FP64, fixed-order reductions), with the residual carried as a pair of
// FP32 numbers instead of one FP64 number, and the rows owned by bricks instead
// of a grid-stride loop:
//   * one CTA per brick (and per SM) for the whole solve (cooperative launch, one
//     wave); every compute lane owns one (x, y) column of its brick, the same in
//     every phase;
//   * the brick's own p, s, x, w = M~u, D^-1 and the residual pair live in the CTA's
//     tensor memory (TMEM, tcgen05.alloc / ld / st) for the whole solve, and u of
//     the brick's rows is still in the shared-memory tile of the last M~ pass, so
//     the vector update reads nothing from global memory and writes only u (which
//     the neighbouring bricks read) into a padded copy; x is written back once at
//     the end;
//   * phase 2 loads the u tile of the brick grown by p from the padded copy as one
//     TMA box (u was written by the neighbouring CTAs in phase 1), applies M~ with
//     the brick kernels of brick.cuh and forms the partial of (w,u);
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
// The error word is read once per CTA (by thread 0, into *verdict), so every
// compute warp of the CTA takes the same branch afterwards.
__device__ __forceinline__ bool compute_grid_barrier(unsigned* bar, int* err, unsigned nblocks, int ncw,
                                                     long long spin_cycles, unsigned long long& epoch,
                                                     volatile int* verdict) {
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
        *verdict = *((volatile int*)err);
    }
    named_bar_sync(2, ncw * 32);
    return *verdict == 0;
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

// ---- tensor memory of the CTA as storage for the brick's CG vectors.  With
// the 32x32b shape, thread t of a warp accesses TMEM lane 32 * (warp % 4) + t,
// one 32-bit column per .x1 access; the allocating warp writes the base address
// into shared memory.  The loaded registers pass through the wait, so that no
// use of them can be scheduled before it.
constexpr unsigned kTmemCols = 512;   // the whole TMEM of the SM (one CTA per SM)
constexpr int kTmemWords = 7;         // p, s, x, w, D^-1, r (high part), r (low part)
__device__ __forceinline__ void tmem_alloc(unsigned* dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ unsigned tmem_ld(unsigned taddr) {
    unsigned v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr) : "memory");
    return v;
}
__device__ __forceinline__ void tmem_st(unsigned taddr, unsigned v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(unsigned& a, unsigned& b, unsigned& c, unsigned& d, unsigned& e,
                                             unsigned& f, unsigned& g) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a), "+r"(b), "+r"(c), "+r"(d), "+r"(e), "+r"(f), "+r"(g)
                 :
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(unsigned& a) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(a) : : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared scratch of the brick PCG, placed in the first kBrickPcgHeader bytes of
// the dynamic shared memory (the stage ring starts after it).
struct BrickPcgShared {
    uint64_t full[4], empty[4];
    uint64_t tile_full;    // the u tile's TMA box has landed
    unsigned tmem;         // TMEM base address (written by tcgen05.alloc)
    int verdict;           // error word as read after the last grid barrier
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

// TMEM columns for a brick of nx x ny x nz rows: its warps (one per 4 x 8 lane
// patch) that share a lane quarter take consecutive slots of kTmemWords * nz
// columns (word k of plane zl at column slot + k * nz + zl); warps without rows
// hold none.
__host__ __device__ constexpr int brick_pcg_tmem_cols(int nx, int ny, int nz) {
    return ((nx + 3) / 4 * ((ny + 7) / 8) + 3) / 4 * kTmemWords * nz;
}

// The residual of the brick PCG as an unevaluated pair hi + lo of FP32 numbers
// (about 48 significant bits; the FP64 pipe of this part issues about 60 times
// more slowly than the FP32 one).  ff_two_sum: Knuth's TwoSum, a + b = s + e
// exactly.  ff_sub_prod: (hi, lo) -= (ahi + alo) s, with ahi s split exactly by
// an FMA (Dekker / Kahan TwoProd), alo s rounded once, then renormalised.
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_sub_prod(float& hi, float& lo, float ahi, float alo, float s) {
    const float p = __fmul_rn(ahi, s);
    const float e = fmaf(ahi, s, -p);          // ahi s = p + e exactly
    const float t = fmaf(alo, s, e);           // the part below p
    float h, err;
    ff_two_sum(hi, -p, h, err);
    const float l = __fsub_rn(__fadd_rn(lo, err), t);
    hi = __fadd_rn(h, l);
    lo = __fsub_rn(l, __fsub_rn(hi, h));
}

// End of an M~ pass: w = acc of the lane's rows into TMEM word 3; returns the
// lane's partial of (w, u) (u = xo, the tile values of the same rows).
template <int BZM>
__device__ __forceinline__ double brick_pcg_keep_w(const float (&acc)[BZM], const float (&xo)[BZM],
                                                   const BrickGeo& g, unsigned tw, int nzs) {
    DotAcc<float> d0;
#pragma unroll
    for (int zl = 0; zl < BZM; ++zl) {
        if (zl >= g.nz || !g.warp_ok) break;   // uniform over the warp
        __syncwarp();
        tmem_st(tw + (unsigned)(3 * nzs + zl), __float_as_uint(acc[zl]));
        if (g.lane_ok) d0.add(xo[zl], acc[zl]);
    }
    tmem_wait_st();
    return d0.value();
}

// Requirements checked by the host before the launch: one CTA per SM (the
// launch asks for enough shared memory that a second CTA cannot fit, so the
// allocation of the whole TMEM never waits) and brick_pcg_tmem_cols(nx, ny, nz)
// <= kTmemCols for every brick.
template <int P, int NS>
__global__ void __launch_bounds__(1024, 1)
    pcg_brick_kernel(const __grid_constant__ BrickMaps maps, const __grid_constant__ BrickMaps umaps,
                     const BrickDesc* __restrict__ bricks, int nF, int stage_floats, float* __restrict__ upad, int XP,
                     CgVecs<float> v, CgCtl c) {
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
        mbar_init(&sh.tile_full, 1);
        sh.done = 0;
        sh.verdict = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(&sh.tmem, kTmemCols);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
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
    // this lane's TMEM words (lane quarter of the warp, column slot of its group)
    const unsigned tw = sh.tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)((warp >> 2) * kTmemWords * g.nz);
    const int nzs = g.nz;
    auto tcol = [&](int k, int zl) { return tw + (unsigned)(k * nzs + zl); };
    unsigned long long fc = 0, epoch = 0;
    float acc[BZM], xo[BZM];
    double part[3];
    bool ok = true;
    // every compute warp of the CTA leaves through here, together (the barrier
    // verdicts are CTA-uniform): TMEM is freed by the warp that allocated it
    auto leave = [&]() {
        tmem_wait_st();
        tmem_fence_before();
        named_bar_sync(1, ncw * 32);
        tmem_fence_after();
        if (warp == 0) tmem_dealloc(sh.tmem, kTmemCols);
        if (threadIdx.x == 0) {
            sh.done = 1;
            __threadfence_block();
        }
        cg_report(c);
    };

    // u of the lane's row zl in the padded copy
    float* const ucol = upad + ((long long)g.z0 * m + g.y0 + g.cy) * XP + g.x0 + g.cx + P;
    const long long uplane = (long long)m * XP;
    // u tile of the brick grown by P (zero outside the grid) as one TMA box.  Called
    // right after a grid barrier: every read of xt in this CTA and every u store of
    // the grid are done; the proxy fence orders them before the async-proxy copy.
    unsigned tile_par = 0;
    auto load_u_tile = [&]() {
        if (threadIdx.x == 0) {
            fence_proxy_async();
            mbar_arrive_expect_tx(&sh.tile_full, (unsigned)(umaps.bx[g.cls] * umaps.by[g.cls] * umaps.bz[g.cls]) * 4u);
            tma_load_3d(xt, &umaps.tm[g.cls], g.x0, g.y0 - P, g.z0 - P, &sh.tile_full);
        }
        if (!mbar_wait(&sh.tile_full, tile_par, kBrickWaitNs)) atomicOr(c.err, 16);
        tile_par ^= 1u;
    };

    // ---- init 1: r = b - M~x, u = D^-1 r; partials (r,u), (r,r), (b,b); TMEM
    // gets p = s = 0, x, D^-1 and r of the lane's rows
    {
        brick_load_tile<P, true>(xt, v.x, g, m, warp, ncw, lane);
        ok = brick_pass<P, true, true, BZM, NS>(g, stages, stage_floats, xt, sh.full, sh.empty, fc, lane, acc, xo);
        fc += nF;
        if (!ok) atomicOr(c.err, 16);
        DotAcc<float> d0, d1, d2;
#pragma unroll
        for (int zl = 0; zl < BZM; ++zl) {
            if (zl >= g.nz || !g.warp_ok) break;   // uniform over the warp
            __syncwarp();
            const long long j = colbase + zl * mm;
            const float bi = g.lane_ok ? v.b[j] : 0.f;
            const float di = g.lane_ok ? v.dinv[j] : 0.f;
            float rhi, rlo;   // r = b - M~x exactly, as an unevaluated pair
            ff_two_sum(bi, -acc[zl], rhi, rlo);
            const float rt = rhi;
            const float ui = di * rt;
            tmem_st(tcol(0, zl), 0u);
            tmem_st(tcol(1, zl), 0u);
            tmem_st(tcol(2, zl), __float_as_uint(xo[zl]));
            tmem_st(tcol(4, zl), __float_as_uint(di));
            tmem_st(tcol(5, zl), __float_as_uint(rhi));
            tmem_st(tcol(6, zl), __float_as_uint(rlo));
            if (g.lane_ok) {
                ucol[zl * uplane] = ui;
                d0.add(rt, ui);
                d1.add(rt, rt);
                d2.add(bi, bi);
            }
        }
        tmem_wait_st();
        part[0] = d0.value();
        part[1] = d1.value();
        part[2] = d2.value();
        compute_block_sum<3>(part, sh.wsum, sh.red, ncw);
        if (threadIdx.x < 3) c.partials[(size_t)blockIdx.x * S + 6 + threadIdx.x] = sh.red[threadIdx.x];
    }
    if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch, &sh.verdict)) return leave();
    // ---- init 2: w = M~u into TMEM; partial (w,u)
    {
        load_u_tile();
        ok = brick_pass<P, true, true, BZM, NS>(g, stages, stage_floats, xt, sh.full, sh.empty, fc, lane, acc, xo);
        fc += nF;
        if (!ok) atomicOr(c.err, 16);
        part[0] = brick_pcg_keep_w<BZM>(acc, xo, g, tw, nzs);

        compute_block_sum<1>(part, sh.wsum, sh.red, ncw);
        if (threadIdx.x == 0) c.partials[(size_t)blockIdx.x * S + 4] = sh.red[0];
    }
    if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch, &sh.verdict)) return leave();
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

    for (int it = 0; it < c.max_it && sh.active; ++it) {
        const int off1 = (it & 1) * 2;
        // ---- phase 1 (the lane's rows): p, s, x, w, D^-1, r from TMEM, u from the
        // tile of the last M~ pass; only u goes to global memory
        {
            const float be = (float)sh.beta, al = (float)sh.alpha;
            const float ahi = (float)sh.alpha, alo = (float)(sh.alpha - (double)ahi);   // alpha as a pair
            const uint64_t pol = l2_evict_last_policy();
            const int plane = g.byb * g.bxb, sb = (P * g.byb + g.cy + P) * g.bxb + g.cx + P;
            DotAcc<float> d0, d1;
#pragma unroll
            for (int zl = 0; zl < BZM; ++zl) {
                if (zl >= g.nz || !g.warp_ok) break;   // uniform over the warp
                __syncwarp();
                unsigned wp = tmem_ld(tcol(0, zl)), ws = tmem_ld(tcol(1, zl)), wx = tmem_ld(tcol(2, zl));
                unsigned ww = tmem_ld(tcol(3, zl)), wd = tmem_ld(tcol(4, zl)), whi = tmem_ld(tcol(5, zl));
                unsigned wlo = tmem_ld(tcol(6, zl));
                const float uo = g.lane_ok ? xt[sb + zl * plane] : 0.f;
                tmem_wait_ld(wp, ws, wx, ww, wd, whi, wlo);
                const float pi = uo + be * __uint_as_float(wp);
                const float si = __uint_as_float(ww) + be * __uint_as_float(ws);
                const float xi = __uint_as_float(wx) + al * pi;
                float rhi = __uint_as_float(whi), rlo = __uint_as_float(wlo);
                ff_sub_prod(rhi, rlo, ahi, alo, si);   // r -= alpha s in pair arithmetic
                const float rt = rhi;
                const float ui = __uint_as_float(wd) * rt;
                tmem_st(tcol(0, zl), __float_as_uint(pi));
                tmem_st(tcol(1, zl), __float_as_uint(si));
                tmem_st(tcol(2, zl), __float_as_uint(xi));
                tmem_st(tcol(5, zl), __float_as_uint(rhi));
                tmem_st(tcol(6, zl), __float_as_uint(rlo));
                if (g.lane_ok) {
                    stv(ucol + zl * uplane, ui, pol);
                    d0.add(rt, ui);
                    d1.add(rt, rt);
                }
            }
            tmem_wait_st();
            part[0] = d0.value();
            part[1] = d1.value();
        }
        compute_block_sum<2>(part, sh.wsum, sh.red, ncw);
        if (threadIdx.x < 2) c.partials[(size_t)blockIdx.x * S + off1 + threadIdx.x] = sh.red[threadIdx.x];
        if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch, &sh.verdict)) return leave();
        // ---- phase 2: w = M~u into TMEM; partial (w,u)
        {
            load_u_tile();
            ok = brick_pass<P, true, true, BZM, NS>(g, stages, stage_floats, xt, sh.full, sh.empty, fc, lane, acc,
                                                    xo);
            fc += nF;
            if (!ok) atomicOr(c.err, 16);
            part[0] = brick_pcg_keep_w<BZM>(acc, xo, g, tw, nzs);
            compute_block_sum<1>(part, sh.wsum, sh.red, ncw);
            if (threadIdx.x == 0) c.partials[(size_t)blockIdx.x * S + 4] = sh.red[0];
        }
        if (!compute_grid_barrier(c.bar, c.err, gridDim.x, ncw, c.spin_cycles, epoch, &sh.verdict)) return leave();
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
    // ---- x of the lane's rows back to global memory (a zero right-hand side has
    // the solution 0)
    {
        const bool zero = !(sh.bnorm > 0.0);
#pragma unroll
        for (int zl = 0; zl < BZM; ++zl) {
            if (zl >= g.nz || !g.warp_ok) break;   // uniform over the warp
            __syncwarp();
            unsigned wx = tmem_ld(tcol(2, zl));
            tmem_wait_ld(wx);
            if (g.lane_ok) v.x[colbase + zl * mm] = zero ? 0.f : __uint_as_float(wx);
        }
    }
    leave();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rel = sh.bnorm > 0.0 ? sqrt(sh.rr) / sh.bnorm : 0.0;
        c.iters_out[0] = sh.iters;
        c.relres_out[0] = rel;
        if (c.iter_acc) atomicAdd((unsigned long long*)c.iter_acc, (unsigned long long)sh.iters);
        if (c.status_acc && c.rtol > 0.0 && rel > c.rtol) atomicOr(c.status_acc, 8);
    }
}

}  // namespace iga
