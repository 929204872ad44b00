// Brick form of the 3-D FP32 surrogate stencil operators (c1, and the mass
// apply inside the persistent PCG).
//
// The grid of rows is cut into bricks (x0 + [0, nx)) x (y0 + [0, ny)) x (z0 + [0, nz))
// of about one SM's share of the rows each.  A CTA owns one brick.  Its fields
// stream through a ring of shared-memory stages filled by TMA (one 4-D tensor-map
// box per field: the brick grown by P on every side except +z, so that both the
// row's own entry F_u[i] and the mirrored entry F_u[i - delta] come from the same
// box); its vector values come from a shared-memory tile of the brick grown by P
// on every side.  Every value a row reads is therefore a shared-memory load, and
// every byte moved from L2 / HBM is moved by the TMA unit, so the number of bytes
// in flight is set by the ring depth and not by registers.
//
// Rows are computed by warps of 4 (x) x 8 (y) columns, each lane marching through
// the brick's nz rows of its column with the results in registers.  A box row of
// the stage is BXB floats with BXB / 4 odd, so the 32 lanes of a warp always read
// 32 different banks (own and mirrored reads alike).
//
// Field order of the padded copy (grouped by (d1, d2), then d3 ascending): the
// vector values x[c + (d1, d2), z + d3] and x[c - (d1, d2), z - d3] of a whole
// group can be read into registers once and reused by the group's fields.  For
// the mass operator the diagonal is field 0 of the copy.
#pragma once

#include <cuda.h>
#include <cstdint>
#include <utility>

#include "iga_internal.cuh"

namespace iga {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// One tiled 4-D TMA box into shared memory, completion counted on bar.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
// One tiled 3-D TMA box into shared memory, completion counted on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
// Orders this thread's generic-proxy accesses (and those it has acquired from
// other threads) before its later async-proxy (TMA) accesses, and back.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

constexpr unsigned long long kBrickWaitNs = 2000000000ull;   // 2 s per wait, then IGA_ERR_TIMEOUT

// ---------------------------------------------------------------- field groups
struct BrickField {
    int d1, d2, d3;   // offset delta of the field (upper half: colex index above the centre)
    int u;            // index of the field in the colex SoA field set (K~ numbering)
    int first;        // 1 if the field opens its (d1, d2) group
};

template <int P>
struct BrickTable {
    static constexpr int PP = 2 * P + 1;
    static constexpr int NF = (PP * PP * PP - 1) / 2;
    BrickField f[NF];
};

// The upper-half offsets of the 3-D stencil of degree P grouped by (d1, d2)
// (colex), d3 ascending inside a group.
template <int P>
constexpr BrickTable<P> make_brick_table() {
    BrickTable<P> t{};
    constexpr int PP = 2 * P + 1, T0 = (PP * PP * PP - 1) / 2;
    int k = 0;
    for (int d2 = -P; d2 <= P; ++d2)
        for (int d1 = -P; d1 <= P; ++d1) {
            bool first = true;
            for (int d3 = 0; d3 <= P; ++d3) {
                const int tt = (d1 + P) + PP * (d2 + P) + PP * PP * (d3 + P);
                if (tt <= T0) continue;   // not in the upper half
                t.f[k].d1 = d1;
                t.f[k].d2 = d2;
                t.f[k].d3 = d3;
                t.f[k].u = tt - T0 - 1;
                t.f[k].first = first ? 1 : 0;
                first = false;
                ++k;
            }
        }
    return t;
}

// ---------------------------------------------------------------- per-brick geometry
struct BrickGeo {
    int x0, y0, z0, nx, ny, nz, cls;
    int bxb, byb, bzb;   // box of this brick's class
    int cx, cy;          // this lane's column inside the brick
    bool lane_ok;        // the column is a row column of the grid
    bool warp_ok;        // the warp's patch intersects the brick
};

__device__ __forceinline__ BrickGeo brick_geo(const BrickMaps& maps, const BrickDesc& b, int warp, int lane) {
    BrickGeo g;
    g.x0 = b.x0;
    g.y0 = b.y0;
    g.z0 = b.z0;
    g.nx = b.nx;
    g.ny = b.ny;
    g.nz = b.nz;
    g.cls = b.cls;
    g.bxb = maps.bx[b.cls];
    g.byb = maps.by[b.cls];
    g.bzb = maps.bz[b.cls];
    const int gx = (b.nx + 3) / 4, gy = (b.ny + 7) / 8;
    g.warp_ok = warp < gx * gy;
    const int px = warp % gx, py = warp / gx;
    g.cx = px * 4 + (lane & 3);
    g.cy = py * 8 + (lane >> 2);
    g.lane_ok = g.warp_ok && g.cx < b.nx && g.cy < b.ny;
    return g;
}

// Vector tile of the brick grown by P on every side ([z][y][x], row pitch bxb,
// plane byb * bxb), zero outside the grid.  Called by the consumer warps only;
// ends with their named barrier.  Each warp loads U tile rows of a 32-column
// chunk (one value per lane and row) before it stores any, so a tile costs about
// rows / (U * ncw) L2 round trips per chunk.  COHERENT: plain loads (vectors
// written earlier in the same persistent launch), else read-only loads.
template <int P, bool COHERENT, int U = 8>
__device__ __forceinline__ void brick_load_tile(float* xt, const float* x, const BrickGeo& g, int m, int cwarp,
                                                int ncw, int lane) {
    const int zt = g.nz + 2 * P, rows = g.byb * zt;
    const long long mm = (long long)m * m;
    for (int xc = 0; xc < g.bxb; xc += 32)
    for (int r0 = cwarp; r0 < rows; r0 += U * ncw) {
        const int ia = xc + lane;
        const int xa = g.x0 - P + ia;
        const bool oka = ia < g.bxb && xa >= 0 && xa < m;
        float va[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = r0 + u * ncw;
            va[u] = 0.f;
            if (r < rows) {
                const int yy = g.y0 - P + r % g.byb, zz = g.z0 - P + r / g.byb;
                if (oka && yy >= 0 && yy < m && zz >= 0 && zz < m) {
                    const float* src = x + zz * mm + (long long)yy * m + xa;
                    va[u] = COHERENT ? *src : __ldg(src);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = r0 + u * ncw;
            if (r < rows && ia < g.bxb) xt[(size_t)r * g.bxb + ia] = va[u];
        }
    }
    named_bar_sync(1, ncw * 32);
}

// Producer (one thread): issues the nF field boxes of one pass over a brick into
// the stage ring.  fc = stages this CTA has issued before the pass (the ring is
// continued across passes).  Returns false if a wait for a free stage timed out.
template <int P, int NS>
__device__ __forceinline__ bool brick_produce(const BrickMaps& maps, const BrickGeo& g, float* stages,
                                              int stage_floats, uint64_t* full, uint64_t* empty, int nF,
                                              unsigned long long fc, uint64_t policy) {
    const CUtensorMap* tm = &maps.tm[g.cls];
    const unsigned bytes = (unsigned)(g.bxb * g.byb * g.bzb) * 4u;
    for (int f = 0; f < nF; ++f) {
        const unsigned long long k = fc + f;
        const int s = (int)(k % NS);
        const unsigned long long use = k / NS;
        if (use > 0 && !mbar_wait(&empty[s], (unsigned)((use - 1) & 1), kBrickWaitNs)) return false;
        mbar_arrive_expect_tx(&full[s], bytes);
        tma_load_4d(stages + (size_t)s * stage_floats, tm, g.x0, g.y0 - P, g.z0 - P, f, &full[s], policy);
    }
    return true;
}

// Bounded wait for the boxes still in flight after the producer's last pass (the
// last min(NS, issued) stages), so that no copy lands after the CTA has exited.
template <int NS>
__device__ __forceinline__ void brick_drain(uint64_t* full, unsigned long long issued) {
    const unsigned long long lo = issued > (unsigned long long)NS ? issued - NS : 0ull;
    for (unsigned long long k = lo; k < issued; ++k)
        (void)mbar_wait(&full[k % NS], (unsigned)((k / NS) & 1), kBrickWaitNs);
}

// ---------------------------------------------------------------- consumer
// State of one consumer lane during a pass over its brick.
template <int P, int BZM>
struct BrickLane {
    const float* stages;
    const float* xt;
    uint64_t* full;
    uint64_t* empty;
    int stage_floats, plane, bxb, sb, nz, lane;
    bool lane_ok;
    unsigned long long k;   // running stage counter of the CTA
    bool ok;                // false once a wait has timed out (no further waits)
};

// Waits for the next stage; returns its base (already offset to this lane's
// own row at zl = 0) or nullptr when the lane has nothing to read.
template <int P, int BZM, int NS>
__device__ __forceinline__ const float* brick_stage_acquire(BrickLane<P, BZM>& c, int& s) {
    s = (int)(c.k % NS);
    if (c.ok && !mbar_wait(&c.full[s], (unsigned)((c.k / NS) & 1), kBrickWaitNs)) c.ok = false;
    return (c.ok && c.lane_ok) ? c.stages + (size_t)s * c.stage_floats + c.sb : nullptr;
}
template <int P, int BZM>
__device__ __forceinline__ void brick_stage_release(BrickLane<P, BZM>& c, int s) {
    __syncwarp();
    if (c.lane == 0) mbar_arrive(&c.empty[s]);
    c.k += 1;
}

// Field (d1, d2, D3) applied to the lane's column.  D3 is a compile-time
// constant (register indices of the group's vector values); d1, d2 are not, so
// the body is one group's worth of code (the instruction cache holds it).
template <int P, bool MASS, bool XREG, int BZM, int NS, int D3>
__device__ __forceinline__ void brick_field(BrickLane<P, BZM>& c, int d1, int d2, float (&acc)[BZM],
                                            const float (&xo)[BZM], const float (&xf)[BZM + P],
                                            const float (&xm)[BZM + P]) {
    int s;
    const float* st = brick_stage_acquire<P, BZM, NS>(c, s);
    if (st) {
        const int moff = D3 * c.plane + d2 * c.bxb + d1;   // F_u[i - delta] relative to F_u[i]
        // the plane step is made opaque so that the compiler marches the
        // pointers instead of keeping every row's address live
        int step = c.plane;
        asm volatile("" : "+r"(step));
        const float* ps = st;
        const float* px = c.xt + c.sb;
#pragma unroll
        for (int zl = 0; zl < BZM; ++zl) {
            if (zl >= c.nz) break;   // uniform over the CTA
            const float so = ps[0], sm = ps[-moff];
            float xp, xq;
            if constexpr (XREG) {
                xp = xf[zl + D3];
                xq = xm[zl + P - D3];
            } else {
                xp = px[moff];
                xq = px[-moff];
                px += step;
            }
            if (MASS) {
                acc[zl] = fmaf(so, xp, acc[zl]);
                acc[zl] = fmaf(sm, xq, acc[zl]);
            } else {
                acc[zl] = fmaf(so, xp - xo[zl], acc[zl]);
                acc[zl] = fmaf(sm, xq - xo[zl], acc[zl]);
            }
            ps += step;
        }
    }
    brick_stage_release<P, BZM>(c, s);
}

// One pass of the operator over the lane's column: acc[zl] = (A x)(c, z0 + zl)
// for zl < nz, xo[zl] = x(c, z0 + zl).  The vector tile must be loaded.  The
// fields come in the grouped order of make_brick_table: groups (d1, d2) in colex
// order, d3 ascending, d3 = 0 only in the upper half.  Returns false if a stage
// wait timed out (the results are then meaningless).
template <int P, bool MASS, bool XREG, int BZM, int NS>
__device__ __forceinline__ bool brick_pass(const BrickGeo& g, const float* stages, int stage_floats, const float* xt,
                                           uint64_t* full, uint64_t* empty, unsigned long long fc, int lane,
                                           float (&acc)[BZM], float (&xo)[BZM]) {
    constexpr int PP = 2 * P + 1;
    BrickLane<P, BZM> c;
    c.stages = stages;
    c.xt = xt;
    c.full = full;
    c.empty = empty;
    c.stage_floats = stage_floats;
    c.plane = g.byb * g.bxb;
    c.bxb = g.bxb;
    c.sb = (P * g.byb + g.cy + P) * g.bxb + g.cx + P;
    c.nz = g.nz;
    c.lane = lane;
    c.lane_ok = g.lane_ok;
    c.k = fc;
    c.ok = true;
#pragma unroll
    for (int zl = 0; zl < BZM; ++zl) {
        xo[zl] = (c.lane_ok && zl < c.nz) ? xt[c.sb + zl * c.plane] : 0.f;
        acc[zl] = 0.f;
    }
    if (MASS) {
        int s;
        const float* st = brick_stage_acquire<P, BZM, NS>(c, s);
        if (st) {
#pragma unroll
            for (int zl = 0; zl < BZM; ++zl)
                if (zl < c.nz) acc[zl] = st[zl * c.plane] * xo[zl];
        }
        brick_stage_release<P, BZM>(c, s);
    }
    float xf[BZM + P], xm[BZM + P];
#pragma unroll 1
    for (int gi = 0; gi < PP * PP; ++gi) {
        const int d1 = gi % PP - P, d2 = gi / PP - P;
        const bool has0 = d2 > 0 || (d2 == 0 && d1 > 0);
        if constexpr (XREG) {
            if (c.lane_ok) {
                // xf[j] = x(c + (d1, d2), z0 + j), xm[j] = x(c - (d1, d2), z0 - P + j)
                const float* pf = c.xt + c.sb + d2 * c.bxb + d1;
                const float* pm = c.xt + c.sb - P * c.plane - d2 * c.bxb - d1;
#pragma unroll
                for (int j = 0; j < BZM + P; ++j) {
                    if (j >= c.nz + P) break;
                    xf[j] = pf[j * c.plane];
                    xm[j] = pm[j * c.plane];
                }
            }
        }
        if (has0) brick_field<P, MASS, XREG, BZM, NS, 0>(c, d1, d2, acc, xo, xf, xm);
        brick_field<P, MASS, XREG, BZM, NS, 1>(c, d1, d2, acc, xo, xf, xm);
        if constexpr (P >= 2) brick_field<P, MASS, XREG, BZM, NS, 2>(c, d1, d2, acc, xo, xf, xm);
    }
    return c.ok;
}

}  // namespace iga
