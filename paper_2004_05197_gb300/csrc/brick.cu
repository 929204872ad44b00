// Brick form of the 3-D FP32 surrogate operators: brick plan (host), padded
// group-ordered copy of the FP32 fields, TMA tensor maps, and the stand-alone
// brick apply kernel (c1: matrix-free use of the stored stencil data, Sec. 3.3;
// K~ in the difference form of Eq. DefinitionOfSurrogateMatrixSymmetricKernel).
//
// Padded copy: field f, row (i1, i2, i3) at f * fsz + (i3 m + i2) XP + i1 + P with
// XP = 4 ceil((m + 2P) / 4) (columns outside [P, m + P) are zero), fields in the
// grouped order of make_brick_table (mass: the diagonal first).  It is a second
// copy next to the colex fields (about 1.06x their size): every other consumer
// keeps reading the colex SoA layout of the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cudaTypedefs.h>

#include "brick.cuh"
#include "iga_internal.cuh"

namespace iga {

// ---------------------------------------------------------------- planner
namespace {

// total split into parts that differ by at most one, the larger ones last (the
// last piece of a direction is the one the grid edge clips).
std::vector<int> split_even(int total, int parts) {
    std::vector<int> s(parts, total / parts);
    for (int k = 0; k < total % parts; ++k) s[parts - 1 - k] += 1;
    return s;
}

// Box width: the warps' columns plus the halo, a multiple of 4 floats (TMA rows
// are 16-byte multiples) with an odd number of 16-byte chunks (conflict-free
// 4 x 8 warp patches).
int box_x(int nx, int P) {
    int b = (nx + 3) / 4 * 4 + 2 * P;
    b = (b + 3) / 4 * 4;
    if (((b / 4) & 1) == 0) b += 4;
    return b;
}

struct Column {
    int x0, nx, y0, ny, bxb, byb, warps;
};

struct PlanResult {
    double cost = 1e300;
    std::vector<BrickDesc> bricks;
    int ncls = 0, bx[kBrickMaxCls], by[kBrickMaxCls], bz[kBrickMaxCls];
    int stage_floats = 0, xt_floats = 0, ns = 0, ncw = 0;
};

// Estimated time of one brick (clocks of one SM): its shared-memory bytes at 128 B
// per clock, its TMA box bytes at its share of the L2 bandwidth (taken as 60 B per
// clock and SM) and its HBM bytes at its share of the HBM bandwidth (21 B per
// clock and SM), the largest of the three plus a part of the others.
double brick_cost(const Column& c, int nz, int P, int nF) {
    const double lds_per_row = 2.0 + 2.0 * (nz + P) / (nz * 2.5);
    const double box = 4.0 * c.bxb * c.byb * (nz + P);
    const double smem = (nF * (box + 128.0 * c.warps * nz * lds_per_row) + 8.0 * c.bxb * c.byb * (nz + 2 * P)) / 128.0;
    const double l2 = nF * box / 60.0;
    const double dram = nF * 4.0 * c.nx * c.ny * nz / 21.0;
    const double hi = std::max(smem, std::max(l2, dram));
    return hi + 0.3 * (smem + l2 + dram - hi) + 2000.0;
}

PlanResult plan_bricks(int m, int P, int nF, int nsm, int bzm, int ncw_max, size_t smem_max) {
    PlanResult best;
    const int GX = (m + 3) / 4, GY = (m + 7) / 8;
    for (int ns = 3; ns >= 2; --ns) {
        for (int nbx = 1; nbx <= std::min(GX, 32); ++nbx) {
            const std::vector<int> gxs = split_even(GX, nbx);
            for (int nby = 1; nby <= std::min(GY, 32); ++nby) {
                const std::vector<int> gys = split_even(GY, nby);
                if (gxs.back() * gys.back() > ncw_max) continue;
                std::vector<Column> cols;
                int xa = 0;
                for (int kx = 0; kx < nbx; ++kx) {
                    const int nx = std::min(4 * gxs[kx], m - xa);
                    int ya = 0;
                    for (int ky = 0; ky < nby; ++ky) {
                        const int ny = std::min(8 * gys[ky], m - ya);
                        Column c{xa, nx, ya, ny, box_x(nx, P), ny + 2 * P, gxs[kx] * ((ny + 7) / 8)};
                        cols.push_back(c);
                        ya += 8 * gys[ky];
                    }
                    xa += 4 * gxs[kx];
                }
                // classes: columns with the same box cross-section share one z split
                std::vector<int> cls_of(cols.size());
                std::vector<Column> reps;
                std::vector<int> count;
                for (size_t i = 0; i < cols.size(); ++i) {
                    int found = -1;
                    for (size_t r = 0; r < reps.size(); ++r)
                        if (reps[r].bxb == cols[i].bxb && reps[r].byb == cols[i].byb) found = (int)r;
                    if (found < 0) {
                        found = (int)reps.size();
                        reps.push_back(cols[i]);
                        count.push_back(0);
                    } else {
                        reps[found].warps = std::max(reps[found].warps, cols[i].warps);
                        reps[found].nx = std::max(reps[found].nx, cols[i].nx);
                        reps[found].ny = std::max(reps[found].ny, cols[i].ny);
                    }
                    cls_of[i] = found;
                    count[found] += 1;
                }
                if ((int)reps.size() > kBrickMaxCls) continue;
                // z splits per class: at least what the register tile (bzm) and the
                // shared memory allow, then more while one wave of bricks remains
                const size_t budget = (smem_max - 1024) / 4 - (size_t)(ns + 1) * 256;   // floats (stage rounding)
                std::vector<int> zc(reps.size());
                bool feasible = true;
                int total = 0;
                for (size_t r = 0; r < reps.size(); ++r) {
                    int z = (m + bzm - 1) / bzm;
                    for (;;) {
                        const int nz = (m + z - 1) / z;
                        const size_t area = (size_t)reps[r].bxb * reps[r].byb;
                        if ((size_t)ns * area * (nz + P) + area * (nz + 2 * P) <= budget) break;
                        if (nz == 1) {
                            feasible = false;
                            break;
                        }
                        ++z;
                    }
                    zc[r] = z;
                    total += count[r] * z;
                }
                if (!feasible) continue;
                for (;;) {
                    int worst = -1;
                    double wc = -1.0;
                    for (size_t r = 0; r < reps.size(); ++r) {
                        const double c = brick_cost(reps[r], (m + zc[r] - 1) / zc[r], P, nF);
                        if (c > wc) {
                            wc = c;
                            worst = (int)r;
                        }
                    }
                    const int nz = (m + zc[worst] - 1) / zc[worst];
                    if (nz <= 1 || total + count[worst] > nsm) break;
                    zc[worst] += 1;
                    total += count[worst];
                }
                double mk = 0.0;
                for (size_t r = 0; r < reps.size(); ++r)
                    mk = std::max(mk, brick_cost(reps[r], (m + zc[r] - 1) / zc[r], P, nF));
                mk *= (double)((total + nsm - 1) / nsm);
                if (ns == 2) mk *= 1.05;   // a shallower ring hides less latency
                if (mk < best.cost) {
                    PlanResult pr;
                    pr.cost = mk;
                    pr.ns = ns;
                    pr.ncls = (int)reps.size();
                    int ncw = 0;
                    size_t stage = 0, xt = 0;
                    for (size_t r = 0; r < reps.size(); ++r) {
                        const int nz = (m + zc[r] - 1) / zc[r];
                        pr.bx[r] = reps[r].bxb;
                        pr.by[r] = reps[r].byb;
                        pr.bz[r] = nz + P;
                        stage = std::max(stage, (size_t)reps[r].bxb * reps[r].byb * (nz + P));
                        xt = std::max(xt, (size_t)reps[r].bxb * reps[r].byb * (nz + 2 * P));
                    }
                    for (size_t i = 0; i < cols.size(); ++i) {
                        const int r = cls_of[i];
                        const std::vector<int> zs = split_even(m, zc[r]);
                        int za = 0;
                        for (int z : zs) {
                            BrickDesc b{cols[i].x0, cols[i].y0, za, cols[i].nx, cols[i].ny, z, r, cols[i].warps};
                            pr.bricks.push_back(b);
                            ncw = std::max(ncw, cols[i].warps);
                            za += z;
                        }
                    }
                    pr.ncw = ncw;
                    pr.stage_floats = (int)((stage + 255) / 256 * 256);   // 1 KB-aligned stages
                    pr.xt_floats = (int)((xt + 255) / 256 * 256);
                    best = pr;
                }
            }
        }
    }
    return best;
}

}  // namespace

// ---------------------------------------------------------------- padded copy
__global__ void brick_relayout_kernel(const float* __restrict__ src, long long pitch, float* __restrict__ dst,
                                      long long fsz, int m, int XP, int P, const int* __restrict__ order,
                                      long long total) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long f = idx / fsz, r = idx - f * fsz;
        const long long line = r / XP;
        const int xr = (int)(r - line * XP) - P;
        float v = 0.f;
        if (xr >= 0 && xr < m) v = src[(size_t)order[f] * pitch + line * m + xr];
        dst[idx] = v;
    }
}

// ---------------------------------------------------------------- apply kernel
// One brick per CTA: warps 0 .. ncw-1 compute, warp ncw issues the field boxes.
// Shared memory: [2 NS mbarriers | NS stages | vector tile].
template <int P, bool MASS, bool XREG, int BZM, int NS>
__global__ void __launch_bounds__(1024, 1)
    brick_apply_kernel(const __grid_constant__ BrickMaps maps, const BrickDesc* __restrict__ bricks, int nF,
                       int stage_floats, const float* __restrict__ x, float* __restrict__ y, int m, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t* full = (uint64_t*)smem_raw;
    uint64_t* empty = full + NS;
    float* stages = (float*)(smem_raw + 1024);
    float* xt = stages + (size_t)NS * stage_floats;
    const int ncw = (int)(blockDim.x >> 5) - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncw);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const BrickDesc b = bricks[blockIdx.x];
    if (warp == ncw) {
        if (lane == 0) {
            const BrickGeo g = brick_geo(maps, b, 0, 0);
            const bool ok = brick_produce<P, NS>(maps, g, stages, stage_floats, full, empty, nF, 0ull,
                                                 l2_evict_first_policy());
            if (!ok) atomicOr(err, 16);
            brick_drain<NS>(full, (unsigned long long)nF);
        }
        return;
    }
    const BrickGeo g = brick_geo(maps, b, warp, lane);
    brick_load_tile<P, false>(xt, x, g, m, warp, ncw, lane);
    float acc[BZM], xo[BZM];
    if (!brick_pass<P, MASS, XREG, BZM, NS>(g, stages, stage_floats, xt, full, empty, 0ull, lane, acc, xo)) {
        if (lane == 0) atomicOr(err, 16);
        return;
    }
    if (g.lane_ok) {
        const long long mm = (long long)m * m;
        float* yc = y + (long long)g.z0 * mm + (long long)(g.y0 + g.cy) * m + g.x0 + g.cx;
#pragma unroll
        for (int zl = 0; zl < BZM; ++zl)
            if (zl < g.nz) yc[zl * mm] = acc[zl];
    }
}

constexpr int kBrickBZM = 12;   // rows per lane column (register tile)
constexpr int kBrickNcwMax = 31;

template <int P, bool MASS, int NS>
static int brick_launch(const BrickOps& bo, const BrickMaps& maps, int nF, const float* x, float* y,
                        cudaStream_t st) {
    // M~: the group's vector values in registers; K~ (difference form, which also
    // holds the row's own values) reads them from the tile (no spills at 64 registers)
    auto fn = brick_apply_kernel<P, MASS, MASS, kBrickBZM, NS>;
    IGA_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    fn<<<bo.nbricks, (bo.ncw + 1) * 32, bo.smem, st>>>(maps, bo.bricks.as<BrickDesc>(), nF, bo.stage_floats, x, y,
                                                      bo.m, bo.err.as<int>());
    IGA_LAUNCH_CHECK("brick_apply_kernel");
    return IGA_OK;
}

template <int P>
static int brick_apply_p(const iga_ops* ops, int which, const float* x, float* y, cudaStream_t st) {
    const BrickOps& bo = *ops->brick;
    const bool mass = which == IGA_OP_M;
    const BrickMaps& maps = mass ? bo.mapM : bo.mapK;
    const int nF = mass ? ops->nM : ops->nK;
    if (bo.ns == 3) return mass ? brick_launch<P, true, 3>(bo, maps, nF, x, y, st)
                                : brick_launch<P, false, 3>(bo, maps, nF, x, y, st);
    return mass ? brick_launch<P, true, 2>(bo, maps, nF, x, y, st) : brick_launch<P, false, 2>(bo, maps, nF, x, y, st);
}

// IGA_PATH_AUTO takes the brick kernels where they measured faster than the row
// kernels on GB300 (cube family, one brick per SM): M~ from about 3,000 rows per
// brick (n_el = 80: 47.7 against 51.1 us), K~ from about 5,000 (n_el = 96: 60.3
// against 64.2 us; n_el = 80: 49.5 against 45.5 us).  Smaller bricks are bound by
// the latency of the field ring.
bool brick_usable(const iga_ops* ops, int which) {
    if (!ops->brick || ops->path == IGA_PATH_ROWS) return false;
    if (ops->path == IGA_PATH_BRICK) return true;
    const double rows = (double)ops->N / ops->brick->nbricks;
    return rows >= (which == IGA_OP_M ? 3000.0 : 5000.0);
}

int brick_apply(const iga_ops* ops, int which, const float* x, float* y, cudaStream_t st) {
    if (!ops->brick) return fail(IGA_ERR_ARG, "no brick form of the operators (3-D FP32 only)");
    return ops->brick->P == 1 ? brick_apply_p<1>(ops, which, x, y, st) : brick_apply_p<2>(ops, which, x, y, st);
}

// ---------------------------------------------------------------- preparation
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static int encode_maps(BrickMaps& maps, const BrickOps& bo, void* base, int nF, const PlanResult& pr) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(IGA_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    std::memset(&maps, 0, sizeof(maps));
    const cuuint64_t dims[4] = {(cuuint64_t)bo.XP, (cuuint64_t)bo.m, (cuuint64_t)bo.m, (cuuint64_t)nF};
    const cuuint64_t strides[3] = {(cuuint64_t)bo.XP * 4, (cuuint64_t)bo.XP * bo.m * 4, (cuuint64_t)bo.fsz * 4};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int c = 0; c < pr.ncls; ++c) {
        const cuuint32_t box[4] = {(cuuint32_t)pr.bx[c], (cuuint32_t)pr.by[c], (cuuint32_t)pr.bz[c], 1};
        const CUresult r = enc(&maps.tm[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(IGA_ERR_CUDA, "cuTensorMapEncodeTiled failed for a brick box");
        maps.bx[c] = pr.bx[c];
        maps.by[c] = pr.by[c];
        maps.bz[c] = pr.bz[c];
    }
    return IGA_OK;
}

// Tensor maps of the padded u copy: 3-D (XP, m, m), one box per class covering
// the class's vector tile (the brick grown by P on every side).
static int encode_tile_maps(BrickMaps& maps, const BrickOps& bo, void* base, const PlanResult& pr) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(IGA_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    std::memset(&maps, 0, sizeof(maps));
    const cuuint64_t dims[3] = {(cuuint64_t)bo.XP, (cuuint64_t)bo.m, (cuuint64_t)bo.m};
    const cuuint64_t strides[2] = {(cuuint64_t)bo.XP * 4, (cuuint64_t)bo.XP * bo.m * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int c = 0; c < pr.ncls; ++c) {
        const cuuint32_t box[3] = {(cuuint32_t)pr.bx[c], (cuuint32_t)pr.by[c], (cuuint32_t)(pr.bz[c] + bo.P)};
        const CUresult r = enc(&maps.tm[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(IGA_ERR_CUDA, "cuTensorMapEncodeTiled failed for a vector tile box");
        maps.bx[c] = pr.bx[c];
        maps.by[c] = pr.by[c];
        maps.bz[c] = pr.bz[c] + bo.P;
    }
    return IGA_OK;
}

int brick_prepare(iga_ops* ops, cudaStream_t st) {
    if (ops->dim != 3 || (ops->p != 1 && ops->p != 2) || !ops->fK32.ptr || !ops->fM32.ptr) return IGA_OK;
    const int P = ops->p, m = ops->m;
    int dev = 0, sms = 152;
    IGA_CUDA(cudaGetDevice(&dev));
    IGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const PlanResult pr = plan_bricks(m, P, ops->nM, sms, kBrickBZM, kBrickNcwMax, 227 * 1024);
    if (pr.bricks.empty()) return IGA_OK;   // no plan: the row kernels stay in use
    std::unique_ptr<BrickOps> bo(new (std::nothrow) BrickOps());
    if (!bo) return fail(IGA_ERR_OOM, "host allocation failed");
    bo->P = P;
    bo->m = m;
    bo->XP = (m + 2 * P + 3) / 4 * 4;
    bo->fsz = (long long)bo->XP * m * m;
    bo->ncw = pr.ncw;
    bo->ns = pr.ns;
    bo->bzm = kBrickBZM;
    bo->nbricks = (int)pr.bricks.size();
    bo->ncls = pr.ncls;
    bo->stage_floats = pr.stage_floats;
    bo->xt_floats = pr.xt_floats;
    bo->smem = 1024 + sizeof(float) * ((size_t)pr.ns * pr.stage_floats + pr.xt_floats);
    bo->host = pr.bricks;
    int rc = bo->bricks.alloc(sizeof(BrickDesc) * pr.bricks.size());
    if (!rc) rc = bo->fK.alloc(sizeof(float) * (size_t)ops->nK * bo->fsz);
    if (!rc) rc = bo->fM.alloc(sizeof(float) * (size_t)ops->nM * bo->fsz);
    if (!rc) rc = bo->err.alloc(64);
    if (rc) return rc;
    // field order of the copies: K~ the grouped table, M~ the diagonal then the table
    std::vector<int> order(ops->nM);
    if (P == 1) {
        constexpr BrickTable<1> t = make_brick_table<1>();
        for (int k = 0; k < BrickTable<1>::NF; ++k) order[k] = t.f[k].u;
    } else {
        constexpr BrickTable<2> t = make_brick_table<2>();
        for (int k = 0; k < BrickTable<2>::NF; ++k) order[k] = t.f[k].u;
    }
    std::vector<int> orderM(ops->nM);
    orderM[0] = 0;
    for (int k = 0; k < ops->nK; ++k) orderM[k + 1] = order[k] + 1;
    DevBuf dord;
    rc = dord.alloc(sizeof(int) * 2 * ops->nM);
    if (rc) return rc;
    IGA_CUDA(cudaMemcpyAsync(bo->bricks.ptr, pr.bricks.data(), sizeof(BrickDesc) * pr.bricks.size(),
                             cudaMemcpyHostToDevice, st));
    IGA_CUDA(cudaMemcpyAsync(dord.ptr, order.data(), sizeof(int) * ops->nK, cudaMemcpyHostToDevice, st));
    IGA_CUDA(cudaMemcpyAsync(dord.as<int>() + ops->nM, orderM.data(), sizeof(int) * ops->nM, cudaMemcpyHostToDevice,
                             st));
    IGA_CUDA(cudaMemsetAsync(bo->err.ptr, 0, 64, st));
    {
        const long long tk = (long long)ops->nK * bo->fsz, tm = (long long)ops->nM * bo->fsz;
        const int gk = (int)std::min<long long>((tk + 255) / 256, (long long)sms * 16);
        const int gm = (int)std::min<long long>((tm + 255) / 256, (long long)sms * 16);
        brick_relayout_kernel<<<gk, 256, 0, st>>>(ops->fK32.as<float>(), ops->pitch, bo->fK.as<float>(), bo->fsz, m,
                                                  bo->XP, P, dord.as<int>(), tk);
        IGA_LAUNCH_CHECK("brick_relayout_kernel");
        brick_relayout_kernel<<<gm, 256, 0, st>>>(ops->fM32.as<float>(), ops->pitch, bo->fM.as<float>(), bo->fsz, m,
                                                  bo->XP, P, dord.as<int>() + ops->nM, tm);
        IGA_LAUNCH_CHECK("brick_relayout_kernel");
    }
    rc = encode_maps(bo->mapK, *bo, bo->fK.ptr, ops->nK, pr);
    if (!rc) rc = encode_maps(bo->mapM, *bo, bo->fM.ptr, ops->nM, pr);
    if (!rc) rc = bo->upad.alloc(sizeof(float) * (size_t)bo->fsz);
    if (!rc) rc = encode_tile_maps(bo->mapU, *bo, bo->upad.ptr, pr);
    if (rc) return rc;
    IGA_CUDA(cudaMemsetAsync(bo->upad.ptr, 0, sizeof(float) * (size_t)bo->fsz, st));
    // dord is freed by its destructor: finish the copies that read it first
    IGA_CUDA(cudaStreamSynchronize(st));
    ops->brick = std::move(bo);
    return IGA_OK;
}

}  // namespace iga

using namespace iga;

extern "C" int iga_ops_set_path(iga_ops* ops, int path) {
    if (!ops) return fail(IGA_ERR_ARG, "null argument");
    if (path != IGA_PATH_AUTO && path != IGA_PATH_ROWS && path != IGA_PATH_BRICK && path != IGA_PATH_ONTHEFLY)
        return fail(IGA_ERR_ARG, "path must be IGA_PATH_AUTO, IGA_PATH_ROWS, IGA_PATH_BRICK or IGA_PATH_ONTHEFLY");
    if (path == IGA_PATH_BRICK && !ops->brick) return fail(IGA_ERR_ARG, "no brick form (3-D, p <= 2 only)");
    if (path == IGA_PATH_ONTHEFLY) {
        const int rc = onthefly_prepare(ops);
        if (rc) return rc;
    }
    ops->path = path;
    return IGA_OK;
}

extern "C" int iga_ops_brick_info(const iga_ops* ops, int* nbricks, int* threads, int* stages, int* smem_bytes,
                                  int* brick_paths) {
    if (!ops) return fail(IGA_ERR_ARG, "null argument");
    const BrickOps* bo = ops->brick.get();
    if (nbricks) *nbricks = bo ? bo->nbricks : 0;
    if (threads) *threads = bo ? (bo->ncw + 1) * 32 : 0;
    if (stages) *stages = bo ? bo->ns : 0;
    if (smem_bytes) *smem_bytes = bo ? (int)bo->smem : 0;
    if (brick_paths)
        *brick_paths = (brick_usable(ops, IGA_OP_K) ? 1 : 0) | (brick_usable(ops, IGA_OP_M) ? 2 : 0);
    return IGA_OK;
}
