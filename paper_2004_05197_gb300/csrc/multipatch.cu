// Multi-patch operators (Sec. 3.2 and Sec. 3.4, remarks on multi-patch
// geometries): every patch keeps its own surrogate fields (its own stencil
// functions, assembled by iga_surrogate_assemble on its own space), and the
// global matrix of the C0-conforming multi-patch space is the sum over patches of
// P_l^T A_l P_l, P_l the map from global to patch-local coefficients.
//
// Applied matrix-free: gather the patch-local vectors, apply every patch's
// stencil operator with the single-patch kernels, and sum the patch results of
// every global function in a fixed order (a function on a shared side belongs
// to two or more patches).  The mass solve is Jacobi-PCG on the global system
// with its scalars on the device; the host checks convergence every kMpCheck
// iterations.
//
// Global numbering: local functions visited patch by patch, each patch in
// colexicographic order; the side functions identified by the interfaces (sides
// of 2-D patches, faces of 3-D patches) form classes, and a class takes the next
// global index at its first member.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "iga_internal.cuh"
#include "leapfrog.cuh"

struct iga_multipatch {
    std::vector<const iga_ops*> patches;
    std::vector<long long> off, n;           // patch-local offsets (concatenated) and sizes
    long long G = 0, L = 0;                  // global and total local counts
    std::vector<long long> l2g_h;            // [L] global index of every local function
    iga::DevBuf l2g;                         // int [L]
    iga::DevBuf gptr, gpatch, glocal;        // CSR global -> (patch, local index), int
    iga::DevBuf poff, pn;                    // long long [npatch]
    iga::DevBuf dinv64, dinv32;              // inverse Jacobi diagonal of the global M~
    iga::DevBuf work;                        // per-call scratch (grown on demand)
};

namespace iga {
namespace {

// Linear (colex) local index of entry e of a side: side 2k is {i_(k+1) = 0}, side
// 2k+1 is {i_(k+1) = m-1}; the entries run colex over the remaining indices.
long long side_index(int dim, int m, int side, long long e) {
    const int axis = side / 2;
    const long long c[2] = {e % m, e / m};   // remaining indices, the first one fastest
    long long idx = 0, stride = 1;
    int r = 0;
    for (int k = 0; k < dim; ++k, stride *= m) idx += stride * (k == axis ? (side % 2 ? m - 1 : 0) : c[r++]);
    return idx;
}

// Entry of side b that meets entry e = u + m v of side a: bit 2 of orient swaps u
// and v, then bit 0 reverses u and bit 1 reverses v (2-D: e = u, bit 0 only).
long long oriented_entry(int dim, int m, int orient, long long e) {
    if (dim == 2) return (orient & 1) ? m - 1 - e : e;
    long long u = e % m, v = e / m;
    if (orient & 4) std::swap(u, v);
    if (orient & 1) u = m - 1 - u;
    if (orient & 2) v = m - 1 - v;
    return u + (long long)m * v;
}

long long uf_find(std::vector<long long>& parent, long long a) {
    while (parent[a] != a) {
        parent[a] = parent[parent[a]];
        a = parent[a];
    }
    return a;
}

// x_l[r][i] = x[r][l2g[off + i]] for the rows of one patch (patch-major layout)
template <typename T>
__global__ void mp_gather_kernel(const T* __restrict__ x, long long G, const int* __restrict__ l2g, long long off,
                                 long long n, T* __restrict__ xl, int R) {
    const long long tot = (long long)R * n;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(k / n);
        const long long i = k % n;
        xl[k] = x[(long long)r * G + l2g[off + i]];
    }
}

// y[r][g] = sum over the (patch, local) entries of g, in CSR order, of y_l
template <typename T>
__global__ void mp_scatter_kernel(const T* __restrict__ yl, const int* __restrict__ gptr, const int* __restrict__ gpatch,
                                  const int* __restrict__ glocal, const long long* __restrict__ poff,
                                  const long long* __restrict__ pn, long long G, int R, T* __restrict__ y) {
    const long long tot = (long long)R * G;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(k / G);
        const long long g = k % G;
        T s = T(0);
        for (int j = gptr[g]; j < gptr[g + 1]; ++j) {
            const int l = gpatch[j];
            s += yl[(long long)R * poff[l] + (long long)r * pn[l] + glocal[j]];
        }
        y[k] = s;
    }
}

// global diagonal of M~: sum of the patch diagonals (field 0 of every patch's M~)
__global__ void mp_diag_kernel(const double* const* __restrict__ fm, const int* __restrict__ gptr,
                               const int* __restrict__ gpatch, const int* __restrict__ glocal, long long G,
                               double* dinv64, float* dinv32, int* bad) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int j = gptr[g]; j < gptr[g + 1]; ++j) d += fm[gpatch[j]][glocal[j]];
        if (!(d > 0.0)) atomicOr(bad, 1);
        dinv64[g] = 1.0 / d;
        dinv32[g] = (float)(1.0 / d);
    }
}

constexpr int kMpThreads = 256;
constexpr int kMpBlocks = 152 * 8;
constexpr int kMpCheck = 16;   // CG iterations between host checks of the multi-patch solve

// per-block FP64 partial sums of K dot products over [R][G] vectors (fixed order)
template <int K>
__device__ __forceinline__ void mp_block_partials(double (&v)[K], double* out) {
    __shared__ double ws[kMpThreads / 32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) ws[w][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int q = 0; q < kMpThreads / 32; ++q) s += ws[q][threadIdx.x];
        out[(size_t)blockIdx.x * K + threadIdx.x] = s;
    }
}

// partials[b][r] of (p_r, q_r)
template <typename T>
__global__ void __launch_bounds__(kMpThreads) mp_dot_kernel(const T* __restrict__ p, const T* __restrict__ q, long long G,
                                                            int r, double* partials) {
    double v[1] = {0.0};
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x)
        v[0] += (double)p[(long long)r * G + g] * (double)q[(long long)r * G + g];
    mp_block_partials<1>(v, partials);
}

// x += alpha p, r -= alpha q, z = D^-1 r; partials (r, r), (r, z) of one right-hand side
template <typename T>
__global__ void __launch_bounds__(kMpThreads) mp_update_kernel(T* x, double* res, T* z, const T* __restrict__ p,
                                                               const T* __restrict__ q, const T* __restrict__ dinv,
                                                               long long G, int r, double alpha, double* partials) {
    double v[2] = {0.0, 0.0};
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long o = (long long)r * G + g;
        x[o] = x[o] + (T)alpha * p[o];
        const double ri = res[o] - alpha * (double)q[o];
        res[o] = ri;
        const T zi = (T)((double)dinv[g] * ri);
        z[o] = zi;
        v[0] += ri * ri;
        v[1] += ri * (double)zi;
    }
    mp_block_partials<2>(v, partials);
}

// r = b - q (q = A x), z = D^-1 r, p = z; partials (r, r), (r, z), (b, b)
template <typename T>
__global__ void __launch_bounds__(kMpThreads) mp_init_kernel(const T* __restrict__ b, const T* __restrict__ q, double* res,
                                                             T* z, T* p, const T* __restrict__ dinv, long long G, int r,
                                                             double* partials) {
    double v[3] = {0.0, 0.0, 0.0};
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long o = (long long)r * G + g;
        const double bi = (double)b[o];
        const double ri = bi - (double)q[o];
        res[o] = ri;
        const T zi = (T)((double)dinv[g] * ri);
        z[o] = zi;
        p[o] = zi;
        v[0] += ri * ri;
        v[1] += ri * (double)zi;
        v[2] += bi * bi;
    }
    mp_block_partials<3>(v, partials);
}

// p = z + beta p
template <typename T>
__global__ void mp_dir_kernel(T* p, const T* __restrict__ z, long long G, int r, double beta) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long o = (long long)r * G + g;
        p[o] = z[o] + (T)beta * p[o];
    }
}

// out[k] = sum over blocks of partials[b][k], fixed order (one block)
template <int K>
__global__ void mp_reduce_kernel(const double* __restrict__ partials, int nb, double* out) {
    __shared__ double ws[kMpThreads / 32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[(size_t)b * K + k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) ws[w][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int q = 0; q < kMpThreads / 32; ++q) s += ws[q][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// CG scalars of one right-hand side, kept on the device between host checks
struct MpScal {
    double rz, rr, bn, alpha, beta;
    int active, iters, brk, pad;
};
// alpha = (r, z) / (p, M p) for every active right-hand side (breakdown: inactive, brk)
__global__ void mp_alpha_kernel(MpScal* sc, const double* __restrict__ red, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || !sc[r].active) return;
    const double pq = red[3 * r];
    if (!(pq > 0.0) || !isfinite(pq)) {
        sc[r].brk = 1;
        sc[r].active = 0;
        sc[r].alpha = 0.0;
        return;
    }
    sc[r].alpha = sc[r].rz / pq;
}
// after the update: count the iteration, test ||r|| <= rtol ||b||, else beta
__global__ void mp_beta_kernel(MpScal* sc, const double* __restrict__ red, double rtol, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || !sc[r].active) return;
    sc[r].iters += 1;
    sc[r].rr = red[3 * r];
    const double rz_new = red[3 * r + 1];
    if (rtol > 0.0 && sqrt(sc[r].rr) <= rtol * sc[r].bn) {
        sc[r].active = 0;
        return;
    }
    sc[r].beta = rz_new / sc[r].rz;
    sc[r].rz = rz_new;
}
// the update with alpha from the device (no work, zero partials, once inactive)
template <typename T>
__global__ void __launch_bounds__(kMpThreads) mp_update_dev_kernel(T* x, double* res, T* z, const T* __restrict__ p,
                                                                   const T* __restrict__ q, const T* __restrict__ dinv,
                                                                   long long G, int r, const MpScal* sc,
                                                                   double* partials) {
    double v[2] = {0.0, 0.0};
    if (sc[r].active) {
        const double alpha = sc[r].alpha;
        for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G;
             g += (long long)gridDim.x * blockDim.x) {
            const long long o = (long long)r * G + g;
            x[o] = x[o] + (T)alpha * p[o];
            const double ri = res[o] - alpha * (double)q[o];
            res[o] = ri;
            const T zi = (T)((double)dinv[g] * ri);
            z[o] = zi;
            v[0] += ri * ri;
            v[1] += ri * (double)zi;
        }
    }
    mp_block_partials<2>(v, partials);
}
// p = z + beta p while active
template <typename T>
__global__ void mp_dir_dev_kernel(T* p, const T* __restrict__ z, long long G, int r, const MpScal* sc) {
    if (!sc[r].active) return;
    const double beta = sc[r].beta;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < G; g += (long long)gridDim.x * blockDim.x) {
        const long long o = (long long)r * G + g;
        p[o] = z[o] + (T)beta * p[o];
    }
}

}  // namespace
}  // namespace iga

using namespace iga;

extern "C" int iga_multipatch_create(int npatch, const iga_ops* const* patches, int ninterface,
                                     const iga_interface* ifs, iga_multipatch** out) {
    if (!out || npatch < 1 || !patches || ninterface < 0 || (ninterface > 0 && !ifs))
        return fail(IGA_ERR_ARG, "bad arguments");
    *out = nullptr;
    for (int l = 0; l < npatch; ++l) {
        if (!patches[l]) return fail(IGA_ERR_ARG, "null patch");
        if (patches[l]->dim != patches[0]->dim) return fail(IGA_ERR_ARG, "patches must share the dimension");
        if (patches[l]->p != patches[0]->p) return fail(IGA_ERR_ARG, "patches must share the degree p");
    }
    iga_multipatch* mp = new (std::nothrow) iga_multipatch();
    if (!mp) return fail(IGA_ERR_OOM, "host allocation failed");
    auto bail = [&](int rc) {
        delete mp;
        return rc;
    };
    mp->patches.assign(patches, patches + npatch);
    mp->off.resize(npatch);
    mp->n.resize(npatch);
    long long L = 0;
    for (int l = 0; l < npatch; ++l) {
        mp->off[l] = L;
        mp->n[l] = patches[l]->N;
        L += patches[l]->N;
    }
    if (L > (1LL << 31) - 1) return bail(fail(IGA_ERR_ARG, "too many local functions for 32-bit indexing"));
    mp->L = L;
    // union-find over the local functions; the class representative is its smallest member
    std::vector<long long> parent(L);
    std::iota(parent.begin(), parent.end(), 0LL);
    for (int f = 0; f < ninterface; ++f) {
        const iga_interface& it = ifs[f];
        const int dim = patches[0]->dim;
        if (it.patch_a < 0 || it.patch_a >= npatch || it.patch_b < 0 || it.patch_b >= npatch ||
            it.side_a < 0 || it.side_a >= 2 * dim || it.side_b < 0 || it.side_b >= 2 * dim)
            return bail(fail(IGA_ERR_ARG, "interface names a patch or side that does not exist"));
        if (it.reversed < 0 || it.reversed > (dim == 2 ? 1 : 7))
            return bail(fail(IGA_ERR_ARG, "orientation must be 0..1 (2-D) or 0..7 (3-D)"));
        const int ma = patches[it.patch_a]->m, mb = patches[it.patch_b]->m;
        if (ma != mb) return bail(fail(IGA_ERR_ARG, "glued sides need the same number of functions"));
        if (it.patch_a == it.patch_b && it.side_a == it.side_b)
            return bail(fail(IGA_ERR_ARG, "a side cannot be glued to itself"));
        const long long ne = dim == 2 ? ma : (long long)ma * ma;
        for (long long k = 0; k < ne; ++k) {
            const long long a = mp->off[it.patch_a] + side_index(dim, ma, it.side_a, k);
            const long long b =
                mp->off[it.patch_b] + side_index(dim, mb, it.side_b, oriented_entry(dim, ma, it.reversed, k));
            const long long ra = uf_find(parent, a), rb = uf_find(parent, b);
            if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
        }
    }
    mp->l2g_h.assign(L, -1);
    std::vector<long long> cls(L, -1);
    long long G = 0;
    for (long long k = 0; k < L; ++k) {
        const long long r = uf_find(parent, k);
        if (cls[r] < 0) cls[r] = G++;
        mp->l2g_h[k] = cls[r];
    }
    mp->G = G;
    // CSR global -> (patch, local), members in visiting order
    std::vector<int> cnt(G + 1, 0), gpatch(L), glocal(L), l2g32(L);
    for (long long k = 0; k < L; ++k) cnt[mp->l2g_h[k] + 1] += 1;
    for (long long g = 0; g < G; ++g) cnt[g + 1] += cnt[g];
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int l = 0; l < npatch; ++l)
        for (long long i = 0; i < mp->n[l]; ++i) {
            const long long k = mp->off[l] + i;
            const long long g = mp->l2g_h[k];
            gpatch[fill[g]] = l;
            glocal[fill[g]] = (int)i;
            ++fill[g];
            l2g32[k] = (int)g;
        }
    int rc = mp->l2g.alloc(sizeof(int) * L);
    if (!rc) rc = mp->gptr.alloc(sizeof(int) * (G + 1));
    if (!rc) rc = mp->gpatch.alloc(sizeof(int) * L);
    if (!rc) rc = mp->glocal.alloc(sizeof(int) * L);
    if (!rc) rc = mp->poff.alloc(sizeof(long long) * npatch);
    if (!rc) rc = mp->pn.alloc(sizeof(long long) * npatch);
    if (!rc) rc = mp->dinv64.alloc(sizeof(double) * G);
    if (!rc) rc = mp->dinv32.alloc(sizeof(float) * G);
    if (rc) return bail(rc);
    DevBuf fm, bad;
    std::vector<const double*> fm_h(npatch);
    for (int l = 0; l < npatch; ++l) fm_h[l] = patches[l]->fM64.as<double>();
    if ((rc = fm.alloc(sizeof(double*) * npatch)) || (rc = bad.alloc(sizeof(int)))) return bail(rc);
    cudaError_t e = cudaMemcpy(mp->l2g.ptr, l2g32.data(), sizeof(int) * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mp->gptr.ptr, cnt.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mp->gpatch.ptr, gpatch.data(), sizeof(int) * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mp->glocal.ptr, glocal.data(), sizeof(int) * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mp->poff.ptr, mp->off.data(), sizeof(long long) * npatch, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mp->pn.ptr, mp->n.data(), sizeof(long long) * npatch, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fm.ptr, fm_h.data(), sizeof(double*) * npatch, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(bad.ptr, 0, sizeof(int));
    if (e != cudaSuccess) return bail(cuda_fail(e, "multipatch upload"));
    const int grid = (int)std::min<long long>((G + 255) / 256, kMpBlocks);
    mp_diag_kernel<<<grid, 256>>>(fm.as<const double*>(), mp->gptr.as<int>(), mp->gpatch.as<int>(),
                                  mp->glocal.as<int>(), G, mp->dinv64.as<double>(), mp->dinv32.as<float>(),
                                  bad.as<int>());
    count_launch();
    int bad_h = 0;
    e = cudaMemcpy(&bad_h, bad.ptr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bail(cuda_fail(e, "mp_diag_kernel"));
    if (bad_h) return bail(fail(IGA_ERR_NONFINITE, "non-positive global mass diagonal"));
    *out = mp;
    return IGA_OK;
}

extern "C" int iga_multipatch_destroy(iga_multipatch* mp) {
    delete mp;
    return IGA_OK;
}

extern "C" int iga_multipatch_size(const iga_multipatch* mp, long long* n_global) {
    if (!mp || !n_global) return fail(IGA_ERR_ARG, "null argument");
    *n_global = mp->G;
    return IGA_OK;
}

extern "C" int iga_multipatch_global_index(const iga_multipatch* mp, int patch, long long* host_map) {
    if (!mp || !host_map) return fail(IGA_ERR_ARG, "null argument");
    if (patch < 0 || patch >= (int)mp->patches.size()) return fail(IGA_ERR_ARG, "no such patch");
    std::memcpy(host_map, mp->l2g_h.data() + mp->off[patch], sizeof(long long) * mp->n[patch]);
    return IGA_OK;
}

namespace iga {
namespace {

// Scratch carve: x_l, y_l [R][L] (dtype), res [R][G] FP64, z, p, q [R][G] (dtype),
// partials [kMpBlocks][3] and reduced scalars [R][3] FP64.
struct MpWork {
    void *xl, *yl, *z, *p, *q;
    double *res, *partials, *red;
    MpScal* scal;
};

size_t mp_work_bytes(const iga_multipatch* mp, size_t es, int R) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return 2 * up(es * R * mp->L) + up(8 * (size_t)R * mp->G) + 3 * up(es * R * mp->G) + up(8 * kMpBlocks * 3) +
           up(8 * 3 * (size_t)R) + up(64 * (size_t)R) + 256;
}

int mp_work(const iga_multipatch* mp, size_t es, int R, MpWork& w) {
    iga_multipatch* m = const_cast<iga_multipatch*>(mp);
    const size_t need = mp_work_bytes(mp, es, R);
    if (m->work.bytes < need) {
        int rc = m->work.alloc(need);
        if (rc) return rc;
    }
    char* p = (char*)m->work.ptr;
    auto take = [&](size_t b) {
        void* o = p;
        p += (b + 255) / 256 * 256;
        return o;
    };
    w.xl = take(es * R * mp->L);
    w.yl = take(es * R * mp->L);
    w.res = (double*)take(8 * (size_t)R * mp->G);
    w.z = take(es * R * mp->G);
    w.p = take(es * R * mp->G);
    w.q = take(es * R * mp->G);
    w.partials = (double*)take(8 * kMpBlocks * 3);
    w.red = (double*)take(8 * 3 * (size_t)R);
    w.scal = (MpScal*)take(64 * (size_t)R);
    return IGA_OK;
}

template <typename T>
int mp_apply_typed(const iga_multipatch* mp, int which, const T* x, T* y, int R, cudaStream_t st, const MpWork& w) {
    T* xl = (T*)w.xl;
    T* yl = (T*)w.yl;
    for (size_t l = 0; l < mp->patches.size(); ++l) {
        const long long n = mp->n[l], base = (long long)R * mp->off[l];
        const int grid = (int)std::min<long long>((R * n + 255) / 256, kMpBlocks);
        mp_gather_kernel<T><<<grid, 256, 0, st>>>(x, mp->G, mp->l2g.as<int>(), mp->off[l], n, xl + base, R);
        IGA_LAUNCH_CHECK("mp_gather_kernel");
        int rc = launch_apply(mp->patches[l], which, sizeof(T) == 8 ? IGA_F64 : IGA_F32, xl + base, yl + base, R, st);
        if (rc) return rc;
    }
    const int grid = (int)std::min<long long>(((long long)R * mp->G + 255) / 256, kMpBlocks);
    mp_scatter_kernel<T><<<grid, 256, 0, st>>>(yl, mp->gptr.as<int>(), mp->gpatch.as<int>(), mp->glocal.as<int>(),
                                               mp->poff.as<long long>(), mp->pn.as<long long>(), mp->G, R, y);
    IGA_LAUNCH_CHECK("mp_scatter_kernel");
    return IGA_OK;
}

template <typename T>
int mp_solve_typed(const iga_multipatch* mp, const T* b, T* x, int R, double rtol, int max_it, int* iters_out,
                   double* relres_out, cudaStream_t st) {
    MpWork w;
    int rc = mp_work(mp, sizeof(T), R, w);
    if (rc) return rc;
    const long long G = mp->G;
    const T* dinv = sizeof(T) == 8 ? (const T*)mp->dinv64.ptr : (const T*)mp->dinv32.ptr;
    T* z = (T*)w.z;
    T* p = (T*)w.p;
    T* q = (T*)w.q;
    const int grid = (int)std::min<long long>((G + kMpThreads - 1) / kMpThreads, kMpBlocks);
    std::vector<double> red(3 * (size_t)R), rz(R), rr(R), bn(R);
    std::vector<int> active(R), iters(R, 0);
    auto reduce_all = [&]() -> int {   // reduced scalars [R][3] to the host
        IGA_CUDA(cudaMemcpyAsync(red.data(), w.red, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, st));
        IGA_CUDA(cudaStreamSynchronize(st));
        return IGA_OK;
    };
    // r = b - A x, z = D^-1 r, p = z
    if ((rc = mp_apply_typed<T>(mp, IGA_OP_M, x, q, R, st, w))) return rc;
    for (int r = 0; r < R; ++r) {
        mp_init_kernel<T><<<grid, kMpThreads, 0, st>>>(b, q, w.res, z, p, dinv, G, r, w.partials);
        IGA_LAUNCH_CHECK("mp_init_kernel");
        mp_reduce_kernel<3><<<1, kMpThreads, 0, st>>>(w.partials, grid, w.red + 3 * r);
        IGA_LAUNCH_CHECK("mp_reduce_kernel");
    }
    if ((rc = reduce_all())) return rc;
    for (int r = 0; r < R; ++r) {
        rr[r] = red[3 * r];
        rz[r] = red[3 * r + 1];
        bn[r] = std::sqrt(red[3 * r + 2]);
        active[r] = bn[r] > 0.0 && !(rtol > 0.0 && std::sqrt(rr[r]) <= rtol * bn[r]);
        if (!(bn[r] > 0.0)) IGA_CUDA(cudaMemsetAsync(x + (size_t)r * G, 0, sizeof(T) * G, st));
    }
    // iterations with the scalars on the device; the host reads them back every
    // kMpCheck iterations (a right-hand side that converges inside a batch stops
    // changing at once: its kernels see active = 0)
    std::vector<MpScal> sc(R);
    for (int r = 0; r < R; ++r) {
        sc[r] = MpScal{rz[r], rr[r], bn[r], 0.0, 0.0, active[r], 0, 0, 0};
    }
    IGA_CUDA(cudaMemcpyAsync(w.scal, sc.data(), sizeof(MpScal) * R, cudaMemcpyHostToDevice, st));
    const int sgrid = (R + 31) / 32;
    for (int it = 0; it < max_it;) {
        bool any = false;
        for (int r = 0; r < R; ++r) any = any || sc[r].active;
        if (!any) break;
        const int nb = std::min(kMpCheck, max_it - it);
        for (int k = 0; k < nb; ++k) {
            if ((rc = mp_apply_typed<T>(mp, IGA_OP_M, p, q, R, st, w))) return rc;
            for (int r = 0; r < R; ++r) {
                mp_dot_kernel<T><<<grid, kMpThreads, 0, st>>>(p, q, G, r, w.partials);
                IGA_LAUNCH_CHECK("mp_dot_kernel");
                mp_reduce_kernel<1><<<1, kMpThreads, 0, st>>>(w.partials, grid, w.red + 3 * r);
                IGA_LAUNCH_CHECK("mp_reduce_kernel");
            }
            mp_alpha_kernel<<<sgrid, 32, 0, st>>>(w.scal, w.red, R);
            IGA_LAUNCH_CHECK("mp_alpha_kernel");
            for (int r = 0; r < R; ++r) {
                mp_update_dev_kernel<T><<<grid, kMpThreads, 0, st>>>(x, w.res, z, p, q, dinv, G, r, w.scal,
                                                                     w.partials);
                IGA_LAUNCH_CHECK("mp_update_dev_kernel");
                mp_reduce_kernel<2><<<1, kMpThreads, 0, st>>>(w.partials, grid, w.red + 3 * r);
                IGA_LAUNCH_CHECK("mp_reduce_kernel");
            }
            mp_beta_kernel<<<sgrid, 32, 0, st>>>(w.scal, w.red, rtol, R);
            IGA_LAUNCH_CHECK("mp_beta_kernel");
            for (int r = 0; r < R; ++r) {
                mp_dir_dev_kernel<T><<<grid, kMpThreads, 0, st>>>(p, z, G, r, w.scal);
                IGA_LAUNCH_CHECK("mp_dir_dev_kernel");
            }
        }
        it += nb;
        IGA_CUDA(cudaMemcpyAsync(sc.data(), w.scal, sizeof(MpScal) * R, cudaMemcpyDeviceToHost, st));
        IGA_CUDA(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r)
            if (sc[r].brk) return fail(IGA_ERR_NONFINITE, "CG breakdown: (p, M p) <= 0 or non-finite");
    }
    for (int r = 0; r < R; ++r) {
        rr[r] = sc[r].rr;
        iters[r] = sc[r].iters;
    }
    bool nc = false;
    for (int r = 0; r < R; ++r) {
        const double rel = bn[r] > 0.0 ? std::sqrt(rr[r]) / bn[r] : 0.0;
        if (iters_out) iters_out[r] = iters[r];
        if (relres_out) relres_out[r] = rel;
        if (rtol > 0.0 && rel > rtol) nc = true;
    }
    IGA_CUDA(cudaStreamSynchronize(st));
    if (nc) return fail(IGA_ERR_NOT_CONVERGED, "multi-patch CG reached max_it before rtol");
    return IGA_OK;
}

// ---------------------------------------------------------------- leapfrog
// b = amp r(t_n) S - K~u (S: the source's global point values, FP64)
template <typename T>
__global__ void mpw_rhs_kernel(const T* __restrict__ ku, const double* __restrict__ src, double scale,
                               T* __restrict__ b, long long G) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G; i += (long long)gridDim.x * blockDim.x)
        b[i] = (T)((src ? scale * src[i] : 0.0) - (double)ku[i]);
}
// u^{n+1} into the u^{n-1} buffers: 2 u^n - u^{n-1} + dt^2 a^n, or u^0 + dt^2/2 a^0
// on the first step.  FP32: the state is the unevaluated pair hi + lo.
__global__ void mpw_update_kernel(const double* __restrict__ u, double* __restrict__ up, const double* __restrict__ a,
                                  double c, int first, long long G) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G; i += (long long)gridDim.x * blockDim.x)
        up[i] = first ? u[i] + c * a[i] : 2.0 * u[i] - up[i] + c * a[i];
}
__global__ void mpw_update_kernel(const float* __restrict__ u, const float* __restrict__ ulo, float* __restrict__ up,
                                  float* __restrict__ uplo, const float* __restrict__ a, float c, int first,
                                  long long G) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G; i += (long long)gridDim.x * blockDim.x) {
        float hn, ln;
        leapfrog_comp(u[i], ulo[i], up[i], uplo[i], __fmul_rn(c, a[i]), first != 0, hn, ln);
        up[i] = hn;
        uplo[i] = ln;
    }
}
// traces[r][n] = sum_k w[r][k] (u + lo)[idx[r][k]]  (one thread per receiver)
template <typename T>
__global__ void mpw_receiver_kernel(const T* __restrict__ u, const T* __restrict__ ulo, const int* __restrict__ idx,
                                    const double* __restrict__ w, int nrec, int nloc, double* __restrict__ traces,
                                    int nsteps, int n) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    double acc = 0.0;
    for (int k = 0; k < nloc; ++k) {
        const int j = idx[(size_t)r * nloc + k];
        acc += w[(size_t)r * nloc + k] * ((double)u[j] + (ulo ? (double)ulo[j] : 0.0));
    }
    traces[(size_t)r * nsteps + n] = acc;
}

// Global point values of the basis at parametric point s of one patch: the patch's
// non-zero local functions mapped to their global indices.
void mp_point(const iga_multipatch* mp, int patch, const double* s, std::vector<int>& gidx, std::vector<double>& gw) {
    const iga_space* sp = mp->patches[patch]->space;
    int nloc = 1;
    for (int d = 0; d < sp->dim; ++d) nloc *= sp->p + 1;
    std::vector<int> idx(nloc);
    std::vector<double> w(nloc);
    point_basis(sp, s, idx.data(), w.data());
    gidx.resize(nloc);
    gw = w;
    for (int k = 0; k < nloc; ++k) gidx[k] = (int)mp->l2g_h[mp->off[patch] + idx[k]];
}

template <typename T>
int mp_leapfrog_typed(const iga_multipatch* mp, double dt, int nsteps, T* u_io, int src_patch, const double* src_s,
                      double f0, double t0, double amp, int nrec, const int* rec_patch, const double* rec_s,
                      double* traces_h, double rtol, int max_it, long long* iters_total, cudaStream_t st) {
    const long long G = mp->G;
    const bool comp = sizeof(T) == 4;
    DevBuf bu, bup, blo, buplo, ba, bb, bku, bsrc, bridx, brw, btr;
    int rc = bu.alloc(sizeof(T) * G);
    if (!rc) rc = bup.alloc(sizeof(T) * G);
    if (!rc) rc = ba.alloc(sizeof(T) * G);
    if (!rc) rc = bb.alloc(sizeof(T) * G);
    if (!rc) rc = bku.alloc(sizeof(T) * G);
    if (!rc && comp) rc = blo.alloc(sizeof(T) * G);
    if (!rc && comp) rc = buplo.alloc(sizeof(T) * G);
    if (rc) return rc;
    const int dim = mp->patches[0]->dim;
    int nloc = 1;
    for (int d = 0; d < dim; ++d) nloc *= mp->patches[0]->p + 1;
    if (src_patch >= 0) {
        std::vector<int> gi;
        std::vector<double> gw, dense(G, 0.0);
        mp_point(mp, src_patch, src_s, gi, gw);
        for (size_t k = 0; k < gi.size(); ++k) dense[gi[k]] += gw[k];
        if ((rc = bsrc.alloc(sizeof(double) * G))) return rc;
        IGA_CUDA(cudaMemcpyAsync(bsrc.ptr, dense.data(), sizeof(double) * G, cudaMemcpyHostToDevice, st));
        IGA_CUDA(cudaStreamSynchronize(st));
    }
    if (nrec > 0) {
        std::vector<int> ri((size_t)nrec * nloc);
        std::vector<double> rw((size_t)nrec * nloc);
        for (int r = 0; r < nrec; ++r) {
            std::vector<int> gi;
            std::vector<double> gw;
            mp_point(mp, rec_patch[r], rec_s + (size_t)r * dim, gi, gw);
            std::copy(gi.begin(), gi.end(), ri.begin() + (size_t)r * nloc);
            std::copy(gw.begin(), gw.end(), rw.begin() + (size_t)r * nloc);
        }
        if ((rc = bridx.alloc(sizeof(int) * ri.size())) || (rc = brw.alloc(sizeof(double) * rw.size())) ||
            (rc = btr.alloc(sizeof(double) * (size_t)nrec * nsteps)))
            return rc;
        IGA_CUDA(cudaMemcpyAsync(bridx.ptr, ri.data(), sizeof(int) * ri.size(), cudaMemcpyHostToDevice, st));
        IGA_CUDA(cudaMemcpyAsync(brw.ptr, rw.data(), sizeof(double) * rw.size(), cudaMemcpyHostToDevice, st));
        IGA_CUDA(cudaStreamSynchronize(st));
    }
    T* u = bu.as<T>();
    T* up = bup.as<T>();
    T* ulo = comp ? blo.as<T>() : nullptr;
    T* uplo = comp ? buplo.as<T>() : nullptr;
    IGA_CUDA(cudaMemcpyAsync(u, u_io, sizeof(T) * G, cudaMemcpyDeviceToDevice, st));
    IGA_CUDA(cudaMemsetAsync(ba.ptr, 0, sizeof(T) * G, st));
    if (comp) IGA_CUDA(cudaMemsetAsync(ulo, 0, sizeof(T) * G, st));
    const int grid = (int)std::min<long long>((G + 255) / 256, kMpBlocks);
    *iters_total = 0;
    for (int n = 0; n < nsteps; ++n) {
        MpWork w;
        if ((rc = mp_work(mp, sizeof(T), 1, w))) return rc;
        if ((rc = mp_apply_typed<T>(mp, IGA_OP_K, u, bku.as<T>(), 1, st, w))) return rc;
        mpw_rhs_kernel<T><<<grid, 256, 0, st>>>(bku.as<T>(), src_patch >= 0 ? bsrc.as<double>() : nullptr,
                                               amp * ricker(n * dt, f0, t0), bb.as<T>(), G);
        IGA_LAUNCH_CHECK("mpw_rhs_kernel");
        int it = 0;
        double rel = 0.0;
        // a^n from the multi-patch PCG started at a^{n-1}
        if ((rc = mp_solve_typed<T>(mp, bb.as<T>(), ba.as<T>(), 1, rtol, max_it, &it, &rel, st))) return rc;
        *iters_total += it;
        if constexpr (sizeof(T) == 8) {
            mpw_update_kernel<<<grid, 256, 0, st>>>((const double*)u, (double*)up, (const double*)ba.ptr,
                                                    (n == 0 ? 0.5 : 1.0) * dt * dt, n == 0, G);
        } else {
            mpw_update_kernel<<<grid, 256, 0, st>>>((const float*)u, (const float*)ulo, (float*)up, (float*)uplo,
                                                    (const float*)ba.ptr, (float)((n == 0 ? 0.5 : 1.0) * dt * dt),
                                                    n == 0, G);
        }
        IGA_LAUNCH_CHECK("mpw_update_kernel");
        std::swap(u, up);
        std::swap(ulo, uplo);
        if (nrec > 0) {
            mpw_receiver_kernel<T><<<(nrec + 127) / 128, 128, 0, st>>>(u, ulo, bridx.as<int>(), brw.as<double>(), nrec,
                                                                     nloc, btr.as<double>(), nsteps, n);
            IGA_LAUNCH_CHECK("mpw_receiver_kernel");
        }
    }
    IGA_CUDA(cudaMemcpyAsync(u_io, u, sizeof(T) * G, cudaMemcpyDeviceToDevice, st));
    if (nrec > 0)
        IGA_CUDA(cudaMemcpyAsync(traces_h, btr.ptr, sizeof(double) * (size_t)nrec * nsteps, cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    return IGA_OK;
}

}  // namespace
}  // namespace iga

extern "C" int iga_multipatch_apply(const iga_multipatch* mp, int which, int dtype, const void* x, void* y, int nrhs,
                                    void* stream) {
    if (!mp || !x || !y) return fail(IGA_ERR_ARG, "null argument");
    if (which != IGA_OP_K && which != IGA_OP_M) return fail(IGA_ERR_ARG, "which must be IGA_OP_K or IGA_OP_M");
    if (dtype != IGA_F32 && dtype != IGA_F64) return fail(IGA_ERR_ARG, "dtype must be IGA_F32 or IGA_F64");
    if (nrhs < 0) return fail(IGA_ERR_ARG, "nrhs must be >= 0");
    if (x == y) return fail(IGA_ERR_ARG, "y must not alias x");
    if (nrhs == 0) return IGA_OK;
    MpWork w;
    const size_t es = dtype == IGA_F64 ? 8 : 4;
    int rc = mp_work(mp, es, nrhs, w);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == IGA_F64 ? mp_apply_typed<double>(mp, which, (const double*)x, (double*)y, nrhs, st, w)
                            : mp_apply_typed<float>(mp, which, (const float*)x, (float*)y, nrhs, st, w);
}

extern "C" int iga_multipatch_mass_solve(const iga_multipatch* mp, int dtype, const void* b, void* x, int nrhs,
                                         double rtol, int max_it, int* iters_out, double* relres_out, void* stream) {
    if (!mp || !b || !x) return fail(IGA_ERR_ARG, "null argument");
    if (dtype != IGA_F32 && dtype != IGA_F64) return fail(IGA_ERR_ARG, "dtype must be IGA_F32 or IGA_F64");
    if (nrhs < 0 || max_it < 0 || !(rtol >= 0.0)) return fail(IGA_ERR_ARG, "bad nrhs / max_it / rtol");
    if (b == x) return fail(IGA_ERR_ARG, "x must not alias b");
    if (nrhs == 0) return IGA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == IGA_F64
               ? mp_solve_typed<double>(mp, (const double*)b, (double*)x, nrhs, rtol, max_it, iters_out, relres_out, st)
               : mp_solve_typed<float>(mp, (const float*)b, (float*)x, nrhs, rtol, max_it, iters_out, relres_out, st);
}

extern "C" int iga_multipatch_leapfrog(const iga_multipatch* mp, int dtype, double dt, int nsteps, void* u,
                                       int src_patch, const double* src_s, double f0, double t0, double amp,
                                       int nrec, const int* rec_patch, const double* rec_s, double* traces,
                                       double cg_rtol, int cg_max_it, long long* cg_iters_out, void* stream) {
    if (!mp || !u) return fail(IGA_ERR_ARG, "null argument");
    if (dtype != IGA_F32 && dtype != IGA_F64) return fail(IGA_ERR_ARG, "dtype must be IGA_F32 or IGA_F64");
    if (!(dt > 0.0) || nsteps < 1 || cg_max_it < 1 || !(cg_rtol >= 0.0))
        return fail(IGA_ERR_ARG, "bad dt / nsteps / cg_max_it / cg_rtol");
    const int npatch = (int)mp->patches.size();
    if (src_patch >= npatch || (src_patch >= 0 && !src_s)) return fail(IGA_ERR_ARG, "bad source");
    if (nrec < 0 || (nrec > 0 && (!rec_patch || !rec_s || !traces))) return fail(IGA_ERR_ARG, "bad receivers");
    for (int r = 0; r < nrec; ++r)
        if (rec_patch[r] < 0 || rec_patch[r] >= npatch) return fail(IGA_ERR_ARG, "receiver patch does not exist");
    if (mp->G > (1LL << 31) - 1) return fail(IGA_ERR_ARG, "too many global functions");
    long long iters = 0;
    cudaStream_t st = (cudaStream_t)stream;
    const int rc = dtype == IGA_F64
                       ? mp_leapfrog_typed<double>(mp, dt, nsteps, (double*)u, src_patch, src_s, f0, t0, amp, nrec,
                                                   rec_patch, rec_s, traces, cg_rtol, cg_max_it, &iters, st)
                       : mp_leapfrog_typed<float>(mp, dt, nsteps, (float*)u, src_patch, src_s, f0, t0, amp, nrec,
                                                  rec_patch, rec_s, traces, cg_rtol, cg_max_it, &iters, st);
    if (cg_iters_out) *cg_iters_out = iters;
    return rc;
}
