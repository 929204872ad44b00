// On-the-fly evaluation of the surrogate stencil functions inside the operator
// apply (Sec. 3.3, last paragraph: in a matrix-free method the stencil-function
// data is read during every matrix-vector product; here the data read is the
// B-spline interpolation coefficients of Sec. 3.3 instead of evaluated fields).
//
// Rows whose whole stencil lies in the surrogate region (i and every neighbour
// i +- delta in Omega~, i.e. every interior index in [lo + p, lo + L - 1 - p]) need
// no stored entry: K~(i, i + delta) = K~_delta(x~_i) and the mirrored
// K~(i, i - delta) = K~_delta(x~_{i - delta}) (Eq. DefinitionOfSurrogateMatrixSymmetric
// / ..SymmetricKernel).  Each apply first contracts the coefficients over
// directions 1..d-1 at every interior line,
//     G_u[line][a] = sum_{b (,c)} C_u[a, span_1 + b (, span_2 + c)] beta_b (beta_c),
// then evaluates
//     K~_u(x~_i) = sum_a G_u[line(i)][span_0(i_0) + a] beta_a(i_0)
// with q + 1 FMAs per entry.  Arithmetic is in the apply's precision (FP32 tables
// for the FP32 apply: an FP64 contraction would cost more than the field stream
// it saves on this part).  Every other row (the boundary band and the rows next
// to it) is applied from the stored fields, as in the row kernels.  The M~
// diagonal always comes from the stored field 0, so the volume-preserving mass
// (whose diagonal is not a stencil-function value) is applied unchanged.
#include <algorithm>
#include <memory>
#include <vector>

#include "iga_internal.cuh"
#include "stencil.cuh"

namespace iga {

// G[u][line][a] for u < nf (offsets t = t0 + 1 + u), lines over the interior indices of
// directions 1..d-1 (colex), a over the ns coefficients of direction 0.
template <int DIM, typename T>
__global__ void otf_lines_kernel(const double* __restrict__ C, int t_first, int nf, long long nsd,
                                 const int* __restrict__ espan, const double* __restrict__ evals, int q, int ns,
                                 int L, long long lines, T* __restrict__ G) {
    const long long total = (long long)nf * lines * ns;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int a0 = (int)(idx % ns);
        const long long line = (idx / ns) % lines;
        const int u = (int)(idx / ((long long)ns * lines));
        const double* c = C + (size_t)(t_first + u) * nsd;
        T acc = T(0);
        if (DIM == 2) {
            const int l1 = (int)line;
            const double* e1 = evals + (size_t)l1 * (q + 1);
            for (int b = 0; b <= q; ++b) acc += (T)c[a0 + (long long)ns * (espan[l1] + b)] * (T)e1[b];
        } else {
            const int l1 = (int)(line % L), l2 = (int)(line / L);
            const double* e1 = evals + (size_t)l1 * (q + 1);
            const double* e2 = evals + (size_t)l2 * (q + 1);
            for (int cc = 0; cc <= q; ++cc) {
                T s = T(0);
                const long long o2 = (long long)ns * ns * (espan[l2] + cc);
                for (int b = 0; b <= q; ++b) s += (T)c[a0 + (long long)ns * (espan[l1] + b) + o2] * (T)e1[b];
                acc += s * (T)e2[cc];
            }
        }
        G[idx] = acc;
    }
}

// y = A x (one right-hand side): on-the-fly rows from G, the rest from the fields.
template <int DIM, int P, typename T, bool MASS>
__global__ void __launch_bounds__(256) otf_apply_kernel(const T* __restrict__ F, long long pitch,
                                                         const T* __restrict__ G, long long lines,
                                                         const int* __restrict__ espan,
                                                         const T* __restrict__ evals, int q, int ns, int L, int lo,
                                                         const T* __restrict__ x, T* __restrict__ y, int N, int m) {
    constexpr int NF = StencilShape<DIM, P>::T0, PP = 2 * P + 1;
    __shared__ int sdl[NF];
    fill_delta_table<DIM, P>(sdl, m);
    const LdgLoad<T> ld{x, N};
    const int dlo = lo + P, dhi = lo + L - 1 - P;   // rows whose whole stencil is surrogate
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int ik[3] = {i % m, (i / m) % m, DIM == 3 ? i / (m * m) : 0};
        bool deep = true;
#pragma unroll
        for (int k = 0; k < DIM; ++k) deep = deep && ik[k] >= dlo && ik[k] <= dhi;
        T acc[1], own[1];
        if (!deep) {
            stencil_row<DIM, P, T, MASS, 1, 4>(F, pitch, ld, i, N, m, acc, own);
            y[i] = acc[0];
            continue;
        }
        const int l0 = ik[0] - lo, l1 = ik[1] - lo, l2 = ik[2] - lo;
        const T xi = __ldg(x + i);
        T a = MASS ? __ldg(F + i) * xi : T(0);
        const long long line = DIM == 3 ? (long long)l1 + (long long)L * l2 : l1;
        // basis values and first coefficient of the indices l0 - P .. l0 + P (direction 0)
        constexpr int QM = 4;   // q <= 3
        T ev[PP][QM];
        int sp[PP];
#pragma unroll
        for (int d = 0; d < PP; ++d) {
            const int l = l0 - P + d;
            sp[d] = espan[l];
#pragma unroll
            for (int b = 0; b < QM; ++b) ev[d][b] = b <= q ? __ldg(evals + (size_t)l * (q + 1) + b) : T(0);
        }
#pragma unroll
        for (int u = 0; u < NF; ++u) {
            const int t = NF + 1 + u;
            const int d0 = t % PP - P, d1 = (t / PP) % PP - P, d2 = DIM == 3 ? t / (PP * PP) - P : 0;
            const int dl = sdl[u];
            // own entry at x~_i, mirrored entry at x~_{i - delta}
            const T* go = G + ((size_t)u * lines + line) * ns + sp[P];
            const long long linem = DIM == 3 ? (long long)(l1 - d1) + (long long)L * (l2 - d2) : (l1 - d1);
            const T* gm = G + ((size_t)u * lines + linem) * ns + sp[P - d0];
            T so = T(0), sm = T(0);
#pragma unroll
            for (int b = 0; b < QM; ++b)
                if (b <= q) {
                    so = fma(__ldg(go + b), ev[P][b], so);
                    sm = fma(__ldg(gm + b), ev[P - d0][b], sm);
                }
            const T xp = __ldg(x + i + dl), xm = __ldg(x + i - dl);
            if (MASS) {
                a = fma(so, xp, a);
                a = fma(sm, xm, a);
            } else {
                a = fma(so, xp - xi, a);
                a = fma(sm, xm - xi, a);
            }
        }
        y[i] = a;
    }
}

template <int DIM, int P, typename T>
static int otf_typed(const iga_ops* ops, int which, const T* x, T* y, int nrhs, cudaStream_t st) {
    const OtfOps& o = *ops->otf;
    const bool mass = which == IGA_OP_M;
    const bool f64 = sizeof(T) == 8;
    T* G = (T*)(mass ? (f64 ? o.gM64.ptr : o.gM32.ptr) : (f64 ? o.gK64.ptr : o.gK32.ptr));
    const T* F = (const T*)(mass ? (f64 ? ops->fM64.ptr : ops->fM32.ptr) : (f64 ? ops->fK64.ptr : ops->fK32.ptr));
    const T* ev = f64 ? (const T*)ops->evals.ptr : (const T*)o.evals32.ptr;
    const double* C = mass ? ops->cM.as<double>() : ops->cK.as<double>();
    long long nsd = 1;
    for (int k = 0; k < DIM; ++k) nsd *= o.ns;
    const int N = (int)ops->N;
    const int t0 = (ops->D - 1) / 2;
    for (int r = 0; r < nrhs; ++r) {
        const long long tot = (long long)o.nf * o.lines * o.ns;
        const int g1 = (int)std::max<long long>(1, std::min<long long>((tot + 255) / 256, 152 * 16));
        otf_lines_kernel<DIM, T><<<g1, 256, 0, st>>>(C, t0 + 1, o.nf, nsd, ops->espan.as<int>(),
                                                     ops->evals.as<double>(), o.q, o.ns, o.L, o.lines, G);
        IGA_LAUNCH_CHECK("otf_lines_kernel");
        const int g2 = (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, 152 * 16));
        if (mass)
            otf_apply_kernel<DIM, P, T, true><<<g2, 256, 0, st>>>(F, ops->pitch, G, o.lines, ops->espan.as<int>(), ev,
                                                                 o.q, o.ns, o.L, o.lo, x + (size_t)r * N,
                                                                 y + (size_t)r * N, N, ops->m);
        else
            otf_apply_kernel<DIM, P, T, false><<<g2, 256, 0, st>>>(F, ops->pitch, G, o.lines, ops->espan.as<int>(),
                                                                  ev, o.q, o.ns, o.L, o.lo, x + (size_t)r * N,
                                                                  y + (size_t)r * N, N, ops->m);
        IGA_LAUNCH_CHECK("otf_apply_kernel");
    }
    return IGA_OK;
}

template <typename T>
static int otf_dispatch(const iga_ops* ops, int which, const T* x, T* y, int nrhs, cudaStream_t st) {
    const int d = ops->dim, p = ops->p;
    if (d == 2 && p == 1) return otf_typed<2, 1, T>(ops, which, x, y, nrhs, st);
    if (d == 2 && p == 2) return otf_typed<2, 2, T>(ops, which, x, y, nrhs, st);
    if (d == 2 && p == 3) return otf_typed<2, 3, T>(ops, which, x, y, nrhs, st);
    if (d == 3 && p == 1) return otf_typed<3, 1, T>(ops, which, x, y, nrhs, st);
    if (d == 3 && p == 2) return otf_typed<3, 2, T>(ops, which, x, y, nrhs, st);
    return fail(IGA_ERR_ARG, "unsupported (dim, p) for the on-the-fly apply");
}

int onthefly_apply(const iga_ops* ops, int which, int dtype, const void* x, void* y, int nrhs, cudaStream_t st) {
    if (!ops->otf) return fail(IGA_ERR_ARG, "on-the-fly tables missing (iga_ops_set_path(IGA_PATH_ONTHEFLY))");
    if (dtype == IGA_F64) return otf_dispatch<double>(ops, which, (const double*)x, (double*)y, nrhs, st);
    return otf_dispatch<float>(ops, which, (const float*)x, (float*)y, nrhs, st);
}

// Tables of the on-the-fly apply (synchronous; allocates G for both operators and
// both precisions).  Needs a surrogate ops (not IGA_TRUE_ONLY).
int onthefly_prepare(iga_ops* ops) {
    if (ops->otf) return IGA_OK;
    if (!ops->cK.ptr || !ops->cM.ptr || !ops->espan.ptr || !ops->evals.ptr)
        return fail(IGA_ERR_ARG, "the on-the-fly apply needs a surrogate ops (not IGA_TRUE_ONLY)");
    std::unique_ptr<OtfOps> o(new (std::nothrow) OtfOps());
    if (!o) return fail(IGA_ERR_OOM, "host allocation failed");
    o->L = ops->m - 4 * ops->p;
    o->lo = 2 * ops->p;
    o->ns = ops->ns;
    o->q = ops->q;
    o->nf = (ops->D - 1) / 2;
    o->lines = 1;
    for (int k = 1; k < ops->dim; ++k) o->lines *= o->L;
    if (o->L < 2 * ops->p + 1) return fail(IGA_ERR_ARG, "mesh too small: no row has a surrogate-only stencil");
    const size_t n = (size_t)o->nf * o->lines * o->ns;
    int rc = o->gK64.alloc(n * 8);
    if (!rc) rc = o->gM64.alloc(n * 8);
    if (!rc) rc = o->gK32.alloc(n * 4);
    if (!rc) rc = o->gM32.alloc(n * 4);
    const size_t ne = ops->evals.bytes / sizeof(double);
    if (!rc) rc = o->evals32.alloc(ne * sizeof(float));
    if (rc) return rc;
    std::vector<double> e(ne);
    std::vector<float> e32(ne);
    IGA_CUDA(cudaMemcpy(e.data(), ops->evals.ptr, ne * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < ne; ++k) e32[k] = (float)e[k];
    IGA_CUDA(cudaMemcpy(o->evals32.ptr, e32.data(), ne * sizeof(float), cudaMemcpyHostToDevice));
    ops->otf = std::move(o);
    return IGA_OK;
}

}  // namespace iga
