// Surrogate assembly on the GPU (FP64 arithmetic throughout).
//
//  a2  sample_rows_kernel  : true rows M_delta(x~_s), K_delta(x~_s) at every sample
//                            row (Eq. StencilRoughDefinition), by Gauss quadrature
//                            over the (p+1)^d elements of supp(phi_s).
//  a3  band_kernel         : true entries of every pair (i, j) with i or j outside
//                            Omega~, by element quadrature of the boundary band,
//                            written straight into the field slots.  Elements are
//                            launched in (p+1)^d colours (e_k mod (p+1)), so no two
//                            concurrent elements share a basis function and the
//                            read-modify-write of a slot needs no atomics
//                            (deterministic).
//  a4  interp_dir_kernel   : B-spline interpolation coefficients of every stencil
//                            function (Sec. 3.3), one direction at a time with the
//                            precomputed inverse of the 1-D collocation matrix.
//  a5  eval_dir_kernel,    : surrogate values K~_delta(x~_i), M~_delta(x~_i) at every
//      eval_last_kernel      interior row whose neighbour i+delta is interior
//                            (Eq. DefinitionOfSurrogateMatrixSymmetric / ..Kernel),
//                            the tensor-product interpolant contracted one direction
//                            at a time over the grid of interior rows.
//      finalize_kernel     : FP32 copies of the fields, inverse Jacobi diagonal of
//                            M~, non-finite check.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "geom.cuh"
#include "quad.cuh"
#include "dfloat.cuh"
#include "stencil.cuh"
#include "host_bspline.h"
#include "iga_internal.cuh"

namespace iga {

// ---------------------------------------------------------------- a3: band elements
// Geometry, coefficient and the pulled-back weights at every Gauss point in FP64;
// the basis products, G grad phi and the element contractions in double-float
// pairs (dfloat.cuh: about 48 significant bits, on the FP32 pipe).  An entry is
// the FP64 sum hi + lo of its pair.
template <int DIM, int P>
__global__ void band_kernel(GeomParams gp, const int* __restrict__ elems, double* __restrict__ fK,
                            double* __restrict__ fM, long long pitch, int lo, int hi, int all_true,
                            int* status) {
    using S = Stencil<DIM, P>;
    extern __shared__ double sm[];
    const int nq = gp.nq;
    int nqd = nq;
#pragma unroll
    for (int k = 1; k < DIM; ++k) nqd *= nq;
    f2* Gq = reinterpret_cast<f2*>(sm);   // [nqd][NS]
    f2* wq = Gq + nqd * S::NS;            // [nqd]
    f2* grad = wq + nqd;                  // [NLOC][nqd][DIM]
    f2* Ggrad = grad + S::NLOC * nqd * DIM;
    f2* val = Ggrad + S::NLOC * nqd * DIM;   // [NLOC][nqd]
    f2* vw = val + S::NLOC * nqd;            // [NLOC][nqd]
    const f2* bv2 = reinterpret_cast<const f2*>(gp.bval2);
    const f2* bd2 = reinterpret_cast<const f2*>(gp.bder2);

    int e[3] = {0, 0, 0};
    decode<DIM>(elems[blockIdx.x], gp.n_el, e);
    for (int q = threadIdx.x; q < nqd; q += blockDim.x) {
        int g[3] = {0, 0, 0};
        decode<DIM>(q, nq, g);
        double G[6], wm;
        const double det = qp_weights(gp, e, g, G, wm);
        if (!(det > 0.0)) atomicOr(status, 2);
#pragma unroll
        for (int k = 0; k < S::NS; ++k) Gq[q * S::NS + k] = df_from(G[k]);
        wq[q] = df_from(wm);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < S::NLOC * nqd; idx += blockDim.x) {
        const int a = idx / nqd, q = idx % nqd;
        int g[3] = {0, 0, 0}, al[3] = {0, 0, 0};
        decode<DIM>(q, nq, g);
        decode<DIM>(a, P + 1, al);
        f2 v[DIM], dv[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int t = (e[k] * nq + g[k]) * (P + 1) + al[k];
            v[k] = bv2[t];
            dv[k] = bd2[t];
        }
        f2 vv = v[0], gr[DIM];
#pragma unroll
        for (int k = 1; k < DIM; ++k) vv = df_mul(vv, v[k]);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            f2 gk = k == 0 ? dv[0] : v[0];
#pragma unroll
            for (int j = 1; j < DIM; ++j) gk = df_mul(gk, j == k ? dv[j] : v[j]);
            gr[k] = gk;
        }
        // G grad phi with G packed symmetric
        const f2* Gp = Gq + q * S::NS;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            f2 acc = {0.f, 0.f};
#pragma unroll
            for (int l = 0; l < DIM; ++l) df_mac(acc, Gp[sym_index(DIM, k, l)], gr[l]);
            Ggrad[(a * nqd + q) * DIM + k] = acc;
            grad[(a * nqd + q) * DIM + k] = gr[k];
        }
        val[a * nqd + q] = vv;
        vw[a * nqd + q] = df_mul(vv, wq[q]);
    }
    __syncthreads();
    const int m = gp.m;
    for (int pidx = threadIdx.x; pidx < S::NLOC * S::NLOC; pidx += blockDim.x) {
        const int a = pidx / S::NLOC, b = pidx % S::NLOC;
        int al[3] = {0, 0, 0}, bl[3] = {0, 0, 0};
        decode<DIM>(a, P + 1, al);
        decode<DIM>(b, P + 1, bl);
        int t = 0, i[3] = {0, 0, 0}, j[3] = {0, 0, 0};
        for (int k = DIM - 1; k >= 0; --k) t = t * S::PP + (bl[k] - al[k] + P);
        if (t < S::T0) continue;                       // lower triangle: stored at the other row
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            i[k] = e[k] + al[k];
            j[k] = e[k] + bl[k];
        }
        if (!all_true && in_range<DIM>(i, lo, hi) && in_range<DIM>(j, lo, hi)) continue;  // surrogate slot
        long long li = 0;
        for (int k = DIM - 1; k >= 0; --k) li = li * m + i[k];
        f2 kv = {0.f, 0.f}, mv = {0.f, 0.f};
        for (int q = 0; q < nqd; ++q) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) df_mac(kv, Ggrad[(a * nqd + q) * DIM + k], grad[(b * nqd + q) * DIM + k]);
            df_mac(mv, vw[a * nqd + q], val[b * nqd + q]);
        }
        if (t > S::T0) fK[(size_t)(t - S::T0 - 1) * pitch + li] += df_value(kv);
        fM[(size_t)(t - S::T0) * pitch + li] += df_value(mv);
    }
}

// ---------------------------------------------------------------- a2: sample rows
// Per support element of the sample row: geometry, coefficient, weights and
// G grad phi_a in FP64 at the Gauss points; the basis of every other local function
// and the contraction over the points in double-float pairs (dfloat.cuh).
template <int DIM, int P>
__global__ void sample_rows_kernel(GeomParams gp, const int* __restrict__ samp, int ns,
                                   double* __restrict__ sK, double* __restrict__ sM, int* status) {
    using S = Stencil<DIM, P>;
    extern __shared__ double sm[];
    const int nq = gp.nq;
    int nqd = nq;
#pragma unroll
    for (int k = 1; k < DIM; ++k) nqd *= nq;
    double* accK = sm;                        // [DD]
    double* accM = accK + S::DD;              // [DD]
    double* Gq = accM + S::DD;                // [nqd][NS]
    double* wq = Gq + nqd * S::NS;            // [nqd]
    f2* Ga = reinterpret_cast<f2*>(wq + nqd);   // [nqd][DIM]   G grad phi_a
    f2* va = Ga + nqd * DIM;                    // [nqd]        phi_a wm
    const f2* bv2 = reinterpret_cast<const f2*>(gp.bval2);
    const f2* bd2 = reinterpret_cast<const f2*>(gp.bder2);

    int sidx[3] = {0, 0, 0}, row[3] = {0, 0, 0};
    decode<DIM>(blockIdx.x, ns, sidx);
#pragma unroll
    for (int k = 0; k < DIM; ++k) row[k] = samp[sidx[k]];
    for (int t = threadIdx.x; t < S::DD; t += blockDim.x) accK[t] = accM[t] = 0.0;

    for (int a = 0; a < S::NLOC; ++a) {
        int al[3] = {0, 0, 0}, e[3] = {0, 0, 0};
        decode<DIM>(a, P + 1, al);
#pragma unroll
        for (int k = 0; k < DIM; ++k) e[k] = row[k] - al[k];   // element with local function a = row
        __syncthreads();
        for (int q = threadIdx.x; q < nqd; q += blockDim.x) {
            int g[3] = {0, 0, 0};
            decode<DIM>(q, nq, g);
            double G[6], wm;
            const double det = qp_weights(gp, e, g, G, wm);
            if (!(det > 0.0)) atomicOr(status, 2);
            double gr[DIM], v, Gg[DIM];
            local_basis<DIM, P>(gp, e, g, al, gr, v);
            sym_matvec<DIM>(G, gr, Gg);
#pragma unroll
            for (int k = 0; k < DIM; ++k) Ga[q * DIM + k] = df_from(Gg[k]);
            va[q] = df_from(v * wm);
        }
        __syncthreads();
        for (int b = threadIdx.x; b < S::NLOC; b += blockDim.x) {
            int bl[3] = {0, 0, 0};
            decode<DIM>(b, P + 1, bl);
            f2 kv = {0.f, 0.f}, mv = {0.f, 0.f};
            for (int q = 0; q < nqd; ++q) {
                int g[3] = {0, 0, 0};
                decode<DIM>(q, nq, g);
                f2 v[DIM], dv[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    const int ti = (e[k] * nq + g[k]) * (P + 1) + bl[k];
                    v[k] = bv2[ti];
                    dv[k] = bd2[ti];
                }
                f2 vv = v[0];
#pragma unroll
                for (int k = 1; k < DIM; ++k) vv = df_mul(vv, v[k]);
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    f2 gk = k == 0 ? dv[0] : v[0];
#pragma unroll
                    for (int j = 1; j < DIM; ++j) gk = df_mul(gk, j == k ? dv[j] : v[j]);
                    df_mac(kv, Ga[q * DIM + k], gk);
                }
                df_mac(mv, va[q], vv);
            }
            int t = 0;
            for (int k = DIM - 1; k >= 0; --k) t = t * S::PP + (bl[k] - al[k] + P);
            accK[t] += df_value(kv);   // distinct t for distinct b within one element
            accM[t] += df_value(mv);
        }
    }
    __syncthreads();
    int nsd = ns;
#pragma unroll
    for (int k = 1; k < DIM; ++k) nsd *= ns;
    for (int t = threadIdx.x; t < S::DD; t += blockDim.x) {
        sK[(size_t)t * nsd + blockIdx.x] = accK[t];
        sM[(size_t)t * nsd + blockIdx.x] = accM[t];
    }
}

// ---------------------------------------------------------------- a4: interpolation
// out[t][c] = sum_j Ainv[c_dir][j] in[t][c with c_dir -> j], for all D stencil functions
__global__ void interp_dir_kernel(const double* __restrict__ in, double* __restrict__ out,
                                  const double* __restrict__ Ainv, int ns, int dim, int dir, int D) {
    int nsd = 1;
    for (int k = 0; k < dim; ++k) nsd *= ns;
    const long long total = (long long)D * nsd;
    int stride_dir = 1;
    for (int k = 0; k < dir; ++k) stride_dir *= ns;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(idx / nsd);
        const int c = (int)(idx % nsd);
        const int cd = (c / stride_dir) % ns;
        const int base = c - cd * stride_dir;
        const double* src = in + (size_t)t * nsd + base;
        double acc = 0.0;
        for (int j = 0; j < ns; ++j) acc += Ainv[cd * ns + j] * src[(size_t)j * stride_dir];
        out[idx] = acc;
    }
}

// ---------------------------------------------------------------- a5: sum-factorised evaluation
// The surrogate value at interior row l = (l_0, .., l_{d-1}) is the tensor B-spline
// sum_{a} C[espan(l_k) + a_k]_k prod_k evals[l_k][a_k].  Every row of Omega~ is a
// tensor-grid point, so the sum is contracted one direction at a time over the whole
// grid: direction k turns the coefficient index (extent ns) into the row index
// (extent L), (q+1) FMAs per output value.  In 3-D this is ns^2 L + ns L^2 + L^3 values
// per field ((q+1) FMAs each) instead of L^3 ((q+1)^3 + (q+1)^2 + (q+1)) row by row:
// about 11x fewer FP64 FMAs at ns = 16, L = 90, q = 2.
//
// eval_dir_kernel: directions 0..d-2.  Tensor layout colex (direction 0 fastest),
// extents L for directions < dir, ns for directions >= dir on input; output has
// extent L in direction dir too.  Fields are contiguous blocks of in_stride / out
// values.
__global__ void eval_dir_kernel(const double* __restrict__ in, long long in_stride, double* __restrict__ out,
                                long long out_per_field, int nf, const int* __restrict__ espan,
                                const double* __restrict__ evals, int q, int ns, int L, int dim, int dir) {
    const long long total = (long long)nf * out_per_field;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(idx / out_per_field);
        long long r = idx % out_per_field;
        long long in_off = 0, in_mul = 1;
        int l = 0;
        long long dir_mul = 1;
        for (int k = 0; k < dim; ++k) {
            const int ext_out = k <= dir ? L : ns;
            const int ext_in = k < dir ? L : ns;
            const int ik = (int)(r % ext_out);
            r /= ext_out;
            if (k == dir) {
                l = ik;
                dir_mul = in_mul;
            } else {
                in_off += ik * in_mul;
            }
            in_mul *= ext_in;
        }
        const double* src = in + (size_t)f * in_stride + in_off + (long long)espan[l] * dir_mul;
        const double* e = evals + (size_t)l * (q + 1);
        double acc = 0.0;
        for (int a = 0; a <= q; ++a) acc += src[(long long)a * dir_mul] * e[a];
        out[idx] = acc;
    }
}

// Last direction (d-1) straight into the field slots: K~_delta(x~_i) / M~_delta(x~_i)
// at every interior row whose neighbour i + delta is interior (the other slots hold
// the band's true entries).  Input extents: L in directions < d-1, ns in d-1.
template <int DIM>
__global__ void eval_last_kernel(const double* __restrict__ in, long long in_stride, int nf, int t_first,
                                 int field_base, const int* __restrict__ espan, const double* __restrict__ evals,
                                 int q, int ns, int L, int lo, int m, int p, double* __restrict__ fields,
                                 long long pitch) {
    long long Ld = L;
    for (int k = 1; k < DIM; ++k) Ld *= L;
    const long long total = (long long)nf * Ld;
    const int PP = 2 * p + 1;
    const long long plane = Ld / L;   // L^{d-1}: stride of direction d-1 in the input
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(idx / Ld);
        const long long r = idx % Ld;
        const int t = t_first + f;
        int l[3] = {0, 0, 0};
        {
            long long rr = r;
            for (int k = 0; k < DIM; ++k) {
                l[k] = (int)(rr % L);
                rr /= L;
            }
        }
        bool ok = true;
        {
            int tt = t;
            for (int k = 0; k < DIM; ++k) {
                const int j = l[k] + (tt % PP - p);
                tt /= PP;
                ok = ok && j >= 0 && j < L;
            }
        }
        if (!ok) continue;   // neighbour outside Omega~: true entry from the band
        const int ll = l[DIM - 1];
        const long long low = r - (long long)ll * plane;   // index of the lower directions
        const double* src = in + (size_t)f * in_stride + low + (long long)espan[ll] * plane;
        const double* e = evals + (size_t)ll * (q + 1);
        double acc = 0.0;
        for (int a = 0; a <= q; ++a) acc += src[(long long)a * plane] * e[a];
        long long li = 0;
        for (int k = DIM - 1; k >= 0; --k) li = li * m + (lo + l[k]);
        fields[(size_t)(t - field_base) * pitch + li] = acc;
    }
}


// ---------------------------------------------------------------- volume-preserving mass
// Sec. 3.4 (remark on volume preservation): M~ = D + M~_0 with D_ii = int phi_i
// det J and M~_0 built like K~ from the mass stencil functions, i.e. the
// off-diagonal entries of M~ are kept and the diagonal becomes
// D_ii - sum_{j != i} [M~]_ij.
//
// lumped_elem_kernel: per element, the integrals of its (p+1)^d local functions,
// ve[a][e] (one thread per element, Gauss points in colex order).
template <int DIM, int P>
__global__ void lumped_elem_kernel(GeomParams gp, double* __restrict__ ve, int nE, int* status) {
    constexpr int NL = DIM == 2 ? (P + 1) * (P + 1) : (P + 1) * (P + 1) * (P + 1);
    const int nq = gp.nq;
    int nqd = nq;
#pragma unroll
    for (int k = 1; k < DIM; ++k) nqd *= nq;
    for (int el = blockIdx.x * blockDim.x + threadIdx.x; el < nE; el += gridDim.x * blockDim.x) {
        int e[3] = {0, 0, 0};
        decode<DIM>(el, gp.n_el, e);
        double acc[NL];
#pragma unroll
        for (int a = 0; a < NL; ++a) acc[a] = 0.0;
        for (int q = 0; q < nqd; ++q) {
            int g[3] = {0, 0, 0};
            decode<DIM>(q, nq, g);
            const double wm = qp_volume(gp, e, g);
            if (!(wm > 0.0)) atomicOr(status, 2);
            double b[DIM][P + 1];
#pragma unroll
            for (int k = 0; k < DIM; ++k)
#pragma unroll
                for (int a = 0; a <= P; ++a) b[k][a] = gp.bval[(e[k] * nq + g[k]) * (P + 1) + a];
#pragma unroll
            for (int a = 0; a < NL; ++a) {
                int al[3] = {0, 0, 0};
                decode<DIM>(a, P + 1, al);
                double v = wm;
#pragma unroll
                for (int k = 0; k < DIM; ++k) v *= b[k][al[k]];
                acc[a] += v;
            }
        }
#pragma unroll
        for (int a = 0; a < NL; ++a) ve[(size_t)a * nE + el] = acc[a];
    }
}

// vp_diag_kernel: D_i = sum over the elements of supp(phi_i) (local index a,
// colex, fixed order) of ve[a][i - a]; then field 0 of M~ = D_i minus the
// off-diagonal row sum sum_u F_u[i] + F_u[i - Delta_u] (entries leaving the grid
// are stored as 0).
template <int DIM, int P>
__global__ void vp_diag_kernel(const double* __restrict__ ve, int n_el, int m, long long N, double* fM,
                               long long pitch) {
    constexpr int NL = DIM == 2 ? (P + 1) * (P + 1) : (P + 1) * (P + 1) * (P + 1);
    constexpr int NF = StencilShape<DIM, P>::T0;
    long long nE = n_el;
    for (int k = 1; k < DIM; ++k) nE *= n_el;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int ii[3] = {0, 0, 0};
        long long r = i;
        for (int k = 0; k < DIM; ++k) {
            ii[k] = (int)(r % m);
            r /= m;
        }
        double d = 0.0;
#pragma unroll
        for (int a = 0; a < NL; ++a) {
            int al[3] = {0, 0, 0};
            decode<DIM>(a, P + 1, al);
            bool ok = true;
            long long el = 0;
            for (int k = DIM - 1; k >= 0; --k) {
                const int ek = ii[k] - al[k];
                ok = ok && ek >= 0 && ek < n_el;
                el = el * n_el + ek;
            }
            if (ok) d += ve[(size_t)a * nE + el];
        }
        double off = 0.0;
        for (int u = 0; u < NF; ++u) {
            const long long dl = field_delta<DIM, P>(u, m);
            const double* F = fM + (size_t)(u + 1) * pitch;
            off += F[i];
            if (i - dl >= 0) off += F[i - dl];
        }
        fM[i] = d - off;
    }
}

// ---------------------------------------------------------------- finalize
__global__ void finalize_kernel(const double* __restrict__ fK, const double* __restrict__ fM, float* fK32,
                                float* fM32, double* dinv64, float* dinv32, int nK, int nM, long long N,
                                long long pitch, int* status) {
    const long long total_k = (long long)nK * pitch, total_m = (long long)nM * pitch;
    int bad = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total_k + total_m;
         idx += (long long)gridDim.x * blockDim.x) {
        const double v = idx < total_k ? fK[idx] : fM[idx - total_k];
        if (!isfinite(v)) bad = 1;
        if (idx < total_k) fK32[idx] = (float)v;
        else fM32[idx - total_k] = (float)v;
        if (idx >= total_k && idx - total_k < N) {
            const double di = 1.0 / v;   // field 0 of M~ is the diagonal
            dinv64[idx - total_k] = di;
            dinv32[idx - total_k] = (float)di;
            if (!(v > 0.0)) bad = 1;
        }
    }
    if (bad) atomicOr(status, 1);
}

// ---------------------------------------------------------------- host side
template <int DIM, int P>
static int launch_band(const iga_space* s, const int* d_elems, int count, iga_ops* ops, int all_true,
                       cudaStream_t st) {
    using S = Stencil<DIM, P>;
    int nqd = 1;
    for (int k = 0; k < DIM; ++k) nqd *= s->nq;
    const size_t smem = sizeof(double) * (nqd * (S::NS + 1) + S::NLOC * nqd * (2 * DIM + 2));
    if (smem > 200 * 1024) return fail(IGA_ERR_ARG, "band quadrature tables exceed shared memory");
    static bool attr_set = false;
    if (!attr_set) {
        IGA_CUDA(cudaFuncSetAttribute(band_kernel<DIM, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        attr_set = true;
    }
    band_kernel<DIM, P><<<count, 128, smem, st>>>(s->gp, d_elems, ops->fK64.as<double>(),
                                                  ops->fM64.as<double>(), ops->pitch, 2 * P, s->m - 2 * P - 1,
                                                  all_true, ops->status.as<int>());
    IGA_LAUNCH_CHECK("band_kernel");
    return IGA_OK;
}

template <int DIM, int P>
static int launch_samples(const iga_space* s, const int* d_samp, iga_ops* ops, cudaStream_t st) {
    using S = Stencil<DIM, P>;
    int nqd = 1, nsd = 1;
    for (int k = 0; k < DIM; ++k) {
        nqd *= s->nq;
        nsd *= ops->ns;
    }
    const size_t smem = sizeof(double) * (2 * S::DD + nqd * (S::NS + 1) + nqd * (DIM + 1));
    sample_rows_kernel<DIM, P><<<nsd, 64, smem, st>>>(s->gp, d_samp, ops->ns, ops->sK.as<double>(),
                                                       ops->sM.as<double>(), ops->status.as<int>());
    IGA_LAUNCH_CHECK("sample_rows_kernel");
    return IGA_OK;
}

template <int DIM, int P>
static int launch_volume_preserving(const iga_space* s, iga_ops* ops, cudaStream_t st) {
    constexpr int NL = DIM == 2 ? (P + 1) * (P + 1) : (P + 1) * (P + 1) * (P + 1);
    long long nE = 1;
    for (int k = 0; k < DIM; ++k) nE *= s->n_el;
    DevBuf ve;
    int rc = ve.alloc(sizeof(double) * NL * nE);
    if (rc) return rc;
    const int ge = (int)std::min<long long>((nE + 127) / 128, 152 * 32);
    lumped_elem_kernel<DIM, P><<<ge, 128, 0, st>>>(s->gp, ve.as<double>(), (int)nE, ops->status.as<int>());
    IGA_LAUNCH_CHECK("lumped_elem_kernel");
    const int gr = (int)std::min<long long>((ops->N + 255) / 256, 152 * 16);
    vp_diag_kernel<DIM, P><<<gr, 256, 0, st>>>(ve.as<double>(), s->n_el, s->m, ops->N, ops->fM64.as<double>(),
                                               ops->pitch);
    IGA_LAUNCH_CHECK("vp_diag_kernel");
    // ve is released when this returns: wait for the kernels that read it
    IGA_CUDA(cudaStreamSynchronize(st));
    return IGA_OK;
}

typedef int (*band_fn)(const iga_space*, const int*, int, iga_ops*, int, cudaStream_t);
typedef int (*samp_fn)(const iga_space*, const int*, iga_ops*, cudaStream_t);

static band_fn pick_band(int dim, int p) {
    if (dim == 2) return p == 1 ? launch_band<2, 1> : p == 2 ? launch_band<2, 2> : launch_band<2, 3>;
    return p == 1 ? launch_band<3, 1> : p == 2 ? launch_band<3, 2> : launch_band<3, 3>;
}
static samp_fn pick_samples(int dim, int p) {
    if (dim == 2) return p == 1 ? launch_samples<2, 1> : p == 2 ? launch_samples<2, 2> : launch_samples<2, 3>;
    return p == 1 ? launch_samples<3, 1> : p == 2 ? launch_samples<3, 2> : launch_samples<3, 3>;
}

// Sampled 0-based indices of one direction (Sec. 5.1): L = m-4p interior points,
// n = ceil((L-1)/M) intervals, offsets round(j (L-1)/n) half away from zero,
// computed exactly as floor((2 j (L-1) + n) / (2 n)).
static std::vector<int> sample_rule(int m, int p, int M) {
    const int lo = 2 * p, L = m - 4 * p;
    std::vector<int> out;
    if (L == 1) {
        out.push_back(lo);
        return out;
    }
    const long long n = (L - 1 + M - 1) / M;
    for (long long j = 0; j <= n; ++j) out.push_back(lo + (int)((2 * j * (L - 1) + n) / (2 * n)));
    return out;
}

struct EventTimer {
    cudaEvent_t ev[6];
    bool ok = false;
    EventTimer() {
        ok = true;
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) ok = false;
    }
    ~EventTimer() {
        for (auto& e : ev) cudaEventDestroy(e);
    }
};

}  // namespace iga

using namespace iga;

extern "C" int iga_surrogate_assemble(iga_space* s, int p, int q, int M, unsigned flags, void* stream,
                                      iga_ops** out) {
    if (!s || !out) return fail(IGA_ERR_ARG, "null argument");
    *out = nullptr;
    if (p != s->p) return fail(IGA_ERR_ARG, "p must equal the space degree");
    const bool true_only = (flags & IGA_TRUE_ONLY) != 0;
    if (!true_only) {
        if (q < 1 || q > 7) return fail(IGA_ERR_ARG, "q must be in 1..7");
        if (M < 1) return fail(IGA_ERR_ARG, "M must be >= 1");
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int dim = s->dim, m = s->m, D = s->D, T0 = (D - 1) / 2;
    iga_ops* ops = new (std::nothrow) iga_ops();
    if (!ops) return fail(IGA_ERR_OOM, "host allocation failed");
    ops->space = s;
    ops->p = p;
    ops->q = q;
    ops->M = M;
    ops->dim = dim;
    ops->m = m;
    ops->D = D;
    ops->nK = T0;
    ops->nM = T0 + 1;
    ops->N = s->N;
    ops->pitch = (s->N + 63) / 64 * 64;
    ops->flags = flags;
    const long long pitch = ops->pitch;
    auto bail = [&](int rc) {
        delete ops;
        return rc;
    };
    int rc = ops->fK64.alloc(sizeof(double) * ops->nK * pitch);
    if (!rc) rc = ops->fM64.alloc(sizeof(double) * ops->nM * pitch);
    if (!rc) rc = ops->fK32.alloc(sizeof(float) * ops->nK * pitch);
    if (!rc) rc = ops->fM32.alloc(sizeof(float) * ops->nM * pitch);
    if (!rc) rc = ops->dinv64.alloc(sizeof(double) * pitch);
    if (!rc) rc = ops->dinv32.alloc(sizeof(float) * pitch);
    if (!rc) rc = ops->status.alloc(sizeof(int) * 4);
    if (rc) return bail(rc);
    if (cudaMemsetAsync(ops->fK64.ptr, 0, ops->fK64.bytes, st) != cudaSuccess ||
        cudaMemsetAsync(ops->fM64.ptr, 0, ops->fM64.bytes, st) != cudaSuccess ||
        cudaMemsetAsync(ops->status.ptr, 0, ops->status.bytes, st) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaMemsetAsync"));

    // ---- a0: band (or all) elements grouped by colour for a3 (an index set of the mesh,
    // built once per space and kept on the device)
    const int ne = s->n_el, P1 = p + 1;
    int ncol = 1;
    for (int k = 0; k < dim; ++k) ncol *= P1;
    const int lk = true_only ? 1 : 0;
    if (s->band_offs[lk].empty()) {
        std::vector<std::vector<int>> colour(ncol);
        long long nel_total = 1;
        for (int k = 0; k < dim; ++k) nel_total *= ne;
        for (long long el = 0; el < nel_total; ++el) {
            long long r = el;
            bool band = false;
            int c = 0, cw = 1;
            for (int k = 0; k < dim; ++k) {
                const int ek = (int)(r % ne);
                r /= ne;
                band = band || ek <= 2 * p - 1 || ek >= ne - 2 * p;
                c += (ek % P1) * cw;
                cw *= P1;
            }
            if (true_only || band) colour[c].push_back((int)el);
        }
        std::vector<int> flat;
        std::vector<int> offs(ncol + 1, 0);
        for (int c = 0; c < ncol; ++c) {
            offs[c] = (int)flat.size();
            flat.insert(flat.end(), colour[c].begin(), colour[c].end());
        }
        offs[ncol] = (int)flat.size();
        if ((rc = s->band_elems[lk].alloc(sizeof(int) * std::max<size_t>(1, flat.size())))) return bail(rc);
        if (!flat.empty()) {
            cudaError_t e = cudaMemcpy(s->band_elems[lk].ptr, flat.data(), sizeof(int) * flat.size(),
                                       cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                s->band_elems[lk].release();
                return bail(cuda_fail(e, "cudaMemcpy(elements)"));
            }
        }
        s->band_offs[lk] = offs;
    }
    const std::vector<int>& offs = s->band_offs[lk];
    ops->n_band = offs[ncol];
    const DevBuf& d_elems = s->band_elems[lk];
    EventTimer tm;
    cudaEventRecord(tm.ev[0], st);
    // ---- a3: band quadrature, one launch per colour
    band_fn bf = pick_band(dim, p);
    for (int c = 0; c < ncol; ++c) {
        const int cnt = offs[c + 1] - offs[c];
        if (cnt == 0) continue;
        if ((rc = bf(s, d_elems.as<int>() + offs[c], cnt, ops, true_only ? 1 : 0, st))) return bail(rc);
    }
    cudaEventRecord(tm.ev[1], st);

    DevBuf d_samp, d_Ainv, d_espan, d_evals, d_tmp;
    if (!true_only) {
        // ---- a0: sampling rule
        ops->samp = sample_rule(m, p, M);
        ops->ns = (int)ops->samp.size();
        const int ns = ops->ns, L = m - 4 * p;
        if (ns < q + 1) return bail(fail(IGA_ERR_ARG, "need at least q+1 samples per direction"));
        int nsd = 1;
        for (int k = 0; k < dim; ++k) nsd *= ns;
        ops->n_samples = nsd;
        if ((rc = d_samp.alloc(sizeof(int) * ns))) return bail(rc);
        cudaMemcpyAsync(d_samp.ptr, ops->samp.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st);
        if ((rc = ops->sK.alloc(sizeof(double) * D * nsd))) return bail(rc);
        if ((rc = ops->sM.alloc(sizeof(double) * D * nsd))) return bail(rc);
        if ((rc = ops->cK.alloc(sizeof(double) * D * nsd))) return bail(rc);
        if ((rc = ops->cM.alloc(sizeof(double) * D * nsd))) return bail(rc);
        if ((rc = d_tmp.alloc(sizeof(double) * D * nsd))) return bail(rc);
        // ---- a2: true rows at the samples
        if ((rc = pick_samples(dim, p)(s, d_samp.as<int>(), ops, st))) return bail(rc);
        cudaEventRecord(tm.ev[2], st);
        // ---- a4: interpolation operators on the host (x~ abscissae, de Boor knots)
        const double h = 1.0 / s->n_el;
        std::vector<double> xs(ns);
        for (int j = 0; j < ns; ++j) xs[j] = (ops->samp[j] + 1 - 0.5 * (p + 1)) * h;
        std::vector<double> kn = hb::averaged_knots(xs, q), Ainv;
        if (!hb::collocation_inverse(kn, q, xs, Ainv))
            return bail(fail(IGA_ERR_ARG, "singular interpolation matrix"));
        std::vector<int> espan(L);
        std::vector<double> evals((size_t)L * (q + 1));
        for (int l = 0; l < L; ++l) {
            const double x = (2 * p + l + 1 - 0.5 * (p + 1)) * h;
            const int mu = hb::find_span(kn, q, x);
            hb::basis_and_derivative(kn, q, mu, x, &evals[(size_t)l * (q + 1)], nullptr);
            espan[l] = mu - q;
        }
        if ((rc = d_Ainv.alloc(sizeof(double) * Ainv.size()))) return bail(rc);
        if ((rc = d_espan.alloc(sizeof(int) * L))) return bail(rc);
        if ((rc = d_evals.alloc(sizeof(double) * evals.size()))) return bail(rc);
        cudaMemcpyAsync(d_Ainv.ptr, Ainv.data(), sizeof(double) * Ainv.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_espan.ptr, espan.data(), sizeof(int) * L, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_evals.ptr, evals.data(), sizeof(double) * evals.size(), cudaMemcpyHostToDevice, st);
        for (int which = 0; which < 2; ++which) {
            double* src = which ? ops->sM.as<double>() : ops->sK.as<double>();
            double* dst = which ? ops->cM.as<double>() : ops->cK.as<double>();
            // ping-pong so the last direction lands in dst
            double* bufs[2] = {dst, d_tmp.as<double>()};
            const double* in = src;
            for (int dir = 0; dir < dim; ++dir) {
                double* o = bufs[(dim - 1 - dir) % 2];
                const long long total = (long long)D * nsd;
                const int grid = (int)std::min<long long>((total + 255) / 256, 4096);
                interp_dir_kernel<<<grid, 256, 0, st>>>(in, o, d_Ainv.as<double>(), ns, dim, dir, D);
                IGA_LAUNCH_CHECK("interp_dir_kernel");
                in = o;
            }
        }
        cudaEventRecord(tm.ev[3], st);
        // ---- a5: surrogate values in Omega~, sum-factorised (one direction per launch),
        // fields in chunks so that the intermediate tensors stay below ~256 MB
        long long Ld = 1;
        for (int k = 0; k < dim; ++k) Ld *= L;
        // values per field after contracting directions 0..k: L^{k+1} ns^{d-1-k}
        std::vector<long long> ext(dim);
        for (int k = 0; k < dim; ++k) {
            long long v = 1;
            for (int j = 0; j < dim; ++j) v *= j <= k ? L : ns;
            ext[k] = v;
        }
        long long per_field = 0;
        for (int k = 0; k + 1 < dim; ++k) per_field += ext[k];
        const int chunk = (int)std::max<long long>(1, std::min<long long>(D, (32LL << 20) / std::max(1LL, per_field)));
        DevBuf d_eval;
        if ((rc = d_eval.alloc(sizeof(double) * std::max(1LL, per_field) * chunk))) return bail(rc);
        for (int which = 0; which < 2; ++which) {
            const int t_begin = which ? T0 : T0 + 1;
            const int fbase = which ? T0 : T0 + 1;
            double* coef = which ? ops->cM.as<double>() : ops->cK.as<double>();
            double* fld = which ? ops->fM64.as<double>() : ops->fK64.as<double>();
            for (int t0c = t_begin; t0c < D; t0c += chunk) {
                const int nf = std::min(chunk, D - t0c);
                const double* in = coef + (size_t)t0c * nsd;
                long long in_stride = nsd;
                double* buf = d_eval.as<double>();
                for (int dir = 0; dir + 1 < dim; ++dir) {
                    const long long total = (long long)nf * ext[dir];
                    const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 16);
                    eval_dir_kernel<<<grid, 256, 0, st>>>(in, in_stride, buf, ext[dir], nf, d_espan.as<int>(),
                                                          d_evals.as<double>(), q, ns, L, dim, dir);
                    IGA_LAUNCH_CHECK("eval_dir_kernel");
                    in = buf;
                    in_stride = ext[dir];
                    buf += (size_t)nf * ext[dir];
                }
                const long long total = (long long)nf * Ld;
                const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 16);
                if (dim == 2)
                    eval_last_kernel<2><<<grid, 256, 0, st>>>(in, in_stride, nf, t0c, fbase, d_espan.as<int>(),
                                                              d_evals.as<double>(), q, ns, L, 2 * p, m, p, fld, pitch);
                else
                    eval_last_kernel<3><<<grid, 256, 0, st>>>(in, in_stride, nf, t0c, fbase, d_espan.as<int>(),
                                                              d_evals.as<double>(), q, ns, L, 2 * p, m, p, fld, pitch);
                IGA_LAUNCH_CHECK("eval_last_kernel");
            }
        }
    } else {
        cudaEventRecord(tm.ev[2], st);
        cudaEventRecord(tm.ev[3], st);
    }
    if (flags & IGA_MASS_VOLUME_PRESERVING) {
        const int d2 = dim * 10 + p;
        rc = d2 == 21   ? launch_volume_preserving<2, 1>(s, ops, st)
             : d2 == 22 ? launch_volume_preserving<2, 2>(s, ops, st)
             : d2 == 23 ? launch_volume_preserving<2, 3>(s, ops, st)
             : d2 == 31 ? launch_volume_preserving<3, 1>(s, ops, st)
             : d2 == 32 ? launch_volume_preserving<3, 2>(s, ops, st)
                        : fail(IGA_ERR_ARG, "unsupported (dim, p) for the volume-preserving mass");
        if (rc) return bail(rc);
    }
    cudaEventRecord(tm.ev[4], st);
    {
        const long long total = (long long)(ops->nK + ops->nM) * pitch;
        const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 16);
        finalize_kernel<<<grid, 256, 0, st>>>(ops->fK64.as<double>(), ops->fM64.as<double>(),
                                              ops->fK32.as<float>(), ops->fM32.as<float>(),
                                              ops->dinv64.as<double>(), ops->dinv32.as<float>(), ops->nK,
                                              ops->nM, ops->N, pitch, ops->status.as<int>());
        IGA_LAUNCH_CHECK("finalize_kernel");
    }
    cudaEventRecord(tm.ev[5], st);
    int status[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(status, ops->status.ptr, sizeof(status), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "surrogate_assemble"));
    if (status[0] & 2) return bail(fail(IGA_ERR_ARG, "non-positive det J at a quadrature point"));
    if (status[0] & 1) return bail(fail(IGA_ERR_NONFINITE, "non-finite or non-positive mass diagonal"));
    float t;
    cudaEventElapsedTime(&t, tm.ev[0], tm.ev[1]);
    ops->t_band = t;
    cudaEventElapsedTime(&t, tm.ev[1], tm.ev[2]);
    ops->t_sample = t;
    cudaEventElapsedTime(&t, tm.ev[2], tm.ev[3]);
    ops->t_interp = t;
    cudaEventElapsedTime(&t, tm.ev[3], tm.ev[4]);
    ops->t_eval = t;
    cudaEventElapsedTime(&t, tm.ev[0], tm.ev[5]);
    ops->t_total = t;
    rc = brick_prepare(ops, st);
    if (rc) return bail(rc);
    // the interpolation coefficients and the evaluation tables stay (2 D ns^d + L (q+2)
    // values): the on-the-fly apply evaluates the stencil functions from them
    if (!true_only) {
        std::swap(ops->espan.ptr, d_espan.ptr);
        std::swap(ops->espan.bytes, d_espan.bytes);
        std::swap(ops->evals.ptr, d_evals.ptr);
        std::swap(ops->evals.bytes, d_evals.bytes);
    }
    if (!(flags & IGA_KEEP_SAMPLES)) {
        ops->sK.release();
        ops->sM.release();
    }
    *out = ops;
    return IGA_OK;
}

extern "C" int iga_sampling_length_for_mesh(double h, int p, int q, double a, double b, double C, double eps,
                                            int* M_out) {
    if (!M_out) return fail(IGA_ERR_ARG, "null argument");
    if (!(h > 0.0) || !(q + b > 0.0) || !(C > 0.0) || !(eps > 0.0) || p < 1)
        return fail(IGA_ERR_ARG, "need h > 0, q + b > 0, C > 0, eps > 0, p >= 1");
    // Eq. MeshDependentSamplingLength, FP64; saturates at INT_MAX
    const double v = std::floor(C * std::pow(h, eps - 1.0 + (p + a) / (q + b)));
    *M_out = v >= 2147483647.0 ? 2147483647 : std::max(1, (int)v);
    return IGA_OK;
}

extern "C" int iga_ops_destroy(iga_ops* ops) {
    delete ops;
    return IGA_OK;
}

extern "C" int iga_ops_info_get(const iga_ops* ops, iga_ops_info* out) {
    if (!ops || !out) return fail(IGA_ERR_ARG, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->N = ops->N;
    out->pitch = ops->pitch;
    out->m = ops->m;
    out->dim = ops->dim;
    out->p = ops->p;
    out->q = ops->q;
    out->M = ops->M;
    out->nK = ops->nK;
    out->nM = ops->nM;
    out->D = ops->D;
    out->ns = ops->ns;
    out->n_band_elements = ops->n_band;
    out->n_sample_rows = ops->n_samples;
    out->t_sample_ms = ops->t_sample;
    out->t_band_ms = ops->t_band;
    out->t_interp_ms = ops->t_interp;
    out->t_eval_ms = ops->t_eval;
    out->t_total_ms = ops->t_total;
    out->workspace_bytes = (long long)ops->work.bytes;
    return IGA_OK;
}

extern "C" int iga_ops_copy_fields(const iga_ops* ops, int which, int dtype, void* dst, void* stream) {
    if (!ops || !dst) return fail(IGA_ERR_ARG, "null argument");
    if (which != IGA_OP_K && which != IGA_OP_M) return fail(IGA_ERR_ARG, "which must be K or M");
    if (dtype != IGA_F32 && dtype != IGA_F64) return fail(IGA_ERR_ARG, "bad dtype");
    const int nf = which == IGA_OP_K ? ops->nK : ops->nM;
    const size_t es = dtype == IGA_F64 ? 8 : 4;
    const DevBuf& src = which == IGA_OP_K ? (dtype == IGA_F64 ? ops->fK64 : ops->fK32)
                                          : (dtype == IGA_F64 ? ops->fM64 : ops->fM32);
    IGA_CUDA(cudaMemcpy2DAsync(dst, es * ops->N, src.ptr, es * ops->pitch, es * ops->N, nf,
                               cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return IGA_OK;
}

extern "C" int iga_ops_copy_samples(const iga_ops* ops, int which, double* dst, void* stream) {
    if (!ops || !dst) return fail(IGA_ERR_ARG, "null argument");
    const DevBuf& src = which == IGA_OP_K ? ops->sK : ops->sM;
    if (!src.ptr) return fail(IGA_ERR_ARG, "samples not kept (assemble with IGA_KEEP_SAMPLES)");
    IGA_CUDA(cudaMemcpyAsync(dst, src.ptr, sizeof(double) * ops->D * ops->n_samples, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    return IGA_OK;
}

extern "C" int iga_ops_sample_indices(const iga_ops* ops, int* host_dst) {
    if (!ops || !host_dst) return fail(IGA_ERR_ARG, "null argument");
    for (int j = 0; j < ops->ns; ++j) host_dst[j] = ops->samp[j];
    return IGA_OK;
}
