// wave_adjoint: gradient of the receiver misfit with respect to the B-spline
// coefficients theta of the wave speed, by the discrete adjoint of the whole
// path (leapfrog with consistent-mass CG, then surrogate assembly).
//
// Forward (FP64, as wave_step):  u^1 = u^0 + dt^2/2 a^0,  u^{n+1} = 2u^n - u^{n-1} + dt^2 a^n,
// M~ a^n = f^n - K~ u^n, traces d^n = R u^n (n = 1..N),
// J = dt/2 sum_n sum_shots |d^n - d_obs^n|^2.
// Only K~ depends on theta.  With ubar^m = dJ/du^m (u^0 is fixed):
//   ubar^N = dt R^T (d^N - d_obs^N),   nu^m = M~^-1 ubar^{m+1},
//   ubar^m = dt R^T (d^m - d_obs^m) + 2 ubar^{m+1} - dt^2 K~ nu^m - ubar^{m+2}   (1 <= m < N)
//   dJ/dK~_ij = - sum_{m=0}^{N-1} c_m dt^2 nu^m_i u^m_j   (c_0 = 1/2, c_m = 1).
// K~ is stored as its upper triangle S_delta[i] = K~(i, i+Delta) with the
// diagonal minus the row sum, so the gradient of a stored value is
//   G_delta[i] = sum_m c_m dt^2 (nu_i - nu_{i+Delta}) (u_i - u_{i+Delta}).
// Checkpoints: (u^n, u^{n-1}, a^{n-1}) and, with a CG start of order K > 0, the K
// older accelerations a^{n-2} .. a^{n-1-K}, every C steps; each segment is
// recomputed from its checkpoint (bitwise identical: the same CG starts) and then
// swept backwards.  The reverse-sweep solves M~ nu^m = ubar^{m+1} start from the
// same polynomial extrapolation, in reverse time, of nu^{m+1}, nu^{m+2}, .. (order
// up to K; only the starting point of each solve changes, every solve still runs
// to cg_rtol).
//
// Back through the assembly (every stored value is linear in true entries):
//   true slots        S = K_ij                                 (band elements)
//   surrogate slots   S = [(E A^-1) x ... ] samples_delta       (Sec. 3.3 interpolation)
//   samples           samples_delta[s] = K(i_s, i_s + delta)    (sample rows)
// and K_ij = sum_q grad phi_i^T (c^2 G^_q) grad phi_j, so
// dJ/dtheta_k = sum_q (2/c(s_q)) Z_q B_k(s_q),  Z_q = sum of slot gradients times the
// entry's integrand at q.  The Z_q live on the tensor grid of Gauss points; the
// last step is a separable contraction with the 1-D theta basis matrices.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_bspline.h"
#include "iga_internal.cuh"
#include "quad.cuh"
#include "stencil.cuh"

namespace iga {

// G_u[i] += c sum_s (nu_i - nu_{i+D}) (u_i - u_{i+D}) for every K~ field u
template <int DIM, int P>
__global__ void grad_accum_kernel(double* __restrict__ G, long long pitch, const double* __restrict__ nu,
                                  const double* __restrict__ u, int nshot, long long ld, int N, int m, double c) {
    constexpr int NF = StencilShape<DIM, P>::T0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        for (int f = 0; f < NF; ++f) {
            const int j = i + field_delta<DIM, P>(f, m);
            if (j >= N) continue;
            double acc = 0.0;
            for (int s = 0; s < nshot; ++s) {
                const size_t o = (size_t)s * ld;
                acc += (nu[o + i] - nu[o + j]) * (u[o + i] - u[o + j]);
            }
            G[(size_t)f * pitch + i] += c * acc;
        }
    }
}

// x = sum_{j <= k} c_j h_j with c_j = (-1)^j C(k+1, j+1): the degree-k polynomial
// through h_0 .. h_k evaluated one step further (start of the next adjoint solve).
struct NuGuess {
    const double* h[IGA_CG_GUESS_MAX + 1];
    double c[IGA_CG_GUESS_MAX + 1];
    int k;
};
__global__ void adj_guess_kernel(double* x, NuGuess g, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int j = 0; j <= g.k; ++j) v += g.c[j] * g.h[j][i];
        x[i] = v;
    }
}
static double binom_coeff(int k, int j) {   // (-1)^j C(k+1, j+1)
    double b = 1.0;
    for (int t = 1; t <= j + 1; ++t) b = b * (k + 2 - t) / t;
    return (j & 1) ? -b : b;
}

// ubar_s += scale sum_rec res[s][rec] R_rec^T (one thread per shot: deterministic)
__global__ void adj_inject_kernel(double* ubar, const int* __restrict__ idx, const double* __restrict__ w,
                                  const double* __restrict__ res, int nshot, int nrec, int nloc, long long ld,
                                  double scale) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshot) return;
    for (int rec = 0; rec < nrec; ++rec) {
        const double r = scale * res[(size_t)s * nrec + rec];
        for (int l = 0; l < nloc; ++l) ubar[(size_t)s * ld + idx[rec * nloc + l]] += w[rec * nloc + l] * r;
    }
}

// ubar_new = 2 ubar1 - dt2 Knu - ubar2
__global__ void adj_update_kernel(double* ubar_new, const double* ubar1, const double* ubar2, const double* Knu,
                                  long long n, double dt2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        ubar_new[i] = 2.0 * ubar1[i] - dt2 * Knu[i] - ubar2[i];
}

__device__ __forceinline__ long long qp_index(const int* e, const int* g, int nq, int nI, int dim) {
    long long li = 0;
    for (int k = dim - 1; k >= 0; --k) li = li * nI + (e[k] * nq + g[k]);
    return li;
}

// Band elements: W[q] += (2/c_q) sum_{true upper slots (a,b)} G_slot grad phi_a^T G_q grad phi_b
template <int DIM, int P>
__global__ void band_grad_kernel(GeomParams gp, const int* __restrict__ elems, const double* __restrict__ Gf,
                                 long long pitch, int lo, int hi, int all_true, double* W) {
    using S = Stencil<DIM, P>;
    extern __shared__ double sm[];
    const int nq = gp.nq;
    int nqd = nq;
#pragma unroll
    for (int k = 1; k < DIM; ++k) nqd *= nq;
    double* Gq = sm;                              // [nqd][NS]
    double* cq = Gq + nqd * S::NS;                // [nqd]
    double* grad = cq + nqd;                      // [NLOC][nqd][DIM]
    double* gw = grad + S::NLOC * nqd * DIM;      // [NLOC][NLOC]
    int e[3] = {0, 0, 0};
    decode<DIM>(elems[blockIdx.x], gp.n_el, e);
    for (int q = threadIdx.x; q < nqd; q += blockDim.x) {
        int g[3] = {0, 0, 0};
        decode<DIM>(q, nq, g);
        double G[6], wm;
        qp_weights(gp, e, g, G, wm);
#pragma unroll
        for (int k = 0; k < S::NS; ++k) Gq[q * S::NS + k] = G[k];
        cq[q] = coef_c(gp, e, g);
    }
    for (int idx = threadIdx.x; idx < S::NLOC * nqd; idx += blockDim.x) {
        const int a = idx / nqd, q = idx % nqd;
        int g[3] = {0, 0, 0}, al[3] = {0, 0, 0};
        decode<DIM>(q, nq, g);
        decode<DIM>(a, P + 1, al);
        double gr[DIM], v;
        local_basis<DIM, P>(gp, e, g, al, gr, v);
#pragma unroll
        for (int k = 0; k < DIM; ++k) grad[(a * nqd + q) * DIM + k] = gr[k];
    }
    const int m = gp.m;
    for (int pidx = threadIdx.x; pidx < S::NLOC * S::NLOC; pidx += blockDim.x) {
        const int a = pidx / S::NLOC, b = pidx % S::NLOC;
        int al[3] = {0, 0, 0}, bl[3] = {0, 0, 0}, i[3] = {0, 0, 0}, j[3] = {0, 0, 0};
        decode<DIM>(a, P + 1, al);
        decode<DIM>(b, P + 1, bl);
        int t = 0;
        for (int k = DIM - 1; k >= 0; --k) t = t * S::PP + (bl[k] - al[k] + P);
        double wv = 0.0;
        if (t > S::T0) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                i[k] = e[k] + al[k];
                j[k] = e[k] + bl[k];
            }
            if (all_true || !(in_range<DIM>(i, lo, hi) && in_range<DIM>(j, lo, hi))) {
                long long li = 0;
                for (int k = DIM - 1; k >= 0; --k) li = li * m + i[k];
                wv = Gf[(size_t)(t - S::T0 - 1) * pitch + li];
            }
        }
        gw[pidx] = wv;
    }
    __syncthreads();
    const int nI = gp.n_el * nq;
    for (int q = threadIdx.x; q < nqd; q += blockDim.x) {
        double z = 0.0;
        for (int a = 0; a < S::NLOC; ++a) {
            double v[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) v[k] = 0.0;
            for (int b = 0; b < S::NLOC; ++b) {
                const double wv = gw[a * S::NLOC + b];
                if (wv == 0.0) continue;
#pragma unroll
                for (int k = 0; k < DIM; ++k) v[k] += wv * grad[(b * nqd + q) * DIM + k];
            }
            double Gv[DIM];
            sym_matvec<DIM>(Gq + q * S::NS, v, Gv);
#pragma unroll
            for (int k = 0; k < DIM; ++k) z += grad[(a * nqd + q) * DIM + k] * Gv[k];
        }
        if (z != 0.0) {
            int g[3] = {0, 0, 0};
            decode<DIM>(q, nq, g);
            atomicAdd(W + qp_index(e, g, nq, nI, DIM), 2.0 / cq[q] * z);
        }
    }
}

// Sample rows: W[q] += (2/c_q) sum_{delta upper} Gs_delta[s] grad phi_a^T G_q grad phi_{a+delta}
template <int DIM, int P>
__global__ void sample_grad_kernel(GeomParams gp, const int* __restrict__ samp, int ns, const double* __restrict__ Gs,
                                   double* W) {
    using S = Stencil<DIM, P>;
    int sidx[3] = {0, 0, 0}, row[3] = {0, 0, 0};
    decode<DIM>(blockIdx.x, ns, sidx);
#pragma unroll
    for (int k = 0; k < DIM; ++k) row[k] = samp[sidx[k]];
    int nsd = ns, nqd = gp.nq;
#pragma unroll
    for (int k = 1; k < DIM; ++k) {
        nsd *= ns;
        nqd *= gp.nq;
    }
    const int nI = gp.n_el * gp.nq;
    // (element a, Gauss point q) pairs of the row's support
    for (int idx = threadIdx.x; idx < S::NLOC * nqd; idx += blockDim.x) {
        const int a = idx / nqd, q = idx % nqd;
        int al[3] = {0, 0, 0}, e[3] = {0, 0, 0}, g[3] = {0, 0, 0};
        decode<DIM>(a, P + 1, al);
        decode<DIM>(q, gp.nq, g);
#pragma unroll
        for (int k = 0; k < DIM; ++k) e[k] = row[k] - al[k];
        double G[6], wm;
        qp_weights(gp, e, g, G, wm);
        const double c = coef_c(gp, e, g);
        double ga[DIM], va, Gga[DIM];
        local_basis<DIM, P>(gp, e, g, al, ga, va);
        sym_matvec<DIM>(G, ga, Gga);
        double z = 0.0;
        for (int b = 0; b < S::NLOC; ++b) {
            int bl[3] = {0, 0, 0};
            decode<DIM>(b, P + 1, bl);
            int t = 0;
            for (int k = DIM - 1; k >= 0; --k) t = t * S::PP + (bl[k] - al[k] + P);
            if (t <= S::T0) continue;
            const double gs = Gs[(size_t)(t - S::T0 - 1) * nsd + blockIdx.x];
            if (gs == 0.0) continue;
            double gb[DIM], vb;
            local_basis<DIM, P>(gp, e, g, bl, gb, vb);
            double d = 0.0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) d += Gga[k] * gb[k];
            z += gs * d;
        }
        if (z != 0.0) atomicAdd(W + qp_index(e, g, gp.nq, nI, DIM), 2.0 / c * z);
    }
}

// Gm[f][l] = G_f[i(l)] if row lo+l and its neighbour lo+l+delta_f are both interior, else 0
template <int DIM, int P>
__global__ void mask_gather_kernel(const double* __restrict__ Gf, long long pitch, double* __restrict__ Gm, int L,
                                   int lo, int m) {
    constexpr int PP = 2 * P + 1;
    const int f = blockIdx.y;
    const int t = StencilShape<DIM, P>::T0 + 1 + f;
    int delta[3] = {0, 0, 0};
    {
        int tt = t;
        for (int k = 0; k < DIM; ++k) {
            delta[k] = tt % PP - P;
            tt /= PP;
        }
    }
    int Ld = L;
    for (int k = 1; k < DIM; ++k) Ld *= L;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < Ld; r += gridDim.x * blockDim.x) {
        int l[3] = {0, 0, 0};
        decode<DIM>(r, L, l);
        bool ok = true;
        long long li = 0;
        for (int k = DIM - 1; k >= 0; --k) {
            ok = ok && l[k] + delta[k] >= 0 && l[k] + delta[k] < L;
            li = li * m + (lo + l[k]);
        }
        Gm[(size_t)f * Ld + r] = ok ? Gf[(size_t)f * pitch + li] : 0.0;
    }
}

// out[t][..c..] = sum_j A[c][j] in[t][..j..] along direction dir; shapes colex (n0 fastest)
__global__ void contract_kernel(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ A,
                                int nT, int n0, int n1, int n2, int dir, int rows) {
    int shp[3] = {n0, n1, n2};
    const int ncol = shp[dir];
    int oshp[3] = {n0, n1, n2};
    oshp[dir] = rows;
    const long long nout_t = (long long)oshp[0] * oshp[1] * oshp[2];
    const long long nin_t = (long long)n0 * n1 * n2;
    long long stride = 1;
    for (int k = 0; k < dir; ++k) stride *= shp[k];
    const long long total = nout_t * nT;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long t = idx / nout_t;
        long long o = idx % nout_t;
        int oc[3];
        for (int k = 0; k < 3; ++k) {
            oc[k] = (int)(o % oshp[k]);
            o /= oshp[k];
        }
        const int c = oc[dir];
        oc[dir] = 0;
        const long long base = t * nin_t + oc[0] + (long long)shp[0] * (oc[1] + (long long)shp[1] * oc[2]);
        double acc = 0.0;
        for (int j = 0; j < ncol; ++j) acc += A[(size_t)c * ncol + j] * in[base + j * stride];
        out[idx] = acc;
    }
}

static int contract(const double* in, double* out, const std::vector<double>& A_h, DevBuf& dA, int nT, int* shape,
                    int dir, int rows, cudaStream_t st) {
    int rc = dA.alloc(sizeof(double) * A_h.size());
    if (rc) return rc;
    IGA_CUDA(cudaMemcpyAsync(dA.ptr, A_h.data(), sizeof(double) * A_h.size(), cudaMemcpyHostToDevice, st));
    long long nout = nT;
    for (int k = 0; k < 3; ++k) nout *= (k == dir ? rows : shape[k]);
    const int grid = (int)std::max<long long>(1, std::min<long long>((nout + 255) / 256, 152 * 16));
    contract_kernel<<<grid, 256, 0, st>>>(in, out, dA.as<double>(), nT, shape[0], shape[1], shape[2], dir, rows);
    IGA_LAUNCH_CHECK("contract_kernel");
    IGA_CUDA(cudaStreamSynchronize(st));   // dA is reused by the next contraction
    shape[dir] = rows;
    return IGA_OK;
}

template <int DIM, int P>
static int adjoint_dp(iga_wave* w, int nsteps, int ckpt, const double* obs, double* J_out, double* grad_out,
                      cudaStream_t st) {
    const iga_ops* ops = w->ops;
    const iga_space* sp = ops->space;
    const long long N = w->N;
    const int nshot = w->nshot, nrec = w->nrec, nloc = w->nloc;
    const double dt = w->desc.dt, dt2 = dt * dt;
    const size_t vec = (size_t)nshot * N;
    const int K = (nsteps + ckpt - 1) / ckpt;
    const int ugrid = (int)std::min<long long>((vec + 255) / 256, 152 * 16);
    int rc;
    // ---- forward with checkpoints (u^n, u^{n-1}, a^{n-1}, a^{n-2} .. a^{n-1-Kg}) at n = k C
    const int Kg = w->desc.cg_guess;
    const int nck = 3 + Kg;   // vectors per checkpoint
    DevBuf ckb;
    if ((rc = ckb.alloc(sizeof(double) * vec * nck * K))) return rc;
    if ((rc = wave_initial_state(w, st))) return rc;
    auto ck_vectors = [&](int k, void** v) {
        v[0] = w->u.ptr;
        v[1] = w->uprev.ptr;
        v[2] = w->a.ptr;
        for (int j = 0; j < Kg; ++j) v[3 + j] = w->ah[j].ptr;
        return ckb.as<double>() + (size_t)nck * k * vec;
    };
    for (int k = 0; k < K; ++k) {
        void* v[3 + IGA_CG_GUESS_MAX];
        double* c = ck_vectors(k, v);
        for (int j = 0; j < nck; ++j)
            IGA_CUDA(cudaMemcpyAsync(c + (size_t)j * vec, v[j], sizeof(double) * vec, cudaMemcpyDeviceToDevice, st));
        if ((rc = wave_step_impl(w, std::min(ckpt, nsteps - k * ckpt), st))) return rc;
    }
    // ---- misfit and residuals res[m][s][rec] = d^m - d_obs^m (m = 1..N, traces index m-1)
    std::vector<double> tr((size_t)nshot * nrec * w->desc.nsteps_max);
    IGA_CUDA(cudaMemcpy(tr.data(), w->traces.ptr, sizeof(double) * tr.size(), cudaMemcpyDeviceToHost));
    std::vector<double> res((size_t)(nsteps + 1) * nshot * nrec, 0.0);
    double J = 0.0;
    for (int s = 0; s < nshot; ++s)
        for (int r = 0; r < nrec; ++r)
            for (int n = 0; n < nsteps; ++n) {
                const double d = tr[((size_t)s * nrec + r) * w->desc.nsteps_max + n] -
                                 obs[((size_t)s * nrec + r) * nsteps + n];
                res[((size_t)(n + 1) * nshot + s) * nrec + r] = d;
                J += 0.5 * dt * d * d;
            }
    if (J_out) *J_out = J;
    if (!grad_out) return IGA_OK;
    DevBuf dres, seg, vb, G;
    if ((rc = dres.alloc(sizeof(double) * res.size()))) return rc;
    IGA_CUDA(cudaMemcpyAsync(dres.ptr, res.data(), sizeof(double) * res.size(), cudaMemcpyHostToDevice, st));
    if ((rc = seg.alloc(sizeof(double) * vec * ckpt))) return rc;
    if ((rc = vb.alloc(sizeof(double) * vec * 5))) return rc;
    if ((rc = G.alloc(sizeof(double) * (size_t)ops->nK * ops->pitch))) return rc;
    IGA_CUDA(cudaMemsetAsync(G.ptr, 0, G.bytes, st));
    IGA_CUDA(cudaMemsetAsync(vb.ptr, 0, vb.bytes, st));
    double* ub1 = vb.as<double>();   // ubar^{m+1}
    double* ub2 = ub1 + vec;         // ubar^{m+2}
    double* ubn = ub2 + vec;         // ubar^m
    double* nu = ubn + vec;          // nu^m (the solve's iterate)
    double* y = nu + vec;
    // nu^{m+1}, nu^{m+2}, .. for the extrapolated start of the reverse solves
    DevBuf nhb;
    if (Kg > 0 && (rc = nhb.alloc(sizeof(double) * vec * (Kg + 1)))) return rc;
    std::vector<double*> nuh;
    for (int j = 0; j <= Kg && Kg > 0; ++j) nuh.push_back(nhb.as<double>() + (size_t)j * vec);
    int n_hist = 0;   // nu vectors solved so far (reverse time)
    // ubar^N = dt R^T res^N
    adj_inject_kernel<<<(nshot + 31) / 32, 32, 0, st>>>(ub1, w->rec_idx.as<int>(), w->rec_w.as<double>(),
                                                        dres.as<double>() + (size_t)nsteps * nshot * nrec, nshot,
                                                        nrec, nloc, N, dt);
    IGA_LAUNCH_CHECK("adj_inject_kernel");
    const int grid = (int)std::min<long long>((N + 255) / 256, 152 * 8);
    for (int k = K - 1; k >= 0; --k) {
        const int n0 = k * ckpt, n1 = std::min(n0 + ckpt, nsteps);
        {
            void* v[3 + IGA_CG_GUESS_MAX];
            const double* c = ck_vectors(k, v);
            for (int j = 0; j < nck; ++j)
                IGA_CUDA(cudaMemcpyAsync(v[j], c + (size_t)j * vec, sizeof(double) * vec, cudaMemcpyDeviceToDevice, st));
        }
        w->step = n0;
        IGA_CUDA(cudaMemcpyAsync(seg.ptr, w->u.ptr, sizeof(double) * vec, cudaMemcpyDeviceToDevice, st));
        for (int j = 1; j < n1 - n0; ++j) {
            if ((rc = wave_step_impl(w, 1, st))) return rc;
            IGA_CUDA(cudaMemcpyAsync(seg.as<double>() + (size_t)j * vec, w->u.ptr, sizeof(double) * vec,
                                     cudaMemcpyDeviceToDevice, st));
        }
        for (int m = n1 - 1; m >= n0; --m) {
            if (Kg > 0 && n_hist >= 2) {
                // extrapolated start from nu^{m+1} .. nu^{m+1+kk}
                NuGuess gs;
                gs.k = std::min(Kg, n_hist - 1);
                for (int j = 0; j <= gs.k; ++j) {
                    gs.h[j] = nuh[j];
                    gs.c[j] = binom_coeff(gs.k, j);
                }
                adj_guess_kernel<<<ugrid, 256, 0, st>>>(nu, gs, (long long)vec);
                IGA_LAUNCH_CHECK("adj_guess_kernel");
            }
            rc = mass_solve_impl(ops, IGA_F64, ub1, nu, N, nshot, w->desc.cg_rtol, w->desc.cg_max_it,
                                 w->desc.solve_flags, nullptr, nullptr, st, w->work.ptr, w->work.bytes, nullptr,
                                 nullptr);
            if (rc) return rc;
            if (Kg > 0) {
                // nuh[0] <- nu^m, older ones shift (the oldest buffer is reused)
                double* oldest = nuh[Kg];
                for (int j = Kg; j > 0; --j) nuh[j] = nuh[j - 1];
                nuh[0] = oldest;
                IGA_CUDA(cudaMemcpyAsync(nuh[0], nu, sizeof(double) * vec, cudaMemcpyDeviceToDevice, st));
                n_hist = std::min(n_hist + 1, Kg + 1);
            }
            grad_accum_kernel<DIM, P><<<grid, 256, 0, st>>>(G.as<double>(), ops->pitch, nu,
                                                            seg.as<double>() + (size_t)(m - n0) * vec, nshot, N,
                                                            (int)N, ops->m, (m == 0 ? 0.5 : 1.0) * dt2);
            IGA_LAUNCH_CHECK("grad_accum_kernel");
            if (m >= 1) {
                if ((rc = launch_apply(ops, IGA_OP_K, IGA_F64, nu, y, nshot, st))) return rc;
                adj_update_kernel<<<ugrid, 256, 0, st>>>(ubn, ub1, ub2, y, (long long)vec, dt2);
                IGA_LAUNCH_CHECK("adj_update_kernel");
                adj_inject_kernel<<<(nshot + 31) / 32, 32, 0, st>>>(ubn, w->rec_idx.as<int>(), w->rec_w.as<double>(),
                                                                    dres.as<double>() + (size_t)m * nshot * nrec,
                                                                    nshot, nrec, nloc, N, dt);
                IGA_LAUNCH_CHECK("adj_inject_kernel");
                double* t = ub2;   // rotate: ubar^{m+2} <- ubar^{m+1}, ubar^{m+1} <- ubar^m
                ub2 = ub1;
                ub1 = ubn;
                ubn = t;
            }
        }
    }
    // ---- back through the assembly onto the Gauss-point grid
    const int nq = sp->nq, nI = sp->n_el * nq;
    size_t nW = 1;
    for (int k = 0; k < DIM; ++k) nW *= (size_t)nI;
    DevBuf Wb, elb;
    if ((rc = Wb.alloc(sizeof(double) * nW))) return rc;
    IGA_CUDA(cudaMemsetAsync(Wb.ptr, 0, Wb.bytes, st));
    const bool true_only = (ops->flags & IGA_TRUE_ONLY) != 0;
    std::vector<int> el;
    {
        long long tot = 1;
        for (int k = 0; k < DIM; ++k) tot *= sp->n_el;
        for (long long e = 0; e < tot; ++e) {
            long long r = e;
            bool band = false;
            for (int k = 0; k < DIM; ++k) {
                const int ek = (int)(r % sp->n_el);
                r /= sp->n_el;
                band = band || ek <= 2 * P - 1 || ek >= sp->n_el - 2 * P;
            }
            if (true_only || band) el.push_back((int)e);
        }
    }
    if ((rc = elb.alloc(sizeof(int) * std::max<size_t>(1, el.size())))) return rc;
    IGA_CUDA(cudaMemcpyAsync(elb.ptr, el.data(), sizeof(int) * el.size(), cudaMemcpyHostToDevice, st));
    {
        using S = Stencil<DIM, P>;
        int nqd = 1;
        for (int k = 0; k < DIM; ++k) nqd *= nq;
        const size_t smem = sizeof(double) * (nqd * (S::NS + 1) + S::NLOC * nqd * DIM + S::NLOC * S::NLOC);
        if (smem > 200 * 1024) return fail(IGA_ERR_ARG, "adjoint quadrature tables exceed shared memory");
        IGA_CUDA(cudaFuncSetAttribute(band_grad_kernel<DIM, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        if (!el.empty()) {
            band_grad_kernel<DIM, P><<<(unsigned)el.size(), 128, smem, st>>>(
                sp->gp, elb.as<int>(), G.as<double>(), ops->pitch, 2 * P, sp->m - 2 * P - 1, true_only ? 1 : 0,
                Wb.as<double>());
            IGA_LAUNCH_CHECK("band_grad_kernel");
        }
    }
    DevBuf b1, b2, dA, dsamp;
    if (!true_only) {
        const int L = sp->m - 4 * P, ns = ops->ns, nK = ops->nK;
        long long Ld = 1, nsd = 1;
        for (int k = 0; k < DIM; ++k) {
            Ld *= L;
            nsd *= ns;
        }
        if ((rc = b1.alloc(sizeof(double) * nK * Ld)) || (rc = b2.alloc(sizeof(double) * nK * Ld))) return rc;
        dim3 g2((unsigned)std::min<long long>((Ld + 255) / 256, 1024), nK);
        mask_gather_kernel<DIM, P><<<g2, 256, 0, st>>>(G.as<double>(), ops->pitch, b1.as<double>(), L, 2 * P, sp->m);
        IGA_LAUNCH_CHECK("mask_gather_kernel");
        // host operators: E^T (ns x L), A^-T (ns x ns)
        const double h = 1.0 / sp->n_el;
        std::vector<double> xs(ns);
        for (int j = 0; j < ns; ++j) xs[j] = (ops->samp[j] + 1 - 0.5 * (P + 1)) * h;
        std::vector<double> kn = hb::averaged_knots(xs, ops->q), Ainv;
        if (!hb::collocation_inverse(kn, ops->q, xs, Ainv)) return fail(IGA_ERR_ARG, "singular interpolation matrix");
        std::vector<double> Et((size_t)ns * L, 0.0), At((size_t)ns * ns);
        std::vector<double> Nv(ops->q + 1);
        for (int l = 0; l < L; ++l) {
            const double x = (2 * P + l + 1 - 0.5 * (P + 1)) * h;
            const int mu = hb::find_span(kn, ops->q, x);
            hb::basis_and_derivative(kn, ops->q, mu, x, Nv.data(), nullptr);
            for (int a = 0; a <= ops->q; ++a) Et[(size_t)(mu - ops->q + a) * L + l] = Nv[a];
        }
        for (int r = 0; r < ns; ++r)
            for (int c2 = 0; c2 < ns; ++c2) At[(size_t)r * ns + c2] = Ainv[(size_t)c2 * ns + r];
        int shape[3] = {L, DIM > 1 ? L : 1, DIM > 2 ? L : 1};
        double* in = b1.as<double>();
        double* out = b2.as<double>();
        for (int dir = 0; dir < DIM; ++dir) {
            if ((rc = contract(in, out, Et, dA, nK, shape, dir, ns, st))) return rc;
            std::swap(in, out);
        }
        for (int dir = 0; dir < DIM; ++dir) {
            if ((rc = contract(in, out, At, dA, nK, shape, dir, ns, st))) return rc;
            std::swap(in, out);
        }
        if ((rc = dsamp.alloc(sizeof(int) * ns))) return rc;
        IGA_CUDA(cudaMemcpyAsync(dsamp.ptr, ops->samp.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
        sample_grad_kernel<DIM, P><<<(unsigned)nsd, 128, 0, st>>>(sp->gp, dsamp.as<int>(), ns, in, Wb.as<double>());
        IGA_LAUNCH_CHECK("sample_grad_kernel");
    }
    // ---- theta contraction: grad[k] = sum_I W[I] prod_d B_{k_d}(s_{I_d})
    const int nth = sp->desc.n_theta, kd = sp->desc.theta_degree;
    std::vector<double> Bt((size_t)nth * nI, 0.0);
    for (int I = 0; I < nI; ++I)
        for (int a = 0; a <= kd; ++a) Bt[(size_t)(sp->tspan_h[I] + a) * nI + I] = sp->tval_h[(size_t)I * (kd + 1) + a];
    DevBuf t1, t2;
    if ((rc = t1.alloc(sizeof(double) * nW)) || (rc = t2.alloc(sizeof(double) * nW))) return rc;
    int shape[3] = {nI, DIM > 1 ? nI : 1, DIM > 2 ? nI : 1};
    const double* in = Wb.as<double>();
    double* bufs[2] = {t1.as<double>(), t2.as<double>()};
    for (int dir = 0; dir < DIM; ++dir) {
        if ((rc = contract(in, bufs[dir % 2], Bt, dA, 1, shape, dir, nth, st))) return rc;
        in = bufs[dir % 2];
    }
    size_t ng = 1;
    for (int k = 0; k < DIM; ++k) ng *= (size_t)nth;
    IGA_CUDA(cudaMemcpy(grad_out, in, sizeof(double) * ng, cudaMemcpyDeviceToHost));
    return IGA_OK;
}

}  // namespace iga

using namespace iga;

extern "C" int iga_wave_adjoint(iga_wave* w, int nsteps, int checkpoint_every, const double* obs, double* J_out,
                                double* grad_theta, void* stream) {
    if (!w || !obs) return fail(IGA_ERR_ARG, "null argument");
    if (w->dtype != IGA_F64) return fail(IGA_ERR_ARG, "wave_adjoint needs an FP64 wave");
    if (w->nrec < 1) return fail(IGA_ERR_ARG, "wave_adjoint needs receivers");
    if (nsteps < 1 || nsteps > w->desc.nsteps_max) return fail(IGA_ERR_ARG, "nsteps must be in 1..nsteps_max");
    if (checkpoint_every < 1) return fail(IGA_ERR_ARG, "checkpoint_every must be >= 1");
    const iga_space* sp = w->ops->space;
    if (grad_theta && sp->desc.coef_kind != IGA_COEF_BSPLINE)
        return fail(IGA_ERR_ARG, "the gradient is taken with respect to a B-spline wave speed");
    cudaStream_t st = (cudaStream_t)stream;
    const int d = sp->dim, p = sp->p;
    // The forward and the recomputed segments use the wave's CG start (cg_guess);
    // the checkpoints carry the acceleration history it needs, so every segment
    // restarts exactly.
    int rc;
    if (d == 2 && p == 1) rc = adjoint_dp<2, 1>(w, nsteps, checkpoint_every, obs, J_out, grad_theta, st);
    else if (d == 2 && p == 2) rc = adjoint_dp<2, 2>(w, nsteps, checkpoint_every, obs, J_out, grad_theta, st);
    else if (d == 2 && p == 3) rc = adjoint_dp<2, 3>(w, nsteps, checkpoint_every, obs, J_out, grad_theta, st);
    else if (d == 3 && p == 1) rc = adjoint_dp<3, 1>(w, nsteps, checkpoint_every, obs, J_out, grad_theta, st);
    else if (d == 3 && p == 2) rc = adjoint_dp<3, 2>(w, nsteps, checkpoint_every, obs, J_out, grad_theta, st);
    else return fail(IGA_ERR_ARG, "unsupported (dim, p) for wave_adjoint");
    if (rc) return rc;
    IGA_CUDA(cudaStreamSynchronize(st));
    return IGA_OK;
}
