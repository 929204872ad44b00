// Leapfrog time stepping of M~ u'' + K~ u = f for many shots at once.
//
// Per step n (t_n = n dt), for all shots r as right-hand sides of one launch:
//   force:    b_r = -K~ u_r            (difference form; fields read once for all shots)
//   source:   b_r += amp ricker(t_n) B(s_src,r)    ((p+1)^d entries per shot)
//   solve:    M~ a_r = b_r by Jacobi-PCG from a_r^{n-1}      (mass_solve path)
//   update:   u_r^{n+1} = 2 u_r^n - u_r^{n-1} + dt^2 a_r     (n = 0: u^0 + dt^2/2 a^0)
//   record:   d_{r,k}^{n+1} = sum_i u_{r,i}^{n+1} B_i(s_rec,k)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "geom.cuh"
#include "host_bspline.h"
#include "iga_internal.cuh"
#include "leapfrog.cuh"
#include "stencil.cuh"

namespace iga {

template <int DIM, int P, typename T, int R>
__global__ void __launch_bounds__(256) force_kernel(const T* __restrict__ F, long long pitch, const T* __restrict__ u,
                                                     T* __restrict__ b, int N, int m) {
    __shared__ int sdl[StencilShape<DIM, P>::T0];
    fill_delta_table<DIM, P>(sdl, m);
    const int dmax = max_delta<DIM, P>(m);
    const LdgLoad<T> ld{u, N};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        T acc[R], own[R];
        if (i >= dmax && i < N - dmax)
            stencil_row_interior<DIM, P, T, false, R, (R >= 4 ? 2 : 4)>(F, pitch, ld, i, sdl, acc, own);
        else
            stencil_row<DIM, P, T, false, R, (R >= 4 ? 2 : 4)>(F, pitch, ld, i, N, m, acc, own);
#pragma unroll
        for (int r = 0; r < R; ++r) b[(size_t)r * N + i] = -acc[r];
    }
}

template <typename T>
__global__ void source_kernel(T* b, const int* idx, const double* w, int nshot, int nloc, long long N, double amp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nshot * nloc) return;
    const int r = k / nloc;
    b[(size_t)r * N + idx[k]] += (T)(amp * w[k]);   // distinct rows within one shot
}

template <typename T>
__global__ void update_kernel(const T* __restrict__ u, T* __restrict__ uprev, const T* __restrict__ a, long long n,
                              double dt2, int first) {
    const T c = (T)dt2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (first) uprev[i] = u[i] + (T)0.5 * c * a[i];
        else uprev[i] = (T)2 * u[i] - uprev[i] + c * a[i];
    }
}

// FP32 state: compensated update of (hi, lo); uprev / uprevlo receive u^{n+1}
__global__ void update_comp_kernel(const float* __restrict__ u, const float* __restrict__ ulo, float* __restrict__ uprev,
                                   float* __restrict__ uprevlo, const float* __restrict__ a, long long n, double dt2,
                                   int first) {
    const float c = (float)(first ? 0.5 * dt2 : dt2);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float hn, ln;
        leapfrog_comp(u[i], ulo[i], uprev[i], uprevlo[i], __fmul_rn(c, a[i]), first != 0, hn, ln);
        uprev[i] = hn;
        uprevlo[i] = ln;
    }
}

// lo: low parts of a compensated FP32 state (nullptr: none)
template <typename T>
__global__ void receiver_kernel(const T* __restrict__ u, const T* __restrict__ lo, const int* __restrict__ idx,
                                const double* __restrict__ w, double* traces, int nshot, int nrec, int nloc, long long N,
                                int nsteps_max, int step) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;   // (shot, receiver)
    if (k >= nshot * nrec) return;
    const int r = k / nrec, rec = k % nrec;
    double acc = 0.0;
    for (int l = 0; l < nloc; ++l) {
        const size_t o = (size_t)r * N + idx[rec * nloc + l];
        acc += w[rec * nloc + l] * ((double)u[o] + (lo ? (double)lo[o] : 0.0));
    }
    traces[((size_t)r * nrec + rec) * nsteps_max + step] = acc;
}

template <typename T>
__global__ void pulse_kernel(GeomParams gp, const double* __restrict__ greville, const double* __restrict__ centres,
                             double width, T* u, T* lo, int nshot, long long N) {
    const long long total = (long long)nshot * N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(k / N);
        long long i = k % N;
        double s[3] = {0, 0, 0}, sc[3] = {0, 0, 0}, x[3] = {0, 0, 0}, xc[3] = {0, 0, 0}, J[3][3];
        for (int d = 0; d < gp.dim; ++d) {
            s[d] = greville[i % gp.m];
            i /= gp.m;
            sc[d] = centres[r * gp.dim + d];
        }
        map_eval(gp, s, x, J);
        map_eval(gp, sc, xc, J);
        double d2 = 0.0;
        for (int d = 0; d < gp.dim; ++d) d2 += (x[d] - xc[d]) * (x[d] - xc[d]);
        const double v = exp(-d2 / (2.0 * width * width));
        u[k] = (T)v;
        if (lo) lo[k] = (T)(v - (double)(T)v);   // FP32: the rounding error of u^0 starts lo
    }
}

// Basis functions non-zero at parametric point s: global indices and values B_i(s).
void point_basis(const iga_space* s, const double* pt, int* idx, double* w) {
    const int p = s->p, P1 = p + 1;
    std::vector<double> vals[3];
    int first[3] = {0, 0, 0};
    std::vector<double> Nv(P1), dN(P1);
    for (int d = 0; d < s->dim; ++d) {
        const double x = std::min(1.0, std::max(0.0, pt[d]));
        const int mu = hb::find_span(s->knots, p, x);
        hb::basis_and_derivative(s->knots, p, mu, x, Nv.data(), dN.data());
        vals[d] = Nv;
        first[d] = mu - p;
    }
    int nloc = 1;
    for (int d = 0; d < s->dim; ++d) nloc *= P1;
    for (int l = 0; l < nloc; ++l) {
        int rem = l;
        long long gi = 0, stride = 1;
        double v = 1.0;
        for (int d = 0; d < s->dim; ++d) {
            const int a = rem % P1;
            rem /= P1;
            gi += (long long)(first[d] + a) * stride;
            stride *= s->m;
            v *= vals[d][a];
        }
        idx[l] = (int)gi;
        w[l] = v;
    }
}

template <int DIM, int P, typename T>
static int force_launch(const iga_wave* w, cudaStream_t st) {
    const iga_ops* ops = w->ops;
    const T* F = sizeof(T) == 8 ? (const T*)ops->fK64.ptr : (const T*)ops->fK32.ptr;
    const int N = (int)ops->N;
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, (long long)sms * 16));
    int r0 = 0;
    while (r0 < w->nshot) {
        const T* u = w->u.as<T>() + (size_t)r0 * N;
        T* b = w->b.as<T>() + (size_t)r0 * N;
        if (w->nshot - r0 >= 4) {
            force_kernel<DIM, P, T, 4><<<grid, 256, 0, st>>>(F, ops->pitch, u, b, N, ops->m);
            r0 += 4;
        } else {
            force_kernel<DIM, P, T, 1><<<grid, 256, 0, st>>>(F, ops->pitch, u, b, N, ops->m);
            r0 += 1;
        }
        IGA_LAUNCH_CHECK("force_kernel");
    }
    return IGA_OK;
}

template <typename T>
static int force_dispatch(const iga_wave* w, cudaStream_t st) {
    const int d = w->ops->dim, p = w->ops->p;
    if (d == 2 && p == 1) return force_launch<2, 1, T>(w, st);
    if (d == 2 && p == 2) return force_launch<2, 2, T>(w, st);
    if (d == 2 && p == 3) return force_launch<2, 3, T>(w, st);
    if (d == 3 && p == 1) return force_launch<3, 1, T>(w, st);
    if (d == 3 && p == 2) return force_launch<3, 2, T>(w, st);
    return fail(IGA_ERR_ARG, "unsupported (dim, p)");
}

double ricker(double t, double f0, double t0) {
    const double a = (3.14159265358979323846 * f0 * (t - t0)) * (3.14159265358979323846 * f0 * (t - t0));
    return (1.0 - 2.0 * a) * std::exp(-a);
}

// Extrapolated start of step n's mass solve, x = sum_{j<=k} c_j h_j with
// h_j = a^{n-1-j} and c_j = (-1)^j C(k+1, j+1) (the polynomial of degree k through
// the last k + 1 accelerations, evaluated one step ahead; exact for accelerations
// that are polynomials of that degree in time).  x may be the buffer of h_k (the
// oldest term), which every element reads before it is written; any rounding only
// moves the CG start.
template <typename T>
struct GuessTerms {
    const T* h[IGA_CG_GUESS_MAX + 1];
    float c[IGA_CG_GUESS_MAX + 1];
    int k;
};

__host__ __device__ inline float guess_coeff(int k, int j) {
    // (-1)^j C(k+1, j+1)
    double b = 1.0;
    for (int t = 1; t <= j + 1; ++t) b = b * (k + 2 - t) / t;
    return (float)((j & 1) ? -b : b);
}

template <typename T>
__global__ void guess_kernel(T* x, GuessTerms<T> g, long long tot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        T v = T(0);
        for (int j = 0; j <= g.k; ++j) v += (T)g.c[j] * g.h[j][i];
        x[i] = v;
    }
}

template <typename T>
static int wave_step_typed(iga_wave* w, int nsteps, cudaStream_t st) {
    const iga_ops* ops = w->ops;
    const long long N = ops->N;
    const long long tot = (long long)w->nshot * N;
    const int ugrid = (int)std::max<long long>(1, std::min<long long>((tot + 255) / 256, 152 * 16));
    long long* iter_acc = w->counters.as<long long>();
    int* status = (int*)(w->counters.as<char>() + 64);
    std::vector<cudaEvent_t> ev;
    if (w->timing) {
        ev.resize((size_t)4 * nsteps);
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    auto destroy_events = [&]() {
        for (auto& e : ev) cudaEventDestroy(e);
    };
    for (int s = 0; s < nsteps; ++s) {
        const int n = w->step;
        if (w->timing) cudaEventRecord(ev[4 * s + 0], st);
        int rc = force_dispatch<T>(w, st);
        if (w->timing) cudaEventRecord(ev[4 * s + 1], st);
        if (rc) {
            destroy_events();
            return rc;
        }
        if (w->desc.with_source) {
            const double amp = w->desc.src_amp * ricker(n * w->desc.dt, w->desc.f0, w->desc.t0);
            const int k = w->nshot * w->nloc;
            source_kernel<T><<<(k + 127) / 128, 128, 0, st>>>(w->b.as<T>(), w->src_idx.as<int>(), w->src_w.as<double>(),
                                                              w->nshot, w->nloc, N, amp);
            IGA_LAUNCH_CHECK("source_kernel");
        }
        // start of the solve: a^{n-1} in place (cg_guess 0, or n = 0 with a^{-1} = 0), else
        // the extrapolation from the last accelerations written into the oldest buffer
        const int K = w->desc.cg_guess;
        const bool extrap = K > 0 && n >= 1;
        if (extrap) {
            GuessTerms<T> g;
            g.k = std::min(K, n - 1);
            for (int j = 0; j <= g.k; ++j) {
                g.h[j] = j == 0 ? w->a.as<T>() : w->ah[j - 1].as<T>();
                g.c[j] = guess_coeff(g.k, j);
            }
            guess_kernel<T><<<ugrid, 256, 0, st>>>(w->ah[K - 1].as<T>(), g, tot);
            IGA_LAUNCH_CHECK("guess_kernel");
        }
        if (w->timing) cudaEventRecord(ev[4 * s + 2], st);
        void* xsol = extrap ? w->ah[K - 1].ptr : w->a.ptr;
        rc = mass_solve_impl(ops, w->dtype, w->b.ptr, xsol, w->N, w->nshot, w->desc.cg_rtol, w->desc.cg_max_it,
                             w->desc.solve_flags, nullptr, nullptr, st, w->work.ptr, w->work.bytes, iter_acc, status);
        if (extrap) {
            // a <- a^n, ah[j] <- a^{n-1-j}
            void* old_a = w->a.ptr;
            w->a.ptr = w->ah[K - 1].ptr;
            for (int j = K - 1; j > 0; --j) w->ah[j].ptr = w->ah[j - 1].ptr;
            w->ah[0].ptr = old_a;
        }
        if (w->timing) cudaEventRecord(ev[4 * s + 3], st);
        w->cg_solves += (w->nshot + 3) / 4;
        if (rc) {
            destroy_events();
            return rc;
        }
        if (sizeof(T) == 4) {
            update_comp_kernel<<<ugrid, 256, 0, st>>>(w->u.as<float>(), w->ulo.as<float>(), w->uprev.as<float>(),
                                                      w->uprevlo.as<float>(), w->a.as<float>(), tot,
                                                      w->desc.dt * w->desc.dt, n == 0 ? 1 : 0);
            IGA_LAUNCH_CHECK("update_comp_kernel");
            std::swap(w->ulo.ptr, w->uprevlo.ptr);
        } else {
            update_kernel<T><<<ugrid, 256, 0, st>>>(w->u.as<T>(), w->uprev.as<T>(), w->a.as<T>(), tot,
                                                    w->desc.dt * w->desc.dt, n == 0 ? 1 : 0);
            IGA_LAUNCH_CHECK("update_kernel");
        }
        std::swap(w->u.ptr, w->uprev.ptr);   // u <- u^{n+1}, uprev <- u^n
        if (w->nrec > 0) {
            const int k = w->nshot * w->nrec;
            receiver_kernel<T><<<(k + 127) / 128, 128, 0, st>>>(w->u.as<T>(), sizeof(T) == 4 ? w->ulo.as<T>() : nullptr,
                                                                w->rec_idx.as<int>(), w->rec_w.as<double>(),
                                                                w->traces.as<double>(), w->nshot, w->nrec, w->nloc, N,
                                                                w->desc.nsteps_max, n);
            IGA_LAUNCH_CHECK("receiver_kernel");
        }
        w->step += 1;
    }
    int st_h = 0;
    cudaError_t e = cudaMemcpyAsync(&st_h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && w->timing) {
        for (int s = 0; s < nsteps; ++s) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, ev[4 * s + 0], ev[4 * s + 1]);
            cudaEventElapsedTime(&b, ev[4 * s + 2], ev[4 * s + 3]);
            w->force_ms += a;
            w->cg_ms += b;
        }
    }
    destroy_events();
    if (e != cudaSuccess) return cuda_fail(e, "wave_step");
    if (st_h & (4 | 16)) return fail(IGA_ERR_TIMEOUT, "a bounded device wait timed out in a CG solve of wave_step");
    if (st_h & 1) return fail(IGA_ERR_NONFINITE, "CG breakdown in a solve of wave_step");
    if (st_h & 8) return fail(IGA_ERR_NOT_CONVERGED, "a CG solve in wave_step missed its tolerance");
    return IGA_OK;
}

// u^0 from the initial condition, u^{-1} and a^{-1} cleared, counters reset.
int wave_initial_state(iga_wave* w, cudaStream_t st) {
    const iga_space* s = w->ops->space;
    const size_t vb = (w->dtype == IGA_F64 ? 8 : 4) * (size_t)w->nshot * w->N;
    IGA_CUDA(cudaMemsetAsync(w->a.ptr, 0, vb, st));
    for (auto& h : w->ah)
        if (h.ptr) IGA_CUDA(cudaMemsetAsync(h.ptr, 0, vb, st));
    IGA_CUDA(cudaMemsetAsync(w->uprev.ptr, 0, vb, st));
    if (w->dtype == IGA_F32) {
        IGA_CUDA(cudaMemsetAsync(w->ulo.ptr, 0, vb, st));
        IGA_CUDA(cudaMemsetAsync(w->uprevlo.ptr, 0, vb, st));
    }
    IGA_CUDA(cudaMemsetAsync(w->traces.ptr, 0, w->traces.bytes, st));
    IGA_CUDA(cudaMemsetAsync(w->counters.ptr, 0, w->counters.bytes, st));
    if (w->desc.init_kind == IGA_INIT_GAUSS_PULSE) {
        const long long tot = (long long)w->nshot * w->N;
        const int grid = (int)std::min<long long>((tot + 255) / 256, 152 * 16);
        if (w->dtype == IGA_F64)
            pulse_kernel<double><<<grid, 256, 0, st>>>(s->gp, w->greville.as<double>(), w->centres.as<double>(),
                                                       w->desc.pulse_width, w->u.as<double>(), nullptr, w->nshot,
                                                       w->N);
        else
            pulse_kernel<float><<<grid, 256, 0, st>>>(s->gp, w->greville.as<double>(), w->centres.as<double>(),
                                                      w->desc.pulse_width, w->u.as<float>(), w->ulo.as<float>(),
                                                      w->nshot, w->N);
        IGA_LAUNCH_CHECK("pulse_kernel");
    } else {
        IGA_CUDA(cudaMemsetAsync(w->u.ptr, 0, vb, st));
    }
    w->step = 0;
    w->cg_solves = 0;
    w->cg_ms = w->force_ms = 0.0;
    // cfl_check 1: estimate at create and at every reset; 2: at create only (a reset
    // re-binds operators of the same problem)
    if (w->desc.cfl_check == 1 || (w->desc.cfl_check == 2 && w->lam_max == 0.0)) {
        int rc = spectrum_impl(w->ops, IGA_F32, 40, &w->lam_min, &w->lam_max, st);
        if (rc) return rc;
    }
    return IGA_OK;
}

int wave_step_impl(iga_wave* w, int nsteps, cudaStream_t st) {
    return w->dtype == IGA_F64 ? wave_step_typed<double>(w, nsteps, st) : wave_step_typed<float>(w, nsteps, st);
}

}  // namespace iga

using namespace iga;

extern "C" int iga_wave_reset(iga_wave* w, const iga_ops* ops, void* stream) {
    if (!w || !ops) return fail(IGA_ERR_ARG, "null argument");
    if (ops->N != w->N || ops->space->dim != w->ops->space->dim || ops->p != w->ops->p)
        return fail(IGA_ERR_ARG, "ops must have the wave's space size and degree");
    w->ops = ops;
    return wave_initial_state(w, (cudaStream_t)stream);
}

extern "C" int iga_wave_set_timing(iga_wave* w, int on) {
    if (!w) return fail(IGA_ERR_ARG, "null argument");
    w->timing = on ? 1 : 0;
    return IGA_OK;
}

extern "C" int iga_wave_stats_get(const iga_wave* w, iga_wave_stats* out) {
    if (!w || !out) return fail(IGA_ERR_ARG, "null argument");
    long long it = 0;
    IGA_CUDA(cudaDeviceSynchronize());
    IGA_CUDA(cudaMemcpy(&it, w->counters.ptr, sizeof(long long), cudaMemcpyDeviceToHost));
    out->steps = w->step;
    out->cg_iterations = it;
    out->cg_solves = w->cg_solves;
    out->cg_ms = w->cg_ms;
    out->force_ms = w->force_ms;
    out->lambda_min = w->lam_min;
    out->lambda_max = w->lam_max;
    return IGA_OK;
}

extern "C" int iga_wave_create(const iga_ops* ops, const iga_wave_desc* desc, iga_wave** out) {
    if (!ops || !desc || !out) return fail(IGA_ERR_ARG, "null argument");
    *out = nullptr;
    const iga_wave_desc& d = *desc;
    if (d.nshot < 1) return fail(IGA_ERR_ARG, "nshot must be >= 1");
    if (d.dtype != IGA_F32 && d.dtype != IGA_F64) return fail(IGA_ERR_ARG, "bad dtype");
    if (!(d.dt > 0.0)) return fail(IGA_ERR_ARG, "dt must be > 0");
    if (d.nsteps_max < 0 || d.nrec < 0 || d.cg_max_it < 1 || !(d.cg_rtol >= 0.0))
        return fail(IGA_ERR_ARG, "bad nsteps_max / nrec / cg parameters");
    if (d.init_kind == IGA_INIT_GAUSS_PULSE && (!d.pulse_centre || !(d.pulse_width > 0)))
        return fail(IGA_ERR_ARG, "GAUSS_PULSE needs centres and a positive width");
    if (d.with_source && !d.src_pos) return fail(IGA_ERR_ARG, "source positions missing");
    if (d.cg_guess < 0 || d.cg_guess > IGA_CG_GUESS_MAX) return fail(IGA_ERR_ARG, "cg_guess must be in 0..6");
    if (d.nrec > 0 && !d.rec_pos) return fail(IGA_ERR_ARG, "receiver positions missing");
    const iga_space* s = ops->space;
    iga_wave* w = new (std::nothrow) iga_wave();
    if (!w) return fail(IGA_ERR_OOM, "host allocation failed");
    w->ops = ops;
    w->desc = d;
    w->desc.pulse_centre = w->desc.src_pos = w->desc.rec_pos = nullptr;
    w->dtype = d.dtype;
    w->nshot = d.nshot;
    w->nrec = d.nrec;
    w->N = ops->N;
    w->step = 0;
    w->nloc = 1;
    for (int k = 0; k < s->dim; ++k) w->nloc *= s->p + 1;
    const size_t es = d.dtype == IGA_F64 ? 8 : 4;
    const size_t vb = es * (size_t)d.nshot * ops->N;
    auto bail = [&](int rc) {
        delete w;
        return rc;
    };
    int rc = w->u.alloc(vb);
    if (!rc) rc = w->uprev.alloc(vb);
    if (!rc) rc = w->a.alloc(vb);
    if (!rc) rc = w->b.alloc(vb);
    if (!rc) rc = w->traces.alloc(sizeof(double) * std::max<size_t>(1, (size_t)d.nshot * d.nrec * d.nsteps_max));
    if (!rc) rc = w->counters.alloc(128);
    if (!rc) rc = w->work.alloc(mass_solve_work_bytes(ops, d.dtype, d.nshot));
    if (!rc && d.dtype == IGA_F32) rc = w->ulo.alloc(vb);
    if (!rc && d.dtype == IGA_F32) rc = w->uprevlo.alloc(vb);
    for (int j = 0; j < d.cg_guess && !rc; ++j) rc = w->ah[j].alloc(vb);
    if (rc) return bail(rc);
    // source / receiver tables
    std::vector<int> idx;
    std::vector<double> wt;
    if (d.with_source) {
        idx.assign((size_t)d.nshot * w->nloc, 0);
        wt.assign(idx.size(), 0.0);
        for (int r = 0; r < d.nshot; ++r)
            point_basis(s, d.src_pos + (size_t)r * s->dim, &idx[(size_t)r * w->nloc], &wt[(size_t)r * w->nloc]);
    } else {
        idx.assign(1, 0);
        wt.assign(1, 0.0);
    }
    if ((rc = w->src_idx.alloc(sizeof(int) * idx.size())) || (rc = w->src_w.alloc(sizeof(double) * wt.size())))
        return bail(rc);
    cudaMemcpy(w->src_idx.ptr, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(w->src_w.ptr, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice);
    idx.assign((size_t)std::max(1, d.nrec) * w->nloc, 0);
    wt.assign(idx.size(), 0.0);
    for (int k = 0; k < d.nrec; ++k)
        point_basis(s, d.rec_pos + (size_t)k * s->dim, &idx[(size_t)k * w->nloc], &wt[(size_t)k * w->nloc]);
    if ((rc = w->rec_idx.alloc(sizeof(int) * idx.size())) || (rc = w->rec_w.alloc(sizeof(double) * wt.size())))
        return bail(rc);
    cudaMemcpy(w->rec_idx.ptr, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(w->rec_w.ptr, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice);
    if (d.init_kind == IGA_INIT_GAUSS_PULSE) {
        std::vector<double> gv(s->m);
        for (int k = 0; k < s->m; ++k) {   // Greville abscissae: mean of knots k+1 .. k+p
            double acc = 0.0;
            for (int l = 1; l <= s->p; ++l) acc += s->knots[k + l];
            gv[k] = acc / s->p;
        }
        if ((rc = w->greville.alloc(sizeof(double) * gv.size())) ||
            (rc = w->centres.alloc(sizeof(double) * d.nshot * s->dim)))
            return bail(rc);
        cudaMemcpy(w->greville.ptr, gv.data(), sizeof(double) * gv.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(w->centres.ptr, d.pulse_centre, sizeof(double) * d.nshot * s->dim, cudaMemcpyHostToDevice);
    }
    if ((rc = wave_initial_state(w, 0))) return bail(rc);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(cuda_fail(e, "wave_create"));
    *out = w;
    return IGA_OK;
}

extern "C" int iga_wave_destroy(iga_wave* w) {
    delete w;
    return IGA_OK;
}

extern "C" int iga_wave_step(iga_wave* w, int nsteps, void* stream) {
    if (!w) return fail(IGA_ERR_ARG, "null argument");
    if (nsteps < 0) return fail(IGA_ERR_ARG, "nsteps must be >= 0");
    if (w->nrec > 0 && w->step + nsteps > w->desc.nsteps_max) return fail(IGA_ERR_ARG, "trace buffer would overflow");
    if (nsteps == 0) return IGA_OK;
    if (w->desc.cfl_check && w->desc.dt * std::sqrt(1.02 * w->lam_max) >= 2.0)
        return fail(IGA_ERR_ARG, "dt exceeds the leapfrog stability limit 2/sqrt(lambda_max)");
    return wave_step_impl(w, nsteps, (cudaStream_t)stream);
}

extern "C" int iga_wave_get_state(const iga_wave* w, void* u, void* u_prev, void* stream) {
    if (!w || !u) return fail(IGA_ERR_ARG, "null argument");
    const size_t vb = (w->dtype == IGA_F64 ? 8 : 4) * (size_t)w->nshot * w->N;
    IGA_CUDA(cudaMemcpyAsync(u, w->u.ptr, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    if (u_prev) IGA_CUDA(cudaMemcpyAsync(u_prev, w->uprev.ptr, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return IGA_OK;
}

extern "C" int iga_wave_traces(const iga_wave* w, double* host_dst, int* nsteps_done) {
    if (!w) return fail(IGA_ERR_ARG, "null argument");
    if (nsteps_done) *nsteps_done = w->step;
    if (!host_dst || w->nrec == 0) return IGA_OK;
    IGA_CUDA(cudaDeviceSynchronize());
    std::vector<double> all((size_t)w->nshot * w->nrec * std::max(1, w->desc.nsteps_max));
    IGA_CUDA(cudaMemcpy(all.data(), w->traces.ptr, sizeof(double) * all.size(), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < (size_t)w->nshot * w->nrec; ++k)
        std::memcpy(host_dst + k * w->step, all.data() + k * w->desc.nsteps_max, sizeof(double) * w->step);
    return IGA_OK;
}

extern "C" int iga_wave_cg_iterations(const iga_wave* w, long long* total) {
    if (!w || !total) return fail(IGA_ERR_ARG, "null argument");
    IGA_CUDA(cudaDeviceSynchronize());
    IGA_CUDA(cudaMemcpy(total, w->counters.ptr, sizeof(long long), cudaMemcpyDeviceToHost));
    return IGA_OK;
}
