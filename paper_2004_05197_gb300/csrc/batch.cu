// Batched persistent leapfrog: several problems (a mesh with all its shots as
// right-hand sides), every time step of all of them in one cooperative launch.
//
// The grid is split into partitions, one per problem (block ranges chosen by
// the tuner, see iga_batch_tune).  A partition synchronises only its own
// blocks (bounded partition barrier), so problems of uneven size run their own
// CG iteration counts without waiting for each other.  Per step n (u^n lives in
// U[n mod 2]):
//   force + source  b_r = -K~ u_r + amp ricker(n dt) S_r      (S_r: B_i(s_src,r), dense)
//   barrier
//   Jacobi-PCG, Chronopoulos-Gear form, all shots of the problem at once
//   update          u^{n+1} = 2u^n - u^{n-1} + dt^2 a^n  (n = 0: u^0 + dt^2/2 a^0) into U[(n+1) mod 2]
//   barrier, receivers of u^{n+1}
// FP32 fields and state, FP64 residual and reductions (as mass_solve).  The CG
// start of step n follows the wave's cg_guess K (a^{n-1}, or the polynomial
// extrapolation in time through the accelerations in A[(n-1..n-1-K) % (K+1)]).
// The step counter lives in device memory, so one captured graph of the launch
// can be replayed for consecutive step ranges.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cg.cuh"
#include "iga_internal.cuh"
#include "leapfrog.cuh"
#include "stencil.cuh"

namespace iga {

constexpr int kBThreads = 512;
constexpr int kBWarps = kBThreads / 32;
constexpr int kBMaxProbs = 16;
template <int R>
constexpr int kBUnroll = R >= 16 ? 1 : 2;   // fields in flight per thread (registers bound R = 16)

struct BatchProb {
    const float* FK;
    const float* FM;
    const float* dinv;
    long long pitch;
    int N, m;
    float* U[2];        // u^n in U[n % 2]
    float* L[2];        // low parts of the compensated state, alongside U
    float* A[IGA_CG_GUESS_MAX + 1];   // CG solutions: a^n in A[n % ring]
    int guess;          // CG start order K (the wave's cg_guess): 0 = a^{n-1} in place
    int ring;           // K + 1 acceleration buffers (1 when K = 0)
    float* b;           // right-hand side
    double* r;          // CG residual (FP64)
    float* cu;          // D^-1 r
    float* cw;          // M~ cu
    float* cp;
    float* cs;
    const float* S;     // dense source weights [R][ld]
    long long ld;       // leading dimension of every [R][.] vector
    const int* rec_idx;
    const double* rec_w;
    int nrec, nloc;
    double* traces;     // [R][nrec][nsteps_max]
    int nsteps_max;
    double dt, f0, t0, amp, rtol;
    int max_it;
    double* partials;   // [nb][10 R]
    unsigned* bar;      // [2]
    int* step;          // global step counter of this problem
    int b0, nb;         // block range of the partition
    long long* iter_acc;
    int* status;        // bit 8: a solve missed rtol
    long long* clk;     // [2]: clock at partition start / end (tuner)
};

__device__ __forceinline__ double ricker_dev(double t, double f0, double t0) {
    const double a = (3.14159265358979323846 * f0 * (t - t0)) * (3.14159265358979323846 * f0 * (t - t0));
    return (1.0 - 2.0 * a) * exp(-a);
}

template <int DIM, int P, int R>
__global__ void __launch_bounds__(kBThreads, 1) batch_kernel(const BatchProb* __restrict__ probs, int nprob,
                                                             int nsteps, int* err) {
    __shared__ BatchProb pb;
    __shared__ int sdlK[StencilShape<DIM, P>::T0];
    __shared__ double wsum[kBWarps * 3 * R];
    __shared__ double red[3 * R], red2[R];
    __shared__ double gam[R], rr[R], bnorm[R], alpha[R], beta[R];
    __shared__ int active[R], iters[R];
    if (threadIdx.x == 0) {
        int k = 0;
        while (k + 1 < nprob && (int)blockIdx.x >= probs[k + 1].b0) ++k;
        pb = probs[k];
    }
    __syncthreads();
    const BatchProb& q = pb;
    const int lb = blockIdx.x - q.b0, nb = q.nb;
    const int row0 = (int)(((long long)q.N * lb) / nb), row1 = (int)(((long long)q.N * (lb + 1)) / nb);
    fill_delta_table<DIM, P>(sdlK, q.m);
    const int dmax = max_delta<DIM, P>(q.m);
    const int n0 = *((volatile int*)q.step);
    constexpr int S10 = 10 * R;
    double part[3 * R];
    if (lb == 0 && threadIdx.x == 0) q.clk[0] = clock64();
    for (int s = 0; s < nsteps; ++s) {
        const int n = n0 + s;
        const float* cur = q.U[n & 1];
        float* nxt = q.U[(n + 1) & 1];   // holds u^{n-1}; receives u^{n+1}
        const float* curlo = q.L[n & 1];
        float* nxtlo = q.L[(n + 1) & 1];
        float* const qa = q.A[n % q.ring];   // receives a^n; holds the CG start
        // ---- CG start extrapolated in time, sum_j (-1)^j C(k+1, j+1) a^{n-1-j}, into
        // A[n % ring] (which held a^{n-1-K}, the oldest term); the force phase's
        // barrier orders it before the mass apply of CG init 1
        if (q.guess > 0 && n >= 1) {
            const int k = min(q.guess, n - 1);
            float c[IGA_CG_GUESS_MAX + 1];
            const float* h[IGA_CG_GUESS_MAX + 1];
            for (int j = 0; j <= k; ++j) {
                double bc = 1.0;
                for (int t = 1; t <= j + 1; ++t) bc = bc * (k + 2 - t) / t;
                c[j] = (float)((j & 1) ? -bc : bc);
                h[j] = q.A[(n - 1 - j + q.ring) % q.ring];
            }
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const long long o = (long long)r * q.ld + i;
                    float v = 0.f;
                    for (int j = 0; j <= k; ++j) v += c[j] * h[j][o];
                    qa[o] = v;
                }
        }
        // ---- force + source
        {
            const float amp = (float)(q.amp * ricker_dev(n * q.dt, q.f0, q.t0));
            const PlainLoadB<float> ld{cur, q.ld};   // u^n was written by other blocks of this launch
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
                float acc[R], own[R];
                if (i >= dmax && i < q.N - dmax)
                    stencil_row_interior<DIM, P, float, false, R, kBUnroll<R>>(q.FK, q.pitch, ld, i, sdlK, acc, own);
                else
                    stencil_row<DIM, P, float, false, R, kBUnroll<R>>(q.FK, q.pitch, ld, i, q.N, q.m, acc, own);
#pragma unroll
                for (int r = 0; r < R; ++r) q.b[r * q.ld + i] = fmaf(amp, q.S[r * q.ld + i], -acc[r]);
            }
        }
        if (!grid_barrier(q.bar, err, nb)) return;
        // ---- CG init 1: r = b - M~a, cu = D^-1 r
        {
            DotAcc<float> dot[3 * R];
            const PlainLoadB<float> ld{qa, q.ld};
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
                float acc[R], own[R];
                if (i >= dmax && i < q.N - dmax)
                    stencil_row_interior<DIM, P, float, true, R, kBUnroll<R>>(q.FM, q.pitch, ld, i, sdlK, acc, own);
                else
                    stencil_row<DIM, P, float, true, R, kBUnroll<R>>(q.FM, q.pitch, ld, i, q.N, q.m, acc, own);
                const float di = q.dinv[i];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const long long o = (long long)r * q.ld + i;
                    const float bi = q.b[o];
                    const double ri = (double)bi - (double)acc[r];   // FP64 residual
                    const float rt = (float)ri;
                    const float ui = di * rt;
                    q.r[o] = ri;
                    q.cu[o] = ui;
                    dot[3 * r].add(rt, ui);
                    dot[3 * r + 1].add(rt, rt);
                    dot[3 * r + 2].add(bi, bi);
                }
            }
            for (int k = 0; k < 3 * R; ++k) part[k] = dot[k].value();
            block_sum<3 * R, kBWarps>(part, wsum, red);
            if (threadIdx.x < 3 * R) q.partials[(size_t)lb * S10 + 6 * R + threadIdx.x] = red[threadIdx.x];
            if (threadIdx.x < R) active[threadIdx.x] = 1;
        }
        if (!grid_barrier(q.bar, err, nb)) return;
        // ---- phase 2 (init): cw = M~ cu
        auto phase2 = [&]() {
            DotAcc<float> dot[R];
            const PlainLoadB<float> ld{q.cu, q.ld};
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
                float acc[R], own[R];
                if (i >= dmax && i < q.N - dmax)
                    stencil_row_interior<DIM, P, float, true, R, kBUnroll<R>>(q.FM, q.pitch, ld, i, sdlK, acc, own);
                else
                    stencil_row<DIM, P, float, true, R, kBUnroll<R>>(q.FM, q.pitch, ld, i, q.N, q.m, acc, own);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (!active[r]) continue;
                    q.cw[(long long)r * q.ld + i] = acc[r];
                    dot[r].add(own[r], acc[r]);
                }
            }
            for (int k = 0; k < R; ++k) part[k] = dot[k].value();
            block_sum<R, kBWarps>(part, wsum, red);
            if (threadIdx.x < R) q.partials[(size_t)lb * S10 + 4 * R + threadIdx.x] = red[threadIdx.x];
        };
        phase2();
        if (!grid_barrier(q.bar, err, nb)) return;
        grid_sum_b<3 * R>(q.partials, nb, S10, 6 * R, red);
        grid_sum_b<R>(q.partials, nb, S10, 4 * R, red2);
        if (threadIdx.x < R) {
            const int r = threadIdx.x;
            gam[r] = red[3 * r];
            rr[r] = red[3 * r + 1];
            bnorm[r] = sqrt(red[3 * r + 2]);
            beta[r] = 0.0;
            iters[r] = 0;
            active[r] = bnorm[r] > 0.0 && !(q.rtol > 0.0 && sqrt(rr[r]) <= q.rtol * bnorm[r]);
            const double d = red2[r];
            if (active[r] && (!(d > 0.0) || !isfinite(d))) {
                active[r] = 0;
                atomicOr(err, 1);
            }
            alpha[r] = active[r] ? gam[r] / d : 0.0;
        }
        __syncthreads();
        for (int r = 0; r < R; ++r)
            if (!(bnorm[r] > 0.0))
                for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) qa[(long long)r * q.ld + i] = 0.f;
        // ---- CG iterations
        for (int it = 0; it < q.max_it; ++it) {
            bool any = false;
            for (int r = 0; r < R; ++r) any = any || active[r];
            if (!any) break;
            const int off1 = (it & 1) * 2 * R;
            DotAcc<float> dot[2 * R];
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
                const float di = q.dinv[i];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (!active[r]) continue;
                    const long long o = (long long)r * q.ld + i;
                    const float be = (float)beta[r], al = (float)alpha[r];
                    const float pi = q.cu[o] + be * q.cp[o];
                    const float si = q.cw[o] + be * q.cs[o];
                    q.cp[o] = pi;
                    q.cs[o] = si;
                    qa[o] = qa[o] + al * pi;
                    const double ri = q.r[o] - alpha[r] * (double)si;   // FP64 residual
                    const float rt = (float)ri;
                    const float ui = di * rt;
                    q.r[o] = ri;
                    q.cu[o] = ui;
                    dot[2 * r].add(rt, ui);
                    dot[2 * r + 1].add(rt, rt);
                }
            }
            for (int k = 0; k < 2 * R; ++k) part[k] = dot[k].value();
            block_sum<2 * R, kBWarps>(part, wsum, red);
            if (threadIdx.x < 2 * R) q.partials[(size_t)lb * S10 + off1 + threadIdx.x] = red[threadIdx.x];
            if (!grid_barrier(q.bar, err, nb)) return;
            phase2();
            if (!grid_barrier(q.bar, err, nb)) return;
            grid_sum_b<2 * R>(q.partials, nb, S10, off1, red);
            grid_sum_b<R>(q.partials, nb, S10, 4 * R, red2);
            if (threadIdx.x < R) {
                const int r = threadIdx.x;
                if (active[r]) {
                    int brk = 0, act = 1;
                    double rro = rr[r];
                    cg_scalars(red[2 * r], red[2 * r + 1], red2[r], q.rtol, bnorm[r], gam[r], alpha[r], beta[r], act,
                               iters[r], rro, &brk);
                    active[r] = act;
                    rr[r] = rro;
                    if (brk && lb == 0) atomicOr(err, 1);
                }
            }
            __syncthreads();
        }
        if (lb == 0 && threadIdx.x < R) {
            const int r = threadIdx.x;
            atomicAdd((unsigned long long*)q.iter_acc, (unsigned long long)iters[r]);
            if (q.rtol > 0.0 && bnorm[r] > 0.0 && sqrt(rr[r]) > q.rtol * bnorm[r]) atomicOr(q.status, 8);
        }
        // ---- leapfrog update into U[(n+1) mod 2]
        {
            const float dt2 = (float)(q.dt * q.dt);
            for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const long long o = (long long)r * q.ld + i;
                    float hn, ln;
                    leapfrog_comp(cur[o], curlo[o], nxt[o], nxtlo[o], __fmul_rn(n == 0 ? 0.5f * dt2 : dt2, qa[o]),
                                  n == 0, hn, ln);
                    nxt[o] = hn;
                    nxtlo[o] = ln;
                }
            }
        }
        if (!grid_barrier(q.bar, err, nb)) return;
        // ---- receivers of u^{n+1} (first block of the partition)
        if (lb == 0 && q.nrec > 0 && n < q.nsteps_max) {
            for (int k = threadIdx.x; k < R * q.nrec; k += blockDim.x) {
                const int r = k / q.nrec, rec = k % q.nrec;
                double acc = 0.0;
                for (int l = 0; l < q.nloc; ++l) {
                    const long long o = (long long)r * q.ld + q.rec_idx[rec * q.nloc + l];
                    acc += q.rec_w[rec * q.nloc + l] * ((double)nxt[o] + (double)nxtlo[o]);
                }
                q.traces[((size_t)r * q.nrec + rec) * q.nsteps_max + n] = acc;
            }
        }
    }
    if (lb == 0 && threadIdx.x == 0) {
        q.clk[1] = clock64();
        *q.step = n0 + nsteps;   // every block of the partition has read the counter (barriers since)
    }
}

}  // namespace iga

// ---------------------------------------------------------------------------- host
struct iga_batch {
    std::vector<iga_wave*> waves;
    int nprob = 0, R = 0, dim = 0, p = 0;
    int total_blocks = 0;
    std::vector<double> weights;          // partition weights (tuner)
    std::vector<int> b0, nb;
    iga::DevBuf probs, work, counters;    // BatchProb[], CG vectors, step / status / clocks
    std::vector<iga::BatchProb> hp;
    cudaGraphExec_t graph = nullptr;
    int graph_nsteps = -1;
    ~iga_batch() {
        if (graph) cudaGraphExecDestroy(graph);
    }
};

namespace iga {

template <int DIM, int P, int R>
static const void* batch_fn() {
    return (const void*)batch_kernel<DIM, P, R>;
}

static const void* pick_batch(int dim, int p, int R) {
#define IGA_BATCH_CASE(DD, PP)                                        \
    if (dim == DD && p == PP) {                                       \
        if (R == 1) return batch_fn<DD, PP, 1>();                     \
        if (R == 4) return batch_fn<DD, PP, 4>();                     \
        if (R == 8) return batch_fn<DD, PP, 8>();                     \
        if (R == 16) return batch_fn<DD, PP, 16>();                   \
    }
    IGA_BATCH_CASE(2, 2)
    IGA_BATCH_CASE(2, 3)
    IGA_BATCH_CASE(3, 2)
#undef IGA_BATCH_CASE
    return nullptr;
}

// Block ranges from the weights: every problem at least one block.
static void split_blocks(iga_batch* b) {
    double tot = 0.0;
    for (double w : b->weights) tot += w;
    b->b0.assign(b->nprob, 0);
    b->nb.assign(b->nprob, 1);
    int left = b->total_blocks - b->nprob;
    std::vector<double> ideal(b->nprob);
    int used = 0;
    for (int k = 0; k < b->nprob; ++k) {
        ideal[k] = left * b->weights[k] / tot;
        const int extra = (int)std::floor(ideal[k]);
        b->nb[k] += extra;
        used += extra;
    }
    while (used < left) {   // largest remainders
        int best = 0;
        double bestr = -1.0;
        for (int k = 0; k < b->nprob; ++k) {
            const double rem = ideal[k] - std::floor(ideal[k]);
            if (rem > bestr) {
                bestr = rem;
                best = k;
            }
        }
        b->nb[best] += 1;
        ideal[best] = std::floor(ideal[best]);
        ++used;
    }
    int s = 0;
    for (int k = 0; k < b->nprob; ++k) {
        b->b0[k] = s;
        s += b->nb[k];
    }
}

static int upload_probs(iga_batch* b, cudaStream_t st) {
    split_blocks(b);
    for (int k = 0; k < b->nprob; ++k) {
        b->hp[k].b0 = b->b0[k];
        b->hp[k].nb = b->nb[k];
    }
    IGA_CUDA(cudaMemcpyAsync(b->probs.ptr, b->hp.data(), sizeof(BatchProb) * b->nprob, cudaMemcpyHostToDevice, st));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_nsteps = -1;
    }
    return IGA_OK;
}

// counters: [0] error word, [16 + 4k .. 16 + 4k + 3] step / iterations / status of problem k,
// then 2 clocks per problem
static int* batch_err(iga_batch* b) { return (int*)b->counters.as<long long>(); }

static int ring_of(const iga_wave* w) { return w->desc.cg_guess + 1; }
static int modr(int n, int r) { return ((n % r) + r) % r; }

// The wave keeps a^{step-1} in a and a^{step-2-j} in ah[j] (j < cg_guess); the
// kernel finds a^n in A[n % ring].
static void accel_buffers(const iga_wave* w, float* A[IGA_CG_GUESS_MAX + 1]) {
    const int R = ring_of(w);
    for (int j = 0; j <= IGA_CG_GUESS_MAX; ++j) A[j] = nullptr;
    A[modr(w->step - 1, R)] = w->a.as<float>();
    for (int j = 0; j + 1 < R; ++j) A[modr(w->step - 2 - j, R)] = w->ah[j].as<float>();
}

// After steps ran in the kernel: the wave's u / uprev / a views for its new step.
static void wave_views(iga_wave* w, const BatchProb& q) {
    w->u.ptr = q.U[w->step & 1];
    w->uprev.ptr = q.U[(w->step + 1) & 1];
    w->ulo.ptr = q.L[w->step & 1];
    w->uprevlo.ptr = q.L[(w->step + 1) & 1];
    const int R = ring_of(w);
    w->a.ptr = q.A[modr(w->step - 1, R)];
    for (int j = 0; j + 1 < R; ++j) w->ah[j].ptr = q.A[modr(w->step - 2 - j, R)];
}

// Bind U[n % 2] and A[n % 3] to the waves' current buffers and load the step
// counters (a wave may have been reset or stepped on its own since the last launch).
static int batch_sync(iga_batch* b, cudaStream_t st) {
    bool dirty = false;
    for (int k = 0; k < b->nprob; ++k) {
        iga_wave* w = b->waves[k];
        BatchProb& q = b->hp[k];
        float* A[IGA_CG_GUESS_MAX + 1];
        accel_buffers(w, A);
        for (int j = 0; j <= IGA_CG_GUESS_MAX; ++j)
            if (A[j] != q.A[j]) {
                q.A[j] = A[j];
                dirty = true;
            }
        if (q.U[w->step & 1] != w->u.ptr || q.U[(w->step + 1) & 1] != w->uprev.ptr ||
            q.L[w->step & 1] != w->ulo.ptr || q.L[(w->step + 1) & 1] != w->uprevlo.ptr) {
            q.U[w->step & 1] = w->u.as<float>();
            q.U[(w->step + 1) & 1] = w->uprev.as<float>();
            q.L[w->step & 1] = w->ulo.as<float>();
            q.L[(w->step + 1) & 1] = w->uprevlo.as<float>();
            dirty = true;
        }
        IGA_CUDA(cudaMemcpyAsync(q.step, &w->step, sizeof(int), cudaMemcpyHostToDevice, st));
        IGA_CUDA(cudaMemsetAsync((long long*)q.step + 2, 0, sizeof(long long), st));   // status
    }
    IGA_CUDA(cudaMemsetAsync(b->counters.ptr, 0, sizeof(long long), st));             // error word
    if (dirty) return upload_probs(b, st);
    return IGA_OK;
}

static int batch_launch(iga_batch* b, int nsteps, cudaStream_t st) {
    int* err = batch_err(b);
    const void* fn = pick_batch(b->dim, b->p, b->R);
    const BatchProb* probs = b->probs.as<BatchProb>();
    int nprob = b->nprob;
    void* args[] = {(void*)&probs, (void*)&nprob, (void*)&nsteps, (void*)&err};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, b->total_blocks, kBThreads, args, 0, st);
    count_launch();
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(batch)");
    return IGA_OK;
}

}  // namespace iga

using namespace iga;

extern "C" int iga_batch_create(int nprob, iga_wave* const* waves, iga_batch** out) {
    if (!waves || !out || nprob < 1 || nprob > kBMaxProbs) return fail(IGA_ERR_ARG, "need 1..16 waves");
    *out = nullptr;
    iga_batch* b = new (std::nothrow) iga_batch();
    if (!b) return fail(IGA_ERR_OOM, "host allocation failed");
    auto bail = [&](int rc) {
        delete b;
        return rc;
    };
    b->nprob = nprob;
    b->waves.assign(waves, waves + nprob);
    b->R = waves[0]->nshot;
    b->dim = waves[0]->ops->dim;
    b->p = waves[0]->ops->p;
    for (int k = 0; k < nprob; ++k) {
        const iga_wave* w = waves[k];
        if (!w) return bail(fail(IGA_ERR_ARG, "null wave"));
        if (w->dtype != IGA_F32) return bail(fail(IGA_ERR_ARG, "batched waves are FP32"));
        if (w->nshot != b->R || w->ops->dim != b->dim || w->ops->p != b->p)
            return bail(fail(IGA_ERR_ARG, "batched waves need the same nshot, dim and p"));
    }
    if (!pick_batch(b->dim, b->p, b->R)) return bail(fail(IGA_ERR_ARG, "unsupported (dim, p, nshot) for a batch"));
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pick_batch(b->dim, b->p, b->R), kBThreads, 0);
    b->total_blocks = sms * std::max(1, per);
    if (b->total_blocks < nprob) return bail(fail(IGA_ERR_ARG, "more problems than co-resident blocks"));
    // CG vectors per problem: r (FP64) + cu, cw, cp, cs (FP32) + dense source weights, plus partials
    size_t bytes = 0;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    for (int k = 0; k < nprob; ++k) {
        const size_t v = (size_t)b->R * waves[k]->N;
        bytes += up(8 * v) + 5 * up(4 * v) + up(sizeof(double) * (size_t)b->total_blocks * 10 * b->R) + up(64);
    }
    int rc = b->work.alloc(bytes);
    if (!rc) rc = b->counters.alloc(sizeof(long long) * (16 + 4 * nprob) + 4096);
    if (!rc) rc = b->probs.alloc(sizeof(BatchProb) * nprob);
    if (rc) return bail(rc);
    cudaMemset(b->work.ptr, 0, b->work.bytes);
    cudaMemset(b->counters.ptr, 0, b->counters.bytes);
    char* wp = b->work.as<char>();
    auto take = [&](size_t n) {
        void* o = wp;
        wp += up(n);
        return o;
    };
    long long* cbase = b->counters.as<long long>() + 16;   // [0..15]: err, spare
    b->hp.resize(nprob);
    for (int k = 0; k < nprob; ++k) {
        iga_wave* w = waves[k];
        const iga_ops* ops = w->ops;
        const size_t v = (size_t)b->R * w->N;
        BatchProb& q = b->hp[k];
        std::memset(&q, 0, sizeof(q));
        q.FK = ops->fK32.as<float>();
        q.FM = ops->fM32.as<float>();
        q.dinv = ops->dinv32.as<float>();
        q.pitch = ops->pitch;
        q.N = (int)w->N;
        q.m = ops->m;
        // u^n of the wave is in U[n % 2]
        q.U[w->step & 1] = w->u.as<float>();
        q.U[(w->step + 1) & 1] = w->uprev.as<float>();
        q.L[w->step & 1] = w->ulo.as<float>();
        q.L[(w->step + 1) & 1] = w->uprevlo.as<float>();
        accel_buffers(w, q.A);
        q.guess = w->desc.cg_guess;
        q.ring = ring_of(w);
        q.b = w->b.as<float>();
        q.r = (double*)take(8 * v);
        q.cu = (float*)take(4 * v);
        q.cw = (float*)take(4 * v);
        q.cp = (float*)take(4 * v);
        q.cs = (float*)take(4 * v);
        float* S = (float*)take(4 * v);
        q.S = S;
        q.ld = w->N;
        q.rec_idx = w->rec_idx.as<int>();
        q.rec_w = w->rec_w.as<double>();
        q.nrec = w->nrec;
        q.nloc = w->nloc;
        q.traces = w->traces.as<double>();
        q.nsteps_max = w->desc.nsteps_max;
        q.dt = w->desc.dt;
        q.f0 = w->desc.f0;
        q.t0 = w->desc.t0;
        q.amp = w->desc.with_source ? w->desc.src_amp : 0.0;
        q.rtol = w->desc.cg_rtol;
        q.max_it = w->desc.cg_max_it;
        q.partials = (double*)take(sizeof(double) * (size_t)b->total_blocks * 10 * b->R);
        q.bar = (unsigned*)take(64);
        q.step = (int*)(cbase + 4 * k);
        q.iter_acc = cbase + 4 * k + 1;
        q.status = (int*)(cbase + 4 * k + 2);
        q.clk = (long long*)(b->counters.as<char>() + sizeof(long long) * (16 + 4 * nprob)) + 2 * k;
        const int step = w->step;
        cudaMemcpy(q.step, &step, sizeof(int), cudaMemcpyHostToDevice);
        // dense source weights from the wave's (index, value) tables
        if (w->desc.with_source) {
            std::vector<int> idx((size_t)b->R * w->nloc);
            std::vector<double> wt(idx.size());
            cudaMemcpy(idx.data(), w->src_idx.ptr, sizeof(int) * idx.size(), cudaMemcpyDeviceToHost);
            cudaMemcpy(wt.data(), w->src_w.ptr, sizeof(double) * wt.size(), cudaMemcpyDeviceToHost);
            std::vector<float> dense(v, 0.f);
            for (int r = 0; r < b->R; ++r)
                for (int l = 0; l < w->nloc; ++l)
                    dense[(size_t)r * w->N + idx[(size_t)r * w->nloc + l]] += (float)wt[(size_t)r * w->nloc + l];
            cudaMemcpy(S, dense.data(), sizeof(float) * v, cudaMemcpyHostToDevice);
        }
        b->weights.push_back((double)w->N);   // work per step ~ rows (iteration counts are mesh-independent)
    }
    rc = upload_probs(b, 0);
    if (!rc) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e, "iga_batch_create");
    }
    if (rc) return bail(rc);
    *out = b;
    return IGA_OK;
}

extern "C" int iga_batch_destroy(iga_batch* b) {
    delete b;
    return IGA_OK;
}

extern "C" int iga_batch_step(iga_batch* b, int nsteps, int use_graph, void* stream) {
    if (!b) return fail(IGA_ERR_ARG, "null argument");
    if (nsteps < 0) return fail(IGA_ERR_ARG, "nsteps must be >= 0");
    for (auto* w : b->waves)
        if (w->nrec > 0 && w->step + nsteps > w->desc.nsteps_max) return fail(IGA_ERR_ARG, "trace buffer would overflow");
    if (nsteps == 0) return IGA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = batch_sync(b, st);
    if (rc) return rc;
    if (use_graph) {
        if (!b->graph || b->graph_nsteps != nsteps) {
            if (b->graph) cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            cudaStream_t cs;
            IGA_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g;
            IGA_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            rc = batch_launch(b, nsteps, cs);
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (rc) return rc;
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(batch)");
            e = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
            b->graph_nsteps = nsteps;
        }
        IGA_CUDA(cudaGraphLaunch(b->graph, st));
        count_launch();
    } else if ((rc = batch_launch(b, nsteps, st))) {
        return rc;
    }
    long long cnt[16 + 4 * kBMaxProbs] = {0};
    IGA_CUDA(cudaMemcpyAsync(cnt, b->counters.ptr, sizeof(long long) * (16 + 4 * b->nprob),
                             cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < b->nprob; ++k) {
        iga_wave* w = b->waves[k];
        w->step += nsteps;
        wave_views(w, b->hp[k]);   // u = U[step % 2], a = A[(step - 1) % 3], ...
    }
    const int errw = (int)cnt[0];
    if (errw & 4) return fail(IGA_ERR_TIMEOUT, "partition barrier timed out in batch");
    if (errw & 1) return fail(IGA_ERR_NONFINITE, "CG breakdown in batch");
    for (int k = 0; k < b->nprob; ++k)
        if ((int)cnt[16 + 4 * k + 2] & 8) return fail(IGA_ERR_NOT_CONVERGED, "a batched CG solve missed its tolerance");
    return IGA_OK;
}

extern "C" int iga_batch_tune(iga_batch* b, int trial_steps, int rounds, void* stream) {
    if (!b || trial_steps < 1 || rounds < 0) return fail(IGA_ERR_ARG, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    // Equalise the partitions' finishing times: each round runs trial_steps steps
    // (state advanced, trace slots rewritten later by the real run) and rescales
    // each weight by its partition's measured time relative to the mean.
    for (int it = 0; it < rounds; ++it) {
        int rc = batch_sync(b, st);
        if (!rc) rc = batch_launch(b, trial_steps, st);
        if (rc) return rc;
        std::vector<long long> clk(2 * b->nprob);
        IGA_CUDA(cudaMemcpyAsync(clk.data(), b->hp[0].clk, sizeof(long long) * 2 * b->nprob, cudaMemcpyDeviceToHost, st));
        IGA_CUDA(cudaStreamSynchronize(st));
        for (auto* w : b->waves) w->step += trial_steps;
        for (int k = 0; k < b->nprob; ++k) wave_views(b->waves[k], b->hp[k]);
        double mean = 0.0;
        std::vector<double> t(b->nprob);
        for (int k = 0; k < b->nprob; ++k) {
            t[k] = (double)std::max<long long>(1, clk[2 * k + 1] - clk[2 * k]);
            mean += t[k] / b->nprob;
        }
        for (int k = 0; k < b->nprob; ++k) b->weights[k] *= std::pow(t[k] / mean, 0.7);
        if ((rc = upload_probs(b, st))) return rc;
    }
    return IGA_OK;
}

extern "C" int iga_batch_partition(const iga_batch* b, int* blocks_out) {
    if (!b || !blocks_out) return fail(IGA_ERR_ARG, "null argument");
    for (int k = 0; k < b->nprob; ++k) blocks_out[k] = b->nb[k];
    return IGA_OK;
}
