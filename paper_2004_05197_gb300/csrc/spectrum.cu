// Extreme eigenvalues of the surrogate pencil K~ v = lambda M~ v.
//
// Lanczos process for A = M~^-1 K~, which is self-adjoint in the M~ inner
// product (Golub & Van Loan, "Matrix Computations", Sec. 10.1, generalised
// form): with v_0 M~-normalised,
//   alpha_j = v_j^T K~ v_j,   w = M~^-1 K~ v_j - alpha_j v_j - beta_{j-1} v_{j-1},
//   beta_j = sqrt(w^T M~ w),  v_{j+1} = w / beta_j.
// The eigenvalues of the tridiagonal T_k = tridiag(beta, alpha, beta) bracket
// the spectrum from inside; the extreme ones converge first.  They are found by
// Sturm-sequence bisection (count of negative pivots of T - x I).
//
// lambda_max bounds the leapfrog step (stable iff dt sqrt(lambda_max) < 2);
// lambda_min < 0 means the surrogate K~ is indefinite (sampling too coarse for
// the coefficient), in which case the wave equation has growing modes.
#include <algorithm>
#include <cmath>
#include <vector>

#include "iga_internal.cuh"

namespace iga {

template <typename T>
__global__ void start_vector_kernel(T* v, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        // integer hash of the index (splitmix64 finaliser) -> uniform value in [-1, 1)
        unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

template <typename T>
__global__ void dot_kernel(const T* a, const T* b, long long n, double* partials) {
    __shared__ double s[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}

// y = a x + b y + c z
template <typename T>
__global__ void axpbypcz_kernel(T* y, const T* x, const T* z, double a, double b, double c, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)(a * (double)x[i] + b * (double)y[i] + (z ? c * (double)z[i] : 0.0));
}

constexpr int kDotBlocks = 512;

template <typename T>
static int dot(const T* a, const T* b, long long n, double* d_part, double* out, cudaStream_t st) {
    dot_kernel<T><<<kDotBlocks, 256, 0, st>>>(a, b, n, d_part);
    IGA_LAUNCH_CHECK("dot_kernel");
    double h[kDotBlocks];
    IGA_CUDA(cudaMemcpyAsync(h, d_part, sizeof(h), cudaMemcpyDeviceToHost, st));
    IGA_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int k = 0; k < kDotBlocks; ++k) s += h[k];
    *out = s;
    return IGA_OK;
}

// Number of eigenvalues of the symmetric tridiagonal (alpha, beta) below x.
static int sturm_count(const std::vector<double>& alpha, const std::vector<double>& beta, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < alpha.size(); ++i) {
        const double b2 = i ? beta[i - 1] * beta[i - 1] : 0.0;
        q = (alpha[i] - x) - (i ? b2 / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

static double tridiag_eig(const std::vector<double>& alpha, const std::vector<double>& beta, int which /*0 min, 1 max*/) {
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < alpha.size(); ++i) {   // Gershgorin interval
        const double r = (i ? std::fabs(beta[i - 1]) : 0.0) + (i + 1 < alpha.size() ? std::fabs(beta[i]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    const int target = which ? (int)alpha.size() - 1 : 0;   // index of the wanted eigenvalue
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(alpha, beta, mid) > target) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

template <typename T>
static int spectrum_typed(const iga_ops* ops, int dtype, int k, double* lam_min, double* lam_max, cudaStream_t st) {
    const long long N = ops->N;
    const int grid = (int)std::min<long long>((N + 255) / 256, 152 * 8);
    DevBuf buf;
    int rc = buf.alloc(sizeof(T) * 4 * (size_t)N + sizeof(double) * kDotBlocks);
    if (rc) return rc;
    T* vprev = buf.as<T>();
    T* v = vprev + N;
    T* w = v + N;
    T* y = w + N;
    double* part = (double*)(y + N);
    iga_ops* mops = const_cast<iga_ops*>(ops);
    const size_t need = mass_solve_work_bytes(ops, dtype, 1);
    if (mops->work.bytes < need && (rc = mops->work.alloc(need))) return rc;
    const double rtol = dtype == IGA_F64 ? 1e-9 : 1e-5;
    start_vector_kernel<T><<<grid, 256, 0, st>>>(v, N);
    IGA_LAUNCH_CHECK("start_vector_kernel");
    IGA_CUDA(cudaMemsetAsync(vprev, 0, sizeof(T) * N, st));
    if ((rc = launch_apply(ops, IGA_OP_M, dtype, v, y, 1, st))) return rc;
    double nrm2 = 0.0;
    if ((rc = dot<T>(v, y, N, part, &nrm2, st))) return rc;
    axpbypcz_kernel<T><<<grid, 256, 0, st>>>(v, v, nullptr, 1.0 / std::sqrt(nrm2), 0.0, 0.0, N);
    IGA_LAUNCH_CHECK("axpbypcz_kernel");
    std::vector<double> alpha, beta;
    double beta_prev = 0.0;
    for (int j = 0; j < k; ++j) {
        if ((rc = launch_apply(ops, IGA_OP_K, dtype, v, y, 1, st))) return rc;
        double a = 0.0;
        if ((rc = dot<T>(v, y, N, part, &a, st))) return rc;
        IGA_CUDA(cudaMemsetAsync(w, 0, sizeof(T) * N, st));
        rc = mass_solve_impl(ops, dtype, y, w, N, 1, rtol, 2000, 0, nullptr, nullptr, st, mops->work.ptr,
                             mops->work.bytes, nullptr, nullptr);
        if (rc && rc != IGA_ERR_NOT_CONVERGED) return rc;
        axpbypcz_kernel<T><<<grid, 256, 0, st>>>(w, v, vprev, -a, 1.0, -beta_prev, N);
        IGA_LAUNCH_CHECK("axpbypcz_kernel");
        if ((rc = launch_apply(ops, IGA_OP_M, dtype, w, y, 1, st))) return rc;
        double b2 = 0.0;
        if ((rc = dot<T>(w, y, N, part, &b2, st))) return rc;
        alpha.push_back(a);
        const double b = std::sqrt(std::max(b2, 0.0));
        if (!(b > 1e-12 * std::fabs(a)) || j == k - 1) break;
        beta.push_back(b);
        std::swap(vprev, v);                               // v_prev <- v
        axpbypcz_kernel<T><<<grid, 256, 0, st>>>(v, w, nullptr, 1.0 / b, 0.0, 0.0, N);   // v <- w / b
        IGA_LAUNCH_CHECK("axpbypcz_kernel");
        beta_prev = b;
    }
    beta.resize(alpha.empty() ? 0 : alpha.size() - 1);
    if (alpha.empty()) return fail(IGA_ERR_NONFINITE, "Lanczos produced no coefficients");
    for (double x : alpha)
        if (!std::isfinite(x)) return fail(IGA_ERR_NONFINITE, "non-finite Lanczos coefficient");
    if (lam_min) *lam_min = tridiag_eig(alpha, beta, 0);
    if (lam_max) *lam_max = tridiag_eig(alpha, beta, 1);
    return IGA_OK;
}

int spectrum_impl(const iga_ops* ops, int dtype, int k, double* lam_min, double* lam_max, cudaStream_t st) {
    return dtype == IGA_F64 ? spectrum_typed<double>(ops, dtype, k, lam_min, lam_max, st)
                            : spectrum_typed<float>(ops, dtype, k, lam_min, lam_max, st);
}

}  // namespace iga

extern "C" int iga_ops_spectrum(const iga_ops* ops, int dtype, int k, double* lam_min, double* lam_max,
                                void* stream) {
    if (!ops) return iga::fail(IGA_ERR_ARG, "null argument");
    if (dtype != IGA_F32 && dtype != IGA_F64) return iga::fail(IGA_ERR_ARG, "bad dtype");
    if (k < 2 || k > 1000) return iga::fail(IGA_ERR_ARG, "k must be in 2..1000");
    return iga::spectrum_impl(ops, dtype, k, lam_min, lam_max, (cudaStream_t)stream);
}
