// Internal declarations of the GB300 surrogate-matrix IGA library.
// Everything here is private to libiga; the public ABI is include/iga.h.
#pragma once

#include <cuda.h>   // CUtensorMap (a type only: the driver call is reached through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/iga.h"

namespace iga {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void count_launch(long long n = 1);

#define IGA_CUDA(call)                                             \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::iga::cuda_fail(e_, #call); \
    } while (0)

#define IGA_LAUNCH_CHECK(what)                                     \
    do {                                                           \
        ::iga::count_launch();                                     \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return ::iga::cuda_fail(e_, what);  \
    } while (0)

constexpr int kMaxDim = 3;
constexpr int kMaxP = 3;
constexpr int kMaxQuad = 8;

// Device-side geometry / coefficient / basis-table bundle (passed by value).
struct GeomParams {
    int dim, p, n_el, m, nq;
    int map_kind;
    double map_param;
    double sector[4];      // ANNULUS_SECTOR: r0, r1, a0, a1
    double box[6];         // BOX: origin (3), extent (3)
    int coef_kind;
    double coef_param;
    const double* theta;   // [n_theta^dim] colex
    int n_theta, theta_deg;
    const double* qs;      // [n_el][nq] parametric coordinate of Gauss point g in element e
    const double* qw;      // [nq] Gauss weight times h
    const double* bval;    // [n_el][nq][p+1] values of local functions e+a at point g
    const double* bder;    // [n_el][nq][p+1] derivatives
    const float* bval2;    // the two tables as FP32 pairs (hi, lo) per entry
    const float* bder2;
    const int* tspan;      // [n_el][nq] first theta function non-zero at the point
    const double* tval;    // [n_el][nq][theta_deg+1] theta basis values at the point
};

// Library-owned device buffers are plain cudaMalloc allocations.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    ~DevBuf();
    int alloc(size_t nbytes);
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Brick form of the 3-D FP32 operators (brick.cu).  A brick is a box of rows
// x0 + [0, nx) x y0 + [0, ny) x z0 + [0, nz); cls selects its tensor-map box.
struct BrickDesc {
    int x0, y0, z0, nx, ny, nz, cls, warps;
};
constexpr int kBrickMaxCls = 12;
struct alignas(64) BrickMaps {
    CUtensorMap tm[kBrickMaxCls];   // one box shape per class, all over the same padded field copy
    int bx[kBrickMaxCls], by[kBrickMaxCls], bz[kBrickMaxCls];
};
struct BrickOps {
    int P = 0, m = 0, XP = 0, ncw = 0, ns = 0, nbricks = 0, ncls = 0, bzm = 0;
    long long fsz = 0;                  // elements of one padded field (XP * m * m)
    int stage_floats = 0, xt_floats = 0;
    size_t smem = 0;                    // dynamic shared memory of the brick kernels
    std::vector<BrickDesc> host;
    DevBuf bricks;                      // [nbricks] BrickDesc
    DevBuf fK, fM;                      // padded, group-ordered FP32 fields
    DevBuf err;                         // device error word of the brick kernels (bit 16: a wait timed out)
    BrickMaps mapK, mapM;
    // padded copy of the PCG's u = D^-1 r ([m][m][XP], x offset P, zero padding) and
    // its tensor maps (box = the class's vector tile: bx x by x (bz + P))
    DevBuf upad;
    BrickMaps mapU;
};

// On-the-fly evaluation of the stencil functions (onthefly.cu): per-line tables
// G[u][line][a] of the interpolation coefficients contracted over directions 1..d-1
// at the line's interior rows (filled by every on-the-fly apply).
struct OtfOps {
    int L = 0, lo = 0, ns = 0, q = 0, nf = 0;
    long long lines = 0;                 // L^(d-1)
    DevBuf gK64, gM64, gK32, gM32;       // [nf][lines][ns]
    DevBuf evals32;                      // FP32 copy of the interior evaluation table
};

}  // namespace iga

struct iga_space {
    iga_space_desc desc;
    int dim, p, n_el, m, nq;
    long long N;
    int D;
    std::vector<double> knots;              // host copy of the open uniform knot vector
    std::vector<double> gauss_x, gauss_w;   // Gauss rule on [0,1]
    std::vector<double> qs_h;               // [n_el][nq] Gauss point coordinates (host copy)
    std::vector<int> tspan_h;               // [n_el][nq] first non-zero theta function (host copy)
    std::vector<double> tval_h;             // [n_el][nq][theta_deg+1] theta basis values (host copy)
    iga::DevBuf theta, qs, qw, bval, bder, bval2, bder2, tspan, tval;
    iga::GeomParams gp;
    // element lists of the band quadrature, grouped by colour, built on the first
    // assembly that needs them ([0]: boundary band, [1]: every element)
    iga::DevBuf band_elems[2];
    std::vector<int> band_offs[2];
};

struct iga_ops {
    const iga_space* space;
    int p, q, M, dim, m, D, nK, nM, ns;
    long long N, pitch;
    unsigned flags;
    std::vector<int> samp;                   // sampled 0-based indices (one direction)
    iga::DevBuf fK64, fM64, fK32, fM32;      // fields [nK|nM][pitch]
    iga::DevBuf dinv64, dinv32;              // inverse Jacobi diagonal of M~
    iga::DevBuf sK, sM, cK, cM;              // samples / coefficients [D][ns^dim]
    iga::DevBuf status;                      // int flags: [0] nonfinite
    iga::DevBuf work;                        // CG workspace of mass_solve (grown on demand)
    std::unique_ptr<iga::BrickOps> brick;    // brick form of the FP32 fields (3-D), else null
    std::unique_ptr<iga::OtfOps> otf;        // tables of the on-the-fly apply (IGA_PATH_ONTHEFLY)
    iga::DevBuf espan, evals;                // interior rows: first coefficient and the q+1 values
                                             // of the interpolation basis at x~ (one direction)
    int path = 0;                            // IGA_PATH_*: which kernels apply the FP32 operators
    int n_band, n_samples;
    float t_sample, t_band, t_interp, t_eval, t_total;
};

struct iga_wave {
    const iga_ops* ops;
    iga_wave_desc desc;
    int dtype, nshot, nrec, nloc, step;
    long long N;
    iga::DevBuf u, uprev, a, b, traces, src_idx, src_w, rec_idx, rec_w, work, counters;
    iga::DevBuf ulo, uprevlo;        // FP32 waves: low parts of the compensated state (hi + lo)
    iga::DevBuf ah[IGA_CG_GUESS_MAX];   // cg_guess = K > 0: ah[j] = a^{n-2-j}, j < K (a holds a^{n-1})
    iga::DevBuf greville, centres;   // pulse initial condition inputs (GAUSS_PULSE)
    int timing = 0;
    long long cg_solves = 0;
    double cg_ms = 0.0, force_ms = 0.0;
    double lam_min = 0.0, lam_max = 0.0;
};

namespace iga {
// kernels implemented in apply.cu / solve.cu, shared launch helpers
int launch_apply(const iga_ops* ops, int which, int dtype, const void* x, void* y, int nrhs,
                 cudaStream_t st);
// b, x: [nrhs][ld] (ld >= N) in the dtype's precision
int mass_solve_impl(const iga_ops* ops, int dtype, const void* b, void* x, long long ld, int nrhs, double rtol,
                    int max_it, unsigned flags, int* iters_out, double* relres_out, cudaStream_t st,
                    void* work, size_t work_bytes, long long* iter_acc, int* status_acc);
size_t mass_solve_work_bytes(const iga_ops* ops, int dtype, int nrhs);
// brick.cu: builds ops->brick (3-D, FP32 fields present); no-op otherwise
int brick_prepare(iga_ops* ops, cudaStream_t st);
bool brick_usable(const iga_ops* ops, int which);
int brick_apply(const iga_ops* ops, int which, const float* x, float* y, cudaStream_t st);
// onthefly.cu: y = A x with the interior stencil functions evaluated from the coefficients
int onthefly_apply(const iga_ops* ops, int which, int dtype, const void* x, void* y, int nrhs, cudaStream_t st);
int onthefly_prepare(iga_ops* ops);
int spectrum_impl(const iga_ops* ops, int dtype, int k, double* lam_min, double* lam_max, cudaStream_t st);
int wave_step_impl(iga_wave* w, int nsteps, cudaStream_t st);
int wave_initial_state(iga_wave* w, cudaStream_t st);
// colex decode of stencil offset t into delta (0..dim-1), values in [-p, p]
inline void decode_offset(int t, int dim, int p, int delta[3]) {
    int P = 2 * p + 1;
    for (int k = 0; k < 3; ++k) {
        delta[k] = (k < dim) ? (t % P) - p : 0;
        t /= P;
    }
}
// The (p+1)^d basis functions of a space that are non-zero at parametric point pt
// (clamped to [0,1]^d): colex indices and values B_i(pt).  Host only.
void point_basis(const iga_space* s, const double* pt, int* idx, double* w);
// Ricker wavelet r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2).  Host only.
double ricker(double t, double f0, double t0);

}  // namespace iga
