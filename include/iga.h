/*
 * iga.h - C ABI of the GB300 (sm_103a) surrogate-matrix IGA wave library.
 *
 * The library implements the data-parallel hot path of the surrogate matrix
 * methodology for isogeometric analysis of waves (Drzisga, Keith, Wohlmuth,
 * arXiv:2004.05197):
 *   (a) Gauss quadrature of the true stiffness / mass rows at a sparse lattice
 *       of sample rows and on the boundary band (Sec. 3.2-3.4, Sec. 5.1),
 *   (b) degree-q B-spline interpolation of every stencil function and
 *       evaluation of the surrogate stencils of every row (Sec. 3.3, Sec. 5.1,
 *       Eq. DefinitionOfSurrogateMatrixSymmetric, ..SymmetricKernel),
 *   (c) matrix-free application of the surrogate operators, Jacobi-PCG on the
 *       consistent surrogate mass and leapfrog time stepping (Sec. 3.3: stored
 *       stencil-function data read during every matrix-vector product).
 *
 * Conventions (every entry point):
 *   - returns int: IGA_OK (0) or a negative IGA_ERR_* code; iga_last_error()
 *     returns a thread-local message for the last failure.  No C++ exception
 *     crosses the ABI.
 *   - handles (iga_space, iga_ops, iga_wave) are opaque and owned by the
 *     library; free them with the matching *_destroy.  A handle must outlive
 *     all stream work that uses it.
 *   - "device pointer" arguments are borrowed CUDA device memory of the
 *     current device; the library never frees them and the caller keeps them
 *     alive until the stream work completes.  "host pointer" arguments are
 *     read (or written) before the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream), owned by the caller.  Calls are asynchronous on that stream
 *     unless they return host data (documented per call).
 *   - Vectors over the basis are stored [nrhs][N] contiguous, global index in
 *     colexicographic order i = i_1 + i_2 m + i_3 m^2 (0-based; Sec. 3.1).
 *   - Stencil offsets delta in {-p..p}^d are enumerated colexicographically,
 *     t = sum_k (delta_k + p) (2p+1)^k; t0 = ((2p+1)^d - 1)/2 is delta = 0 and
 *     t > t0 exactly when the linear offset Delta = delta_1 + delta_2 m + ... > 0.
 *   - Stencil fields (structure-of-arrays, row pitch `pitch` >= N):
 *       K~ field f (0 <= f < nK = t0):    F_K[f][i] = K~(i, i + Delta_{t0+1+f})
 *       M~ field f (0 <= f < nM = t0+1): F_M[f][i] = M~(i, i + Delta_{t0+f})
 *     (upper triangle of the symmetric matrices; 0 where the column leaves
 *     the index grid).  The K~ diagonal is not stored: by
 *     Eq. DefinitionOfSurrogateMatrixSymmetricKernel it is minus the
 *     off-diagonal row sum, and the K~ apply uses the difference form
 *     (K~x)_i = sum_{j != i} K~_ij (x_j - x_i).
 */
#ifndef IGA_H
#define IGA_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define IGA_OK                  0
#define IGA_ERR_ARG            -1   /* invalid argument or unsupported configuration */
#define IGA_ERR_OOM            -2   /* device or host allocation failed */
#define IGA_ERR_CUDA           -3   /* a CUDA runtime call failed */
#define IGA_ERR_NOT_CONVERGED  -4   /* CG reached max_it before rtol for some RHS */
#define IGA_ERR_NONFINITE      -5   /* a NaN / Inf was detected on the device */
#define IGA_ERR_TIMEOUT        -6   /* a bounded device-side wait gave up */

/* ---- enumerations ---------------------------------------------------- */
#define IGA_MAP_IDENTITY         0  /* F(s) = s */
#define IGA_MAP_ANNULUS_QUARTER  1  /* F(s,t) = ((1+s) cos(pi t/2), (1+s) sin(pi t/2)) */
#define IGA_MAP_CUBE_SINE        2  /* x_k = s_k + a sin(pi s) sin(pi t) sin(pi u), a = map_param */
#define IGA_MAP_ANNULUS_SECTOR   3  /* F(s,t) = (r cos a, r sin a), r = r0 + (r1-r0) s,
                                       a = a0 + (a1-a0) t, (r0, r1, a0, a1) = sector[]: one patch of
                                       a multi-patch annulus; det J = (r1-r0)(a1-a0) r must be > 0 */
#define IGA_MAP_BOX              4  /* x_k = o_k + e_k s_k, (o_1..o_3, e_1..e_3) = box[]: an
                                       axis-aligned box, one patch of a multi-patch brick; a
                                       negative e_k runs s_k against x_k; det J = prod e_k > 0 */

#define IGA_COEF_CONST    0  /* c = coef_param */
#define IGA_COEF_SINCOS   1  /* c(x) = 1 + coef_param sin(2 pi x_1) cos(2 pi x_2), x = F(s) physical */
#define IGA_COEF_BSPLINE  2  /* c(s) = sum_k theta_k B_k(s), open uniform knots on [0,1]^d */

#define IGA_F32 0   /* FP32 stencil fields and vectors, FP64 reductions */
#define IGA_F64 1   /* FP64 everywhere */

#define IGA_OP_K 0  /* surrogate stiffness K~ */
#define IGA_OP_M 1  /* surrogate mass M~ */

/* surrogate_assemble flags */
#define IGA_TRUE_ONLY     1u  /* full quadrature of every entry: the true K, M (no surrogate) */
#define IGA_KEEP_SAMPLES  2u  /* keep sample tables and interpolation coefficients for export */
#define IGA_MASS_VOLUME_PRESERVING 4u
/* volume-preserving surrogate mass (Sec. 3.4, remark on volume preservation):
   M~ = D + M~_0, D_ii = int_Omega B_i (Gauss quadrature of phi_i det J), M~_0
   built like K~ from the mass stencil functions.  The off-diagonal entries are
   those of the plain M~; the stored diagonal becomes D_ii - sum_{j!=i} M~_ij,
   so sum_ij M~_ij = |Omega| (up to quadrature of det J).  Every consumer of the
   M~ fields (apply, mass_solve, waves, adjoint) uses it unchanged. */

/* mass_solve flags */
#define IGA_SOLVE_PLAIN   1u  /* non-persistent schedule: one launch per CG phase, host-side
                                 convergence test every iteration (reference schedule) */
#define IGA_SOLVE_GRAPH   2u  /* graph schedule: the phases as full-occupancy launches in one CUDA
                                 graph whose conditional WHILE node iterates until the device decides
                                 convergence (no grid barrier, no host round trip); falls back to
                                 the persistent schedule when the stream is being captured */
#define IGA_SOLVE_REFINE  4u  /* FP64 solves only: iterative refinement, the FP64 residual
                                 b - M~x with the FP64 fields, the correction from the FP32
                                 Jacobi-PCG on the FP32 fields, x += d in FP64, until the FP64
                                 residual meets rtol (same stopping rule as the FP64 solve).
                                 Synchronises the stream once per refinement; iters_out
                                 counts the FP32 CG iterations.  Combines with
                                 IGA_SOLVE_PLAIN / IGA_SOLVE_GRAPH for the inner solves */

/* wave initial conditions */
#define IGA_INIT_ZERO         0
#define IGA_INIT_GAUSS_PULSE  1  /* u0_i = exp(-|F(gamma_i) - F(s_c)|^2 / (2 w^2)), Greville gamma */

typedef struct iga_space iga_space;
typedef struct iga_ops iga_ops;
typedef struct iga_wave iga_wave;

/* ---- space ------------------------------------------------------------
 * Tensor-product B-spline space of degree p on open uniform knots with n_el
 * elements in every direction (Sec. 3.1: m = n_el + p functions per direction,
 * h = 1/(m-p)), the geometry map and the wave-speed coefficient c (stiffness
 * weight c^2, Eq. LinearWaveEnergy).
 */
typedef struct iga_space_desc {
    int dim;               /* 2 or 3 */
    int p;                 /* spline degree, 1..3 */
    int n_el;              /* elements per direction, >= 4p+2 */
    int map_kind;          /* IGA_MAP_* (ANNULUS_QUARTER needs dim 2, CUBE_SINE dim 3) */
    double map_param;      /* CUBE_SINE amplitude */
    int coef_kind;         /* IGA_COEF_* */
    double coef_param;     /* CONST: c; SINCOS: amplitude */
    const double* theta;   /* host pointer, BSPLINE: n_theta^dim coefficients, colex; copied */
    int n_theta;           /* BSPLINE: coefficients per direction (> theta_degree) */
    int theta_degree;      /* BSPLINE: degree of the coefficient spline, 1..5 */
    int quad_pts;          /* Gauss points per direction and element; 0 => p+1 (Sec. 5.1); <= 8 */
    double sector[4];      /* ANNULUS_SECTOR: r0, r1, a0, a1 (radians) */
    double box[6];         /* BOX: o_1, o_2, o_3, e_1, e_2, e_3 (2-D uses the first two of each) */
} iga_space_desc;

typedef struct iga_space_info {
    int dim, p, n_el, m;
    long long N;           /* m^dim */
    int D;                 /* (2p+1)^dim stencil offsets (Sec. 3.2) */
    int nK, nM;            /* stored K~ / M~ fields: (D-1)/2 and (D+1)/2 */
    int interior_lo, interior_hi;  /* 0-based Omega~ index range per direction: [2p, m-2p-1] */
} iga_space_info;

/* Validates desc, uploads the quadrature / basis tables and, for
 * IGA_COEF_BSPLINE, a copy of theta.  Errors: IGA_ERR_ARG for unsupported
 * dim / p / n_el / map / quad_pts or a non-positive det J found at a
 * quadrature point. Synchronous. */
int iga_space_create(const iga_space_desc* desc, iga_space** out);
int iga_space_destroy(iga_space* space);
int iga_space_info_get(const iga_space* space, iga_space_info* out);

/* ---- surrogate assembly -----------------------------------------------
 * surrogate_assemble(p, q, M): sample rows by the rule of Sec. 5.1 (every
 * (L-1)/ceil((L-1)/M)-th of the L = m-4p interior points per direction,
 * rounded half away from zero), true rows at the samples by Gauss
 * quadrature, degree-q interpolation with de Boor-averaged knots taken from
 * the samples (Sec. 3.3), true entries of every pair (i,j) with i or j
 * outside Omega~ by element quadrature of the boundary band, and the fields
 * of Eq. DefinitionOfSurrogateMatrixSymmetric / ..SymmetricKernel.
 * p must equal the space's degree; q >= 1; at least q+1 samples per
 * direction; M >= 1 (M = 1 gives the true matrices up to rounding).
 * Builds FP64 fields and FP32 copies, and the inverse Jacobi diagonal of M~.
 * Asynchronous on `stream` except for a final status check (synchronises).
 */
/* Mesh-dependent sampling length (Sec. 5.2, Eq. MeshDependentSamplingLength):
 * M(h) = max{1, floor(C h^(eps - 1 + (p+a)/(q+b)))}, evaluated in FP64 on the
 * host, saturating at INT_MAX.  With q + b > p + a and eps small the sampling
 * distance H = M h shrinks more slowly than h, so H^(q+b) = o(h^(p+a)).
 * Needs h > 0, q + b > 0, C > 0, eps > 0, p >= 1 (else IGA_ERR_ARG).
 * Synchronous, no device work. */
int iga_sampling_length_for_mesh(double h, int p, int q, double a, double b, double C, double eps,
                                 int* M_out);

int iga_surrogate_assemble(iga_space* space, int p, int q, int M, unsigned flags,
                           void* stream, iga_ops** out);
int iga_ops_destroy(iga_ops* ops);

typedef struct iga_ops_info {
    long long N;
    long long pitch;        /* row pitch of the fields (elements) */
    int m, dim, p, q, M;
    int nK, nM, D;
    int ns;                 /* samples per direction */
    int n_band_elements;    /* elements quadrated for the true entries */
    int n_sample_rows;      /* ns^dim */
    double t_sample_ms, t_band_ms, t_interp_ms, t_eval_ms, t_total_ms; /* device time */
    long long workspace_bytes; /* CG workspace the library holds for iga_mass_solve on this
                                  ops (0 until the first such call) */
} iga_ops_info;
int iga_ops_info_get(const iga_ops* ops, iga_ops_info* out);

/* Copies the fields of `which` (IGA_OP_K / IGA_OP_M) in `dtype` into dst
 * (device pointer, nK or nM rows of N elements, packed [f][N]). Async. */
int iga_ops_copy_fields(const iga_ops* ops, int which, int dtype, void* dst, void* stream);
/* Copies the sample table of `which` into dst (device pointer, double,
 * [D][ns^dim], sample index colex): the true row entries at the sample rows.
 * Needs IGA_KEEP_SAMPLES. Async. */
int iga_ops_copy_samples(const iga_ops* ops, int which, double* dst, void* stream);
/* Copies the 0-based sampled indices of one direction to a host array of
 * ns ints. Synchronous (host data only). */
int iga_ops_sample_indices(const iga_ops* ops, int* host_dst);

/* ---- matrix-free operators -----------------------------------------------
 * stencil_apply: y = A x for A = K~ or M~, the surrogate matrices of
 * Eq. DefinitionOfSurrogateMatrixSymmetric (mass) and
 * Eq. DefinitionOfSurrogateMatrixSymmetricKernel (stiffness: off-diagonal
 * entries from the stencil functions, diagonal = minus the off-diagonal row
 * sum), applied matrix-free from the stored stencil data as Sec. 3.3 describes
 * for matrix-free methods.  Row i reads its upper entries F_u[i] and, by
 * symmetry, its lower entries F_u[i - Delta_u]; K~ is applied in the
 * difference form (K~x)_i = sum_{j != i} K~_ij (x_j - x_i), exact on constants.
 * nrhs vectors; x, y device pointers [nrhs][N] of `dtype` (float or double);
 * y must not alias x (IGA_ERR_ARG).  Each field element is read once per call
 * for all nrhs vectors (row kernels) or once per vector (brick kernels of 3-D
 * FP32 operators, see iga_ops_set_path).  Asynchronous on `stream`.
 */
int iga_stencil_apply(const iga_ops* ops, int which, int dtype, const void* x, void* y,
                      int nrhs, void* stream);

/* Which kernels run the FP32 operators of a 3-D ops (stencil_apply and the
 * persistent mass solve; FP64 and 2-D operators always use the row kernels).
 *   IGA_PATH_AUTO  (default) the brick kernels where a brick form exists and its
 *                  bricks are large enough to be faster (about 3,000 rows per
 *                  brick for M~, 5,000 for K~), else the row kernels
 *   IGA_PATH_ROWS  one thread per row, fields read from the colex SoA layout
 *   IGA_PATH_BRICK the brick kernels (IGA_ERR_ARG if the ops has no brick form)
 * Brick form (built by surrogate_assemble for dim 3, p <= 2): the rows are cut
 * into about one brick per SM; each CTA streams its brick's fields through a
 * TMA ring of shared-memory stages from a second, padded and group-ordered copy
 * of the FP32 fields (about 1.06x the colex FP32 fields), so every field and
 * vector value a row needs is read from shared memory (Sec. 3.3: matrix-free use
 * of the stored stencil data).  Results equal the row kernels' up to the FP32
 * summation order.  Host-only, synchronous. */
#define IGA_PATH_AUTO  0
#define IGA_PATH_ROWS  1
#define IGA_PATH_BRICK 2
/* IGA_PATH_ONTHEFLY (iga_stencil_apply only, FP32 and FP64, every supported dim
 * and p; solves run as under IGA_PATH_AUTO): the stencil functions are evaluated
 * inside each apply from the B-spline interpolation coefficients of Sec. 3.3
 * instead of being read from the stored fields, for every row whose whole
 * stencil is surrogate (every interior index of the row in [3p, m-3p-1]); the
 * other rows and the M~ diagonal are read from the stored fields.  Each apply
 * first contracts the coefficients over directions 1..d-1 at every interior line
 * (a table of (D-1)/2 (m-4p)^(d-1) ns values), then evaluates each entry with q+1
 * FMAs.  Setting it allocates those tables (synchronous; IGA_ERR_ARG for an
 * IGA_TRUE_ONLY ops or a mesh with no such row).  Results equal the stored-field
 * apply up to rounding. */
#define IGA_PATH_ONTHEFLY 3
int iga_ops_set_path(iga_ops* ops, int path);
/* Brick plan of an ops (all outputs nullable host pointers; zeros without a
 * brick form): bricks (= CTAs of a brick launch), threads per CTA, ring
 * stages, dynamic shared memory bytes per CTA, and brick_paths: which FP32
 * operators run on brick kernels under the current path setting (bit 0: K~
 * apply; bit 1: M~ apply and the persistent single-RHS mass solve).  Host-only. */
int iga_ops_brick_info(const iga_ops* ops, int* nbricks, int* threads, int* stages, int* smem_bytes,
                       int* brick_paths);

/* mass_solve: Jacobi-PCG on M~ a = b for nrhs right-hand sides.  The paper
 * gives no solver for the consistent mass: the preconditioned CG here (Jacobi
 * preconditioner, Chronopoulos-Gear arrangement of the recurrence, same iterates
 * as textbook PCG) is the library's choice.  Arguments: device
 * pointers [nrhs][N] of `dtype`; x holds the initial guess on entry and the
 * solution on exit.  Stops each RHS when ||r||_2 <= rtol ||b||_2 (rtol = 0:
 * exactly max_it iterations).  FP32 dtype: FP32 fields / vectors, FP64
 * residual and dot products.  Default schedule: one persistent cooperative
 * launch for all iterations with device-side convergence; IGA_SOLVE_PLAIN:
 * one launch per phase and a host convergence test per iteration.
 * FP32 3-D operators with a brick form (see iga_ops_set_path) run the brick
 * form of the persistent launch for single right-hand sides.
 * iters_out / relres_out: host arrays of nrhs (nullable).  The call always
 * synchronises the stream and reads the solver status back, also when both are
 * NULL.  Returns IGA_ERR_NOT_CONVERGED if some RHS missed rtol (x still holds
 * the last iterate), IGA_ERR_NONFINITE on a CG breakdown, IGA_ERR_TIMEOUT if a
 * bounded device-side wait (grid barrier, field ring) gave up. */
int iga_mass_solve(const iga_ops* ops, int dtype, const void* b, void* x, int nrhs,
                   double rtol, int max_it, unsigned flags, int* iters_out,
                   double* relres_out, void* stream);

/* mass_solve_noalloc: the paper has no counterpart to this entry point; it is
 * an operational variant of iga_mass_solve.  Same arguments, solver, results
 * and return codes, but no device memory is allocated: the CG workspace is a
 * fixed array of IGA_NOALLOC_SCRATCH_BYTES compiled into the library instead
 * of a buffer the library cudaMallocs on first use.  It is for callers that
 * cannot have the library allocate: cudaMalloc / cudaFree may synchronise the
 * whole device and stall the caller's other streams inside a latency-bound
 * loop, and a caller whose device memory is managed by another allocator (a
 * framework's caching allocator, a fixed memory budget) needs the library's
 * footprint known up front.
 * Limit: the workspace for (N, dtype, nrhs) must fit in the array.  It is
 * about 40 N bytes for FP64 with nrhs < 4 and 160 N with nrhs >= 4 (FP32:
 * 24 N and 96 N), plus ~100 KB; e.g. FP64 single-RHS solves up to about
 * 1.6 M rows.  Larger requests return IGA_ERR_ARG before any work.
 * Set-up: every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress); the first call on a device may load the
 * module that holds the array, so make that first call before any stream
 * capture.  With lazy module loading (the CUDA default) only devices on which
 * this entry point runs hold the array; with CUDA_MODULE_LOADING=EAGER every
 * device that loads the library does.  The call synchronises the stream (the
 * solver status is always read back into host memory).
 * IGA_SOLVE_GRAPH is rejected (IGA_ERR_ARG): that schedule instantiates a CUDA
 * graph per call, which may reserve device resources; so is IGA_SOLVE_REFINE,
 * whose extra vectors the fixed array is not sized for.
 * Sharing: all calls on a device use the same array, so calls that overlap in
 * time (different streams or host threads) race and corrupt one another;
 * the caller must serialise them (e.g. one stream). */
#define IGA_NOALLOC_SCRATCH_BYTES (64u << 20)
int iga_mass_solve_noalloc(const iga_ops* ops, int dtype, const void* b, void* x, int nrhs,
                           double rtol, int max_it, unsigned flags, int* iters_out,
                           double* relres_out, void* stream);

/* Self-test of the bounded grid barrier that the persistent CG kernels use (a
 * failure-detection check that faults nothing): one cooperative launch of
 * `blocks` blocks (1 <= blocks <= the SM count) whose barrier waits for
 * `expected` arrivals, each waiting block giving up after limit_ms
 * milliseconds of SM clock.  Returns IGA_OK when the barrier opened
 * (expected <= blocks), IGA_ERR_TIMEOUT when the wait ran out (expected >
 * blocks: the arrival that nothing makes); the device context stays usable
 * either way.  Synchronises the stream. */
int iga_barrier_selftest(int blocks, int expected, double limit_ms, void* stream);

/* ---- spectrum --------------------------------------------------------------
 * Extreme eigenvalues of the pencil K~ v = lambda M~ v by k Lanczos steps in the
 * M~ inner product (each step: one K~ apply, one mass solve, one M~ apply).
 * The leapfrog step is stable iff dt sqrt(lambda_max) < 2 (no CFL is given in
 * the paper); lambda_min < 0 reports an indefinite surrogate K~ (sampling
 * length too large for the coefficient).  Synchronous (host scalars). */
int iga_ops_spectrum(const iga_ops* ops, int dtype, int k, double* lambda_min, double* lambda_max,
                     void* stream);

/* ---- wave time stepping ------------------------------------------------
 * Leapfrog for M~ u'' + K~ u = f (unit density, natural boundary
 * conditions): a^n solves M~ a^n = f^n - K~ u^n by Jacobi-PCG started from
 * a^{n-1}; u^{n+1} = 2u^n - u^{n-1} + dt^2 a^n, first step u^1 = u^0 + dt^2/2 a^0
 * (v^0 = 0).  Point source f_i^n = amp r(t_n) B_i(s_src), Ricker
 * r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t_n = n dt.
 * Receivers record d^n = sum_i u_i^n B_i(s_rec) after every step.
 */
#define IGA_CG_GUESS_MAX 6   /* highest extrapolation order of the CG start (cg_guess) */

typedef struct iga_wave_desc {
    int nshot;                  /* independent shots advanced together (multi-RHS) */
    int dtype;                  /* IGA_F32 or IGA_F64 */
    unsigned solve_flags;       /* IGA_SOLVE_PLAIN for the plain schedule */
    double dt;
    int init_kind;              /* IGA_INIT_* */
    const double* pulse_centre; /* host [nshot][dim] parametric centres (GAUSS_PULSE) */
    double pulse_width;
    int with_source;            /* 1: Ricker point source per shot */
    const double* src_pos;      /* host [nshot][dim] parametric source positions */
    double f0, t0, src_amp;
    int nrec;                   /* receivers, shared by all shots */
    const double* rec_pos;      /* host [nrec][dim] parametric receiver positions */
    int nsteps_max;             /* capacity of the trace buffer (steps) */
    double cg_rtol;
    int cg_max_it;
    int cfl_check;              /* 1: estimate lambda_max(M~^-1 K~) by Lanczos at create and at every
                                   reset; 2: at create only; 0: off.  With an estimate, steps
                                   with dt sqrt(lambda_max) >= 2 are refused (IGA_ERR_ARG) */
    int cg_guess;               /* start of step n's mass solve: the polynomial extrapolation in
                                   time of order K = cg_guess (0..IGA_CG_GUESS_MAX) through the last
                                   K + 1 accelerations, sum_{j=0..K} (-1)^j C(K+1, j+1) a^{n-1-j}:
                                   0 = a^{n-1}; 1 = 2a^{n-1} - a^{n-2}; 2 = 3a^{n-1} - 3a^{n-2} +
                                   a^{n-3}; ...  The order drops to what the steps done so far
                                   allow (a^{-1} = 0 at n = 0, order min(K, n - 1) after).  Only
                                   the starting point of the CG changes; every solve still runs
                                   to cg_rtol.  K extra acceleration vectors per shot are kept.
                                   wave_adjoint uses the same order in its forward and
                                   recomputed sweeps (checkpoints keep the K accelerations)
                                   and in reverse time for its adjoint solves */
} iga_wave_desc;

int iga_wave_create(const iga_ops* ops, const iga_wave_desc* desc, iga_wave** out);
int iga_wave_destroy(iga_wave* wave);
/* Advances every shot by nsteps of the leapfrog scheme M~ a^n = f^n - K~ u^n,
 * u^{n+1} = 2 u^n - u^{n-1} + dt^2 a^n (the paper solves no transient problem
 * with the surrogate matrices; Sec. 4.6 gives the setting, the scheme is this
 * library's).  Async on stream; returns (after synchronising)
 * IGA_ERR_NOT_CONVERGED if a CG solve missed its tolerance, IGA_ERR_NONFINITE
 * on a CG breakdown, IGA_ERR_TIMEOUT if a bounded device wait of a solve gave
 * up, IGA_ERR_ARG if the trace buffer would overflow. */
int iga_wave_step(iga_wave* wave, int nsteps, void* stream);
/* Copies u^n (and u^{n-1} if u_prev != NULL) into device buffers [nshot][N] of the
 * wave's dtype. Async. */
int iga_wave_get_state(const iga_wave* wave, void* u, void* u_prev, void* stream);
/* Copies the traces recorded so far to a host array [nshot][nrec][nsteps_done]
 * (double) and returns the step count in *nsteps_done. Synchronous. */
int iga_wave_traces(const iga_wave* wave, double* host_dst, int* nsteps_done);
/* Total CG iterations summed over steps and shots since creation. */
int iga_wave_cg_iterations(const iga_wave* wave, long long* total);

/* Rebinds the wave to `ops` (same space size and dtype support) and restarts
 * it: initial condition recomputed, step counter, traces, CG counters and
 * timing statistics cleared, a^{-1} = 0.  No allocation. Async on stream. */
int iga_wave_reset(iga_wave* wave, const iga_ops* ops, void* stream);

/* Per-wave statistics. With timing on, every force (K~ apply) launch and every
 * CG solve of wave_step is bracketed by CUDA events on the launching stream
 * and the elapsed device times are accumulated when wave_step synchronises. */
typedef struct iga_wave_stats {
    long long steps;          /* steps advanced since creation / reset */
    long long cg_iterations;  /* CG iterations summed over steps and shots */
    long long cg_solves;      /* CG solves issued (one per step per chunk of <= 4 shots) */
    double cg_ms;             /* device time of the CG solves (timing on) */
    double force_ms;          /* device time of the force launches (timing on) */
    double lambda_min;        /* Lanczos estimates of the pencil (K~, M~) (cfl_check on, else 0) */
    double lambda_max;
} iga_wave_stats;
int iga_wave_set_timing(iga_wave* wave, int on);
int iga_wave_stats_get(const iga_wave* wave, iga_wave_stats* out);

/* ---- batched persistent stepping -------------------------------------------
 * A batch advances several FP32 waves (one mesh each, all with the same nshot
 * in {1, 4, 8, 16} and the same dim / p; meshes of uneven size allowed) by
 * nsteps leapfrog steps in ONE cooperative persistent launch: the grid is split
 * into one block partition per wave, each partition runs its own force, CG
 * (Chronopoulos-Gear Jacobi-PCG, per-shot convergence, bounded partition
 * barriers) and update for every step.  The waves keep owning their state,
 * traces and counters (wave_get_state / wave_traces work as usual).
 * use_graph = 1 captures the launch in a CUDA graph on first use and replays it
 * (the step counters live in device memory).  The batch borrows the waves: they
 * must outlive it.  Synchronous (reads back the status word). */
typedef struct iga_batch iga_batch;
int iga_batch_create(int nprob, iga_wave* const* waves, iga_batch** out);
int iga_batch_destroy(iga_batch* batch);
int iga_batch_step(iga_batch* batch, int nsteps, int use_graph, void* stream);
/* Tuner of the block partition: `rounds` trial launches of trial_steps steps
 * each (the waves advance; reset them afterwards), rescaling each partition's
 * share by its measured time so that all partitions finish together. */
int iga_batch_tune(iga_batch* batch, int trial_steps, int rounds, void* stream);
/* Blocks per partition (host array of nprob ints). */
int iga_batch_partition(const iga_batch* batch, int* blocks_out);

/* ---- adjoint ------------------------------------------------------------
 * wave_adjoint: restarts the wave (FP64 only) from its initial condition, runs
 * nsteps leapfrog steps with checkpoints (u^n, u^{n-1}, a^{n-1} and the cg_guess
 * older accelerations) every checkpoint_every steps, evaluates the receiver misfit
 *     J = dt/2 sum_shots sum_receivers sum_{n=1..nsteps} (d^n - obs^n)^2
 * and, if grad_theta != NULL, its gradient with respect to the B-spline
 * coefficients theta of the wave speed (space created with IGA_COEF_BSPLINE) by
 * the discrete adjoint of leapfrog + CG + surrogate assembly (segments are
 * recomputed from their checkpoints).  The paper has no adjoint; this is the
 * differentiation of its surrogate model.
 *   obs        host [nshot][nrec][nsteps] observed traces
 *   J_out      host scalar (nullable)
 *   grad_theta host [n_theta^dim], colex (nullable: misfit only)
 * Synchronous.  Errors: IGA_ERR_ARG (FP32 wave, no receivers, nsteps outside
 * 1..nsteps_max, coefficient not a B-spline), CG errors as in wave_step. */
int iga_wave_adjoint(iga_wave* wave, int nsteps, int checkpoint_every, const double* obs, double* J_out,
                     double* grad_theta, void* stream);

/* ---- multi-patch ---------------------------------------------------------
 * Sec. 3.2 and Sec. 3.4 (remarks on multi-patch geometries): a domain split into
 * 2-D or 3-D patches, each with its own map, coefficient and surrogate fields
 * (one iga_ops per patch, assembled on its own space), glued along whole sides
 * (2-D) or faces (3-D) into the C0-conforming multi-patch space.  The global matrix is the sum over
 * patches of P_l^T A_l P_l.  Global numbering: the local functions are visited
 * patch by patch, each patch in colex order, and every class of functions
 * identified by the interfaces takes the next global index at its first member.
 */
typedef struct iga_multipatch iga_multipatch;
typedef struct iga_interface {
    int patch_a, side_a;   /* side 2k = {i_(k+1) = 0}, side 2k+1 = {i_(k+1) = m-1}: 0..3 in 2-D,
                              0..5 in 3-D; its entries run colex over the remaining indices */
    int patch_b, side_b;   /* the two sides must have the same number m of functions */
    int reversed;          /* orientation.  2-D: 0 = entry k meets entry k, 1 = entry m-1-k.
                              3-D (entry (u, v) of side a, u the faster index): bit 2 swaps u
                              and v, then bit 0 reverses u (u -> m-1-u) and bit 1 reverses v;
                              the result is the entry of side b that meets it */
} iga_interface;

/* patches: npatch borrowed iga_ops (same dimension and p; they must outlive the
 * handle).  Builds the numbering and the inverse Jacobi diagonal of the global M~.
 * Errors: IGA_ERR_ARG (bad interface or orientation, unequal sides, mixed dimensions),
 * IGA_ERR_NONFINITE (non-positive global mass diagonal).  Synchronous. */
int iga_multipatch_create(int npatch, const iga_ops* const* patches, int ninterface,
                          const iga_interface* interfaces, iga_multipatch** out);
int iga_multipatch_destroy(iga_multipatch* mp);
/* Number of global functions.  Host only. */
int iga_multipatch_size(const iga_multipatch* mp, long long* n_global);
/* Global index of every local function of `patch` (colex), into host_map[N_patch]. */
int iga_multipatch_global_index(const iga_multipatch* mp, int patch, long long* host_map);
/* y = A x for the global K~ or M~; x, y device [nrhs][n_global] of dtype (y must not
 * alias x).  Gathers the patch vectors, applies every patch operator, sums the
 * patch results of every global function in a fixed order.  Async on stream. */
int iga_multipatch_apply(const iga_multipatch* mp, int which, int dtype, const void* x, void* y,
                         int nrhs, void* stream);
/* Jacobi-PCG on the global M~ a = b, b / x device [nrhs][n_global] (x: initial guess
 * in, solution out), stop when ||r||_2 <= rtol ||b||_2; FP32 dtype: FP32 vectors,
 * FP64 residual and dot products.  The CG scalars stay on the device; the host
 * reads them back every 16 iterations to test convergence (a right-hand side that
 * converges inside such a batch stops changing at once).  Synchronous.  Returns
 * IGA_ERR_NOT_CONVERGED / IGA_ERR_NONFINITE as mass_solve. */
int iga_multipatch_mass_solve(const iga_multipatch* mp, int dtype, const void* b, void* x, int nrhs,
                              double rtol, int max_it, int* iters_out, double* relres_out,
                              void* stream);

/* Leapfrog on the multi-patch surrogate operators: the scheme of iga_wave_step
 * (Sec. 4.6 time stepping with surrogate matrices; the scheme itself is this
 * library's, the paper has none) on the glued space:
 *   u^{n+1} = 2 u^n - u^{n-1} + dt^2 a^n,  M~ a^n = f^n - K~ u^n,
 *   u^1 = u^0 + dt^2/2 a^0 (zero initial velocity),
 * a^n by the multi-patch Jacobi-PCG (rtol cg_rtol, at most cg_max_it iterations per
 * step) started from a^{n-1} (0 at n = 0), f^n = amp r(n dt) B(s_src) with the Ricker
 * wavelet r(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2) and B(s_src)
 * the global basis at parametric point src_s of patch src_patch (src_patch < 0: no
 * source), and receiver traces d_r^n = sum_i u_i^n B_i(rec_s[r]) in patch
 * rec_patch[r] for n = 1..nsteps.  FP32 carries the state as an unevaluated pair
 * of FP32 numbers (the applies read the high part).
 *   u       device [n_global] of dtype: u^0 in, u^nsteps out
 *   src_s   host [dim] parametric point; rec_patch host [nrec]; rec_s host [nrec][dim]
 *   traces  host [nrec][nsteps] FP64 (nullable when nrec = 0)
 *   cg_iters_out host, nullable: CG iterations summed over the steps
 * Host-driven like iga_multipatch_mass_solve; synchronous.  Errors: IGA_ERR_ARG,
 * and the CG errors of iga_multipatch_mass_solve. */
int iga_multipatch_leapfrog(const iga_multipatch* mp, int dtype, double dt, int nsteps, void* u,
                            int src_patch, const double* src_s, double f0, double t0, double amp,
                            int nrec, const int* rec_patch, const double* rec_s, double* traces,
                            double cg_rtol, int cg_max_it, long long* cg_iters_out, void* stream);

/* ---- misc ------------------------------------------------------------- */
const char* iga_last_error(void);
/* Number of library kernel launches issued since load (for launch accounting). */
long long iga_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* IGA_H */
