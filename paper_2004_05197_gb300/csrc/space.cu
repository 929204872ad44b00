// Space creation: knot vector, Gauss rule, per-element basis tables, theta
// tables; error bookkeeping and small ABI helpers.
//
// Host numerics (own implementations of published methods):
//  * open uniform knot vector of Sec. 3.1;
//  * Gauss-Legendre nodes by Newton's method on the Legendre polynomial,
//    evaluated with its three-term recurrence; weights 2 / ((1-x^2) P_n'(x)^2);
//  * B-spline values and first derivatives of the p+1 functions non-zero on a
//    knot span by the triangular Cox-de Boor scheme (de Boor, "A Practical
//    Guide to Splines", Ch. X).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <atomic>

#include "host_bspline.h"
#include "iga_internal.cuh"

namespace iga {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return IGA_ERR_CUDA;
}
void count_launch(long long n) { g_launches += n; }

DevBuf::~DevBuf() { release(); }
int DevBuf::alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    cudaError_t e = cudaMalloc(&ptr, nbytes);
    if (e != cudaSuccess) {
        ptr = nullptr;
        (void)cudaGetLastError();
        return fail(IGA_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    bytes = nbytes;
    return IGA_OK;
}
void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

template <class T>
static int upload(DevBuf& buf, const std::vector<T>& v) {
    int rc = buf.alloc(v.size() * sizeof(T));
    if (rc) return rc;
    IGA_CUDA(cudaMemcpy(buf.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return IGA_OK;
}

}  // namespace iga

using namespace iga;

extern "C" const char* iga_last_error(void) { return g_last_error.c_str(); }
extern "C" long long iga_launch_count(void) { return g_launches.load(); }

extern "C" int iga_space_create(const iga_space_desc* desc, iga_space** out) {
    if (!desc || !out) return fail(IGA_ERR_ARG, "null argument");
    *out = nullptr;
    const iga_space_desc& d = *desc;
    if (d.dim != 2 && d.dim != 3) return fail(IGA_ERR_ARG, "dim must be 2 or 3");
    if (d.p < 1 || d.p > kMaxP) return fail(IGA_ERR_ARG, "p must be in 1..3");
    if (d.n_el < 4 * d.p + 2) return fail(IGA_ERR_ARG, "n_el must be >= 4p+2");
    const int nq = d.quad_pts > 0 ? d.quad_pts : d.p + 1;
    if (nq > kMaxQuad) return fail(IGA_ERR_ARG, "quad_pts must be <= 8");
    if (d.map_kind == IGA_MAP_ANNULUS_QUARTER && d.dim != 2)
        return fail(IGA_ERR_ARG, "ANNULUS_QUARTER map is 2-D");
    if (d.map_kind == IGA_MAP_CUBE_SINE && d.dim != 3) return fail(IGA_ERR_ARG, "CUBE_SINE map is 3-D");
    if (d.map_kind < 0 || d.map_kind > 4) return fail(IGA_ERR_ARG, "unknown map_kind");
    if (d.map_kind == IGA_MAP_BOX) {
        double det = 1.0;
        for (int k = 0; k < d.dim; ++k) det *= d.box[3 + k];
        if (!(det > 0.0)) return fail(IGA_ERR_ARG, "BOX map needs a positive extent product (det J > 0)");
    }
    if (d.map_kind == IGA_MAP_ANNULUS_SECTOR) {
        if (d.dim != 2) return fail(IGA_ERR_ARG, "ANNULUS_SECTOR map is 2-D");
        const double dr = d.sector[1] - d.sector[0], da = d.sector[3] - d.sector[2];
        if (!(d.sector[0] > 0.0) || !(d.sector[1] > 0.0) || !(dr * da > 0.0))
            return fail(IGA_ERR_ARG, "ANNULUS_SECTOR needs radii > 0 and (r1 - r0)(a1 - a0) > 0");
    }
    if (d.coef_kind < 0 || d.coef_kind > 2) return fail(IGA_ERR_ARG, "unknown coef_kind");
    if (d.coef_kind == IGA_COEF_SINCOS && d.dim != 2) return fail(IGA_ERR_ARG, "SINCOS coefficient is 2-D");
    if (d.coef_kind == IGA_COEF_BSPLINE) {
        if (!d.theta) return fail(IGA_ERR_ARG, "theta is null");
        if (d.theta_degree < 1 || d.theta_degree > 5) return fail(IGA_ERR_ARG, "theta_degree must be 1..5");
        if (d.n_theta <= d.theta_degree) return fail(IGA_ERR_ARG, "n_theta must exceed theta_degree");
    }
    long long N = 1;
    for (int k = 0; k < d.dim; ++k) N *= (d.n_el + d.p);
    if (N > (1LL << 31) - 1) return fail(IGA_ERR_ARG, "too many basis functions for 32-bit indexing");

    iga_space* s = new (std::nothrow) iga_space();
    if (!s) return fail(IGA_ERR_OOM, "host allocation failed");
    s->desc = d;
    s->desc.theta = nullptr;
    s->dim = d.dim;
    s->p = d.p;
    s->n_el = d.n_el;
    s->m = d.n_el + d.p;
    s->nq = nq;
    s->N = N;
    s->D = 1;
    for (int k = 0; k < d.dim; ++k) s->D *= 2 * d.p + 1;
    s->knots = hb::open_uniform_knots(d.n_el, d.p);
    hb::gauss_legendre01(nq, s->gauss_x, s->gauss_w);

    // per-element tables: every 1-D element e, Gauss point g, local function a = 0..p
    const double h = 1.0 / d.n_el;
    std::vector<double> qs(d.n_el * nq), qw(nq), bval(d.n_el * nq * (d.p + 1)), bder(bval.size());
    for (int g = 0; g < nq; ++g) qw[g] = s->gauss_w[g] * h;
    std::vector<double> N0(d.p + 1), N1(d.p + 1);
    for (int e = 0; e < d.n_el; ++e) {
        for (int g = 0; g < nq; ++g) {
            const double x = (e + s->gauss_x[g]) * h;
            qs[e * nq + g] = x;
            const int span = e + d.p;   // knots[span] <= x < knots[span+1]
            hb::basis_and_derivative(s->knots, d.p, span, x, N0.data(), N1.data());
            for (int a = 0; a <= d.p; ++a) {
                bval[(e * nq + g) * (d.p + 1) + a] = N0[a];
                bder[(e * nq + g) * (d.p + 1) + a] = N1[a];
            }
        }
    }
    int rc = upload(s->qs, qs);
    if (!rc) rc = upload(s->qw, qw);
    if (!rc) rc = upload(s->bval, bval);
    if (!rc) rc = upload(s->bder, bder);
    {   // FP32 pairs hi + lo of the tables (the band quadrature's double-float path)
        std::vector<float> bv2(2 * bval.size()), bd2(2 * bder.size());
        for (size_t i = 0; i < bval.size(); ++i) {
            bv2[2 * i] = (float)bval[i];
            bv2[2 * i + 1] = (float)(bval[i] - (double)bv2[2 * i]);
            bd2[2 * i] = (float)bder[i];
            bd2[2 * i + 1] = (float)(bder[i] - (double)bd2[2 * i]);
        }
        if (!rc) rc = upload(s->bval2, bv2);
        if (!rc) rc = upload(s->bder2, bd2);
    }
    std::vector<int> tspan(d.n_el * nq, 0);
    std::vector<double> tval;
    if (!rc && d.coef_kind == IGA_COEF_BSPLINE) {
        const int k = d.theta_degree;
        std::vector<double> tk = hb::open_uniform_knots(d.n_theta - k, k);
        tval.assign((size_t)d.n_el * nq * (k + 1), 0.0);
        std::vector<double> T0(k + 1), T1(k + 1);
        for (int i = 0; i < d.n_el * nq; ++i) {
            const double x = qs[i];
            const int span = hb::find_span(tk, k, x);
            hb::basis_and_derivative(tk, k, span, x, T0.data(), T1.data());
            tspan[i] = span - k;
            for (int a = 0; a <= k; ++a) tval[(size_t)i * (k + 1) + a] = T0[a];
        }
        size_t nth = 1;
        for (int kk = 0; kk < d.dim; ++kk) nth *= (size_t)d.n_theta;
        std::vector<double> th(desc->theta, desc->theta + nth);
        rc = upload(s->theta, th);
        if (!rc) rc = upload(s->tval, tval);
    } else if (!rc) {
        rc = upload(s->tval, std::vector<double>(1, 0.0));
        if (!rc) rc = upload(s->theta, std::vector<double>(1, 0.0));
    }
    if (!rc) rc = upload(s->tspan, tspan);
    s->qs_h = qs;
    s->tspan_h = tspan;
    s->tval_h = tval;
    if (rc) {
        delete s;
        return rc;
    }
    GeomParams& gp = s->gp;
    gp.dim = d.dim;
    gp.p = d.p;
    gp.n_el = d.n_el;
    gp.m = s->m;
    gp.nq = nq;
    gp.map_kind = d.map_kind;
    gp.map_param = d.map_param;
    for (int k = 0; k < 4; ++k) gp.sector[k] = d.sector[k];
    for (int k = 0; k < 6; ++k) gp.box[k] = d.box[k];
    gp.coef_kind = d.coef_kind;
    gp.coef_param = d.coef_param;
    gp.theta = s->theta.as<double>();
    gp.n_theta = d.n_theta;
    gp.theta_deg = d.theta_degree;
    gp.qs = s->qs.as<double>();
    gp.qw = s->qw.as<double>();
    gp.bval = s->bval.as<double>();
    gp.bder = s->bder.as<double>();
    gp.bval2 = s->bval2.as<float>();
    gp.bder2 = s->bder2.as<float>();
    gp.tspan = s->tspan.as<int>();
    gp.tval = s->tval.as<double>();
    *out = s;
    return IGA_OK;
}

extern "C" int iga_space_destroy(iga_space* space) {
    delete space;
    return IGA_OK;
}

extern "C" int iga_space_info_get(const iga_space* s, iga_space_info* out) {
    if (!s || !out) return fail(IGA_ERR_ARG, "null argument");
    out->dim = s->dim;
    out->p = s->p;
    out->n_el = s->n_el;
    out->m = s->m;
    out->N = s->N;
    out->D = s->D;
    out->nK = (s->D - 1) / 2;
    out->nM = (s->D + 1) / 2;
    out->interior_lo = 2 * s->p;
    out->interior_hi = s->m - 2 * s->p - 1;
    return IGA_OK;
}
