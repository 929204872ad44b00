// Device-side geometry maps, wave-speed coefficients and pulled-back quadrature
// weights at Gauss points (shared by the assembly and wave kernels).
//
// At a Gauss point with parametric coordinate s and weight w the integrands of
// Eq. weakforms become
//   K:  grad phi_i^T  G  grad phi_j,   G = w c^2 det J  J^-1 J^-T   (symmetric)
//   M:  phi_i phi_j  wm,               wm = w det J
// with the c^2 weight of the acoustic energy (Eq. LinearWaveEnergy).
#pragma once

#include "iga_internal.cuh"

namespace iga {

// Symmetric d x d matrix packed as (00, 01, 02, 11, 12, 22) for d = 3 and (00, 01, 11) for d = 2.
__host__ __device__ constexpr int sym_index(int d, int a, int b) {
    return d == 2 ? (a + b)
                  : (a > b ? sym_index(d, b, a)
                           : (a == 0 ? b : (a == 1 ? 2 + b : 5)));
}

__device__ inline void map_eval(const GeomParams& gp, const double* s, double* x, double J[3][3]) {
    const int d = gp.dim;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) J[a][b] = (a == b) ? 1.0 : 0.0;
    if (gp.map_kind == IGA_MAP_ANNULUS_QUARTER) {
        double sn, cs;
        sincospi(0.5 * s[1], &sn, &cs);
        const double r = 1.0 + s[0];
        const double hp = 0.5 * 3.14159265358979323846;
        x[0] = r * cs;
        x[1] = r * sn;
        J[0][0] = cs;
        J[0][1] = -r * hp * sn;
        J[1][0] = sn;
        J[1][1] = r * hp * cs;
    } else if (gp.map_kind == IGA_MAP_ANNULUS_SECTOR) {
        const double dr = gp.sector[1] - gp.sector[0], da = gp.sector[3] - gp.sector[2];
        const double r = gp.sector[0] + dr * s[0];
        double sn, cs;
        sincos(gp.sector[2] + da * s[1], &sn, &cs);
        x[0] = r * cs;
        x[1] = r * sn;
        J[0][0] = dr * cs;
        J[0][1] = -r * da * sn;
        J[1][0] = dr * sn;
        J[1][1] = r * da * cs;
    } else if (gp.map_kind == IGA_MAP_BOX) {
        for (int k = 0; k < d; ++k) {
            x[k] = gp.box[k] + gp.box[3 + k] * s[k];
            J[k][k] = gp.box[3 + k];
        }
    } else if (gp.map_kind == IGA_MAP_CUBE_SINE) {
        double sn[3], cs[3];
        for (int k = 0; k < 3; ++k) sincospi(s[k], &sn[k], &cs[k]);
        const double g = sn[0] * sn[1] * sn[2];
        const double pi = 3.14159265358979323846;
        const double dg[3] = {pi * cs[0] * sn[1] * sn[2], pi * sn[0] * cs[1] * sn[2],
                              pi * sn[0] * sn[1] * cs[2]};
        for (int a = 0; a < 3; ++a) {
            x[a] = s[a] + gp.map_param * g;
            for (int b = 0; b < 3; ++b) J[a][b] += gp.map_param * dg[b];
        }
    } else {
        for (int k = 0; k < d; ++k) x[k] = s[k];
    }
}

// Wave speed squared at the point (table entry e_k, g_k per direction for the
// theta spline, physical x for the analytic coefficient).
__device__ inline double coef_c2(const GeomParams& gp, const int* e, const int* g, const double* x) {
    if (gp.coef_kind == IGA_COEF_CONST) return gp.coef_param * gp.coef_param;
    if (gp.coef_kind == IGA_COEF_SINCOS) {
        const double c = 1.0 + gp.coef_param * sinpi(2.0 * x[0]) * cospi(2.0 * x[1]);
        return c * c;
    }
    // tensor B-spline: sum over the (deg+1)^d non-zero functions
    const int k1 = gp.theta_deg + 1;
    const int nt = gp.n_theta;
    int span[3] = {0, 0, 0};
    const double* v[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < gp.dim; ++k) {
        const int idx = e[k] * gp.nq + g[k];
        span[k] = gp.tspan[idx];
        v[k] = gp.tval + (size_t)idx * k1;
    }
    double c = 0.0;
    if (gp.dim == 2) {
        for (int b = 0; b < k1; ++b) {
            double row = 0.0;
            for (int a = 0; a < k1; ++a) row += gp.theta[(span[1] + b) * nt + span[0] + a] * v[0][a];
            c += row * v[1][b];
        }
    } else {
        for (int cc = 0; cc < k1; ++cc) {
            double plane = 0.0;
            for (int b = 0; b < k1; ++b) {
                double row = 0.0;
                for (int a = 0; a < k1; ++a)
                    row += gp.theta[((size_t)(span[2] + cc) * nt + span[1] + b) * nt + span[0] + a] *
                           v[0][a];
                plane += row * v[1][b];
            }
            c += plane * v[2][cc];
        }
    }
    return c * c;
}

// Wave speed c at the point (tensor B-spline coefficient only; used by the adjoint).
__device__ inline double coef_c(const GeomParams& gp, const int* e, const int* g) {
    const int k1 = gp.theta_deg + 1;
    const int nt = gp.n_theta;
    int span[3] = {0, 0, 0};
    const double* v[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < gp.dim; ++k) {
        const int idx = e[k] * gp.nq + g[k];
        span[k] = gp.tspan[idx];
        v[k] = gp.tval + (size_t)idx * k1;
    }
    double c = 0.0;
    if (gp.dim == 2) {
        for (int b = 0; b < k1; ++b)
            for (int a = 0; a < k1; ++a) c += gp.theta[(span[1] + b) * nt + span[0] + a] * v[0][a] * v[1][b];
    } else {
        for (int cc = 0; cc < k1; ++cc)
            for (int b = 0; b < k1; ++b)
                for (int a = 0; a < k1; ++a)
                    c += gp.theta[((size_t)(span[2] + cc) * nt + span[1] + b) * nt + span[0] + a] * v[0][a] * v[1][b] *
                         v[2][cc];
    }
    return c;
}

// Pulled-back weights at Gauss point (e, g): G (packed symmetric) and wm.
// Returns det J (callers flag det J <= 0).
// Volume weight w det J at Gauss point g of element e (integrands without
// derivatives, e.g. the lumped mass).
__device__ inline double qp_volume(const GeomParams& gp, const int* e, const int* g) {
    const int d = gp.dim;
    double s[3] = {0, 0, 0}, x[3] = {0, 0, 0}, J[3][3];
    double w = 1.0;
    for (int k = 0; k < d; ++k) {
        s[k] = gp.qs[e[k] * gp.nq + g[k]];
        w *= gp.qw[g[k]];
    }
    map_eval(gp, s, x, J);
    double det;
    if (d == 2)
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    else
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    return w * det;
}

__device__ inline double qp_weights(const GeomParams& gp, const int* e, const int* g, double* G,
                                    double& wm) {
    const int d = gp.dim;
    double s[3] = {0, 0, 0}, x[3] = {0, 0, 0}, J[3][3];
    double w = 1.0;
    for (int k = 0; k < d; ++k) {
        s[k] = gp.qs[e[k] * gp.nq + g[k]];
        w *= gp.qw[g[k]];
    }
    map_eval(gp, s, x, J);
    const double c2 = coef_c2(gp, e, g, x);
    double det;
    if (d == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double id = 1.0 / det;
        // J^-1 = id [[J11, -J01], [-J10, J00]];  G = w c2 det J^-1 J^-T
        const double i00 = J[1][1] * id, i01 = -J[0][1] * id, i10 = -J[1][0] * id, i11 = J[0][0] * id;
        const double f = w * c2 * det;
        G[0] = f * (i00 * i00 + i01 * i01);
        G[1] = f * (i00 * i10 + i01 * i11);
        G[2] = f * (i10 * i10 + i11 * i11);
    } else {
        double C[3][3];  // cofactors: J^-1 = C^T / det
        C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
        const double id = 1.0 / det;
        double Ji[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Ji[a][b] = C[b][a] * id;
        const double f = w * c2 * det;
        int n = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) {
                G[n++] = f * (Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2]);
            }
    }
    wm = w * det;
    return det;
}

}  // namespace iga
