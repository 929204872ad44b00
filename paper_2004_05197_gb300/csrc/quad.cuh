// Quadrature helpers shared by the assembly kernels and their reverse-mode
// (adjoint) counterparts: stencil sizes, colex digit decoding, local basis
// values / gradients from the per-element 1-D tables, symmetric 2x2 / 3x3
// products.
#pragma once

#include "geom.cuh"

namespace iga {

template <int DIM, int P>
struct Stencil {
    static constexpr int P1 = P + 1;
    static constexpr int NLOC = DIM == 2 ? P1 * P1 : P1 * P1 * P1;
    static constexpr int PP = 2 * P + 1;
    static constexpr int DD = DIM == 2 ? PP * PP : PP * PP * PP;
    static constexpr int T0 = (DD - 1) / 2;
    static constexpr int NS = DIM == 2 ? 3 : 6;   // packed symmetric entries of G
};

// colex decode of a local index into DIM digits of base `base`
template <int DIM>
__device__ __forceinline__ void decode(int idx, int base, int* out) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        out[k] = idx % base;
        idx /= base;
    }
}

template <int DIM>
__device__ __forceinline__ bool in_range(const int* i, int lo, int hi) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k) ok = ok && (i[k] >= lo) && (i[k] <= hi);
    return ok;
}

// grad phi_a(q) and phi_a(q) from the 1-D tables of element e at point g
template <int DIM, int P>
__device__ __forceinline__ void local_basis(const GeomParams& gp, const int* e, const int* g,
                                            const int* a, double* grad, double& val) {
    double v[DIM], dv[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const int idx = (e[k] * gp.nq + g[k]) * (P + 1) + a[k];
        v[k] = gp.bval[idx];
        dv[k] = gp.bder[idx];
    }
    val = 1.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) val *= v[k];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double gk = 1.0;
#pragma unroll
        for (int j = 0; j < DIM; ++j) gk *= (j == k) ? dv[j] : v[j];
        grad[k] = gk;
    }
}

template <int DIM>
__device__ __forceinline__ void sym_matvec(const double* G, const double* x, double* y) {
    if (DIM == 2) {
        y[0] = G[0] * x[0] + G[1] * x[1];
        y[1] = G[1] * x[0] + G[2] * x[1];
    } else {
        y[0] = G[0] * x[0] + G[1] * x[1] + G[2] * x[2];
        y[1] = G[1] * x[0] + G[3] * x[1] + G[4] * x[2];
        y[2] = G[2] * x[0] + G[4] * x[1] + G[5] * x[2];
    }
}

}  // namespace iga
