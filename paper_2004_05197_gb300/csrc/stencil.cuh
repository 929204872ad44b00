// Matrix-free application of the symmetric surrogate stencil operators.
//
// Storage (upper triangle, structure of arrays): off-diagonal field u holds
// A(i, i + Delta_u) for offset t = t0 + 1 + u (Delta_u > 0).  Row i of A needs
// its own upper entries F_u[i] and, by symmetry, its lower entries
// A(i, i - Delta_u) = F_u[i - Delta_u]; every field element is therefore read
// by two rows, once as "upper" and once as "mirrored", and each apply streams
// every field once from HBM (the second read of an element comes from L2: the
// two rows are at most Delta_max = p (1 + m + m^2) apart).
//
//   K~ (difference form, kernel preserving, Eq. ..SymmetricKernel):
//       (K~x)_i = sum_u F_u[i] (x_{i+Delta_u} - x_i) + F_u[i-Delta_u] (x_{i-Delta_u} - x_i)
//   M~: (M~x)_i = F_diag[i] x_i + sum_u F_u[i] x_{i+Delta_u} + F_u[i-Delta_u] x_{i-Delta_u}
//
// Entries whose column leaves the index grid are stored as 0, so a wrapped
// linear neighbour contributes nothing; only the linear range [0, N) is guarded,
// by clamping the neighbour index (every address stays inside its buffer).
#pragma once

#include "iga_internal.cuh"

namespace iga {

template <int DIM, int P>
struct StencilShape {
    static constexpr int PP = 2 * P + 1;
    static constexpr int DD = DIM == 2 ? PP * PP : PP * PP * PP;
    static constexpr int T0 = (DD - 1) / 2;   // number of off-diagonal fields
};

// Linear offset of off-diagonal field u (t = t0 + 1 + u) for row length m.
template <int DIM, int P>
__host__ __device__ constexpr int field_delta(int u, int m) {
    return ((StencilShape<DIM, P>::T0 + 1 + u) % (2 * P + 1) - P) +
           (((StencilShape<DIM, P>::T0 + 1 + u) / (2 * P + 1)) % (2 * P + 1) - P) * m +
           (DIM == 3 ? (((StencilShape<DIM, P>::T0 + 1 + u) / ((2 * P + 1) * (2 * P + 1))) % (2 * P + 1) - P) *
                           m * m
                     : 0);
}

// One output row of the operator for R right-hand sides whose vectors start at
// x[r * xs] (r < R).  Returns the row values in acc.
template <int DIM, int P, typename T, bool MASS, int R>
__device__ __forceinline__ void stencil_row(const T* __restrict__ F, long long pitch, const T* __restrict__ x,
                                            long long xs, int i, int N, int m, T* acc) {
    constexpr int NF = StencilShape<DIM, P>::T0;
    const T* Foff = MASS ? F + pitch : F;   // mass: field 0 is the diagonal
    T xi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) xi[r] = __ldg(x + r * xs + i);
    if (MASS) {
        const T d = __ldg(F + i);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = d * xi[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = T(0);
    }
#pragma unroll
    for (int u = 0; u < NF; ++u) {
        const int dl = field_delta<DIM, P>(u, m);
        const T* Fu = Foff + (size_t)u * pitch;
        // neighbour indices are clamped to the row itself when they leave [0, N),
        // so every address formed is inside its buffer; the value is then masked
        const int ip = i + dl, im = i - dl;
        const bool okp = ip < N, okm = im >= 0;
        const int ipc = okp ? ip : i, imc = okm ? im : i;
        const T s = __ldg(Fu + i);
        const T smv = __ldg(Fu + imc);
        const T sm = okm ? smv : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T xpv = __ldg(x + r * xs + ipc);
            const T xmv = __ldg(x + r * xs + imc);
            const T xp = okp ? xpv : T(0);
            const T xm = okm ? xmv : T(0);
            if (MASS) {
                acc[r] = fma(s, xp, acc[r]);
                acc[r] = fma(sm, xm, acc[r]);
            } else {
                acc[r] = fma(s, xp - xi[r], acc[r]);
                acc[r] = fma(sm, xm - xi[r], acc[r]);
            }
        }
    }
}

}  // namespace iga
