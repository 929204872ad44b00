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
//
// The field loop is unrolled UNR-fold with run-time offsets, so a thread keeps
// only UNR fields in flight: few registers, many resident warps, and 4 UNR
// independent loads per thread in flight to cover HBM latency.
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
__host__ __device__ __forceinline__ int field_delta(int u, int m) {
    constexpr int PP = 2 * P + 1;
    const int t = StencilShape<DIM, P>::T0 + 1 + u;
    const int d1 = t % PP - P;
    const int d2 = (t / PP) % PP - P;
    const int d3 = DIM == 3 ? t / (PP * PP) - P : 0;
    return d1 + (d2 + d3 * m) * m;
}

// Vector loaders: read-only vectors go through the non-coherent path; vectors
// written by other blocks of a persistent launch use ordinary coherent loads.
template <typename T>
struct LdgLoad {
    const T* x;
    long long xs;
    __device__ __forceinline__ T operator()(int r, int idx) const { return __ldg(x + r * xs + idx); }
};

// One output row of the operator for R right-hand sides given by a loader.
// own[r] receives the row's own vector value (ld(r, i)).
template <int DIM, int P, typename T, bool MASS, int R, int UNR, class Load>
__device__ __forceinline__ void stencil_row(const T* __restrict__ F, long long pitch, const Load& ld, int i, int N,
                                            int m, T* acc, T* own) {
    constexpr int NF = StencilShape<DIM, P>::T0;
#pragma unroll
    for (int r = 0; r < R; ++r) own[r] = ld(r, i);
    if (MASS) {
        const T d = __ldg(F + i);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = d * own[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = T(0);
    }
    const T* Foff = MASS ? F + pitch : F;
#pragma unroll UNR
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
            const T xpv = ld(r, ipc);
            const T xmv = ld(r, imc);
            const T xp = okp ? xpv : T(0);
            const T xm = okm ? xmv : T(0);
            if (MASS) {
                acc[r] = fma(s, xp, acc[r]);
                acc[r] = fma(sm, xm, acc[r]);
            } else {
                acc[r] = fma(s, xp - own[r], acc[r]);
                acc[r] = fma(sm, xm - own[r], acc[r]);
            }
        }
    }
}

}  // namespace iga
