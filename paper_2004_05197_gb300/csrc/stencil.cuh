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

// Field loads: read-only, streamed once per apply (the mirrored second read of an
// element is served by L2).  NA = true: the loads do not allocate in L1, leaving it
// to the gathered vector values that neighbouring rows reuse (measured on the
// stand-alone 62-field FP32 apply: 68 -> 63 us with 16 fields in flight; inside the
// persistent CG kernels, whose vector loads are coherent, it measured no better, so
// they keep the default read-only path).
template <bool NA, typename T>
__device__ __forceinline__ T ld_field(const T* p) {
    if constexpr (!NA) {
        return __ldg(p);
    } else if constexpr (sizeof(T) == 4) {
        float v;
        asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    } else {
        double v;
        asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    }
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
template <int DIM, int P, typename T, bool MASS, int R, int UNR, class Load, bool NA = false>
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
        const T s = ld_field<NA>(Fu + i);
        const T smv = ld_field<NA>(Fu + imc);
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

// One row computed by a whole warp: the fields are split across the lanes
// (u = lane, lane + 32, ..) with the same clamped neighbour handling as
// stencil_row, then summed with a fixed butterfly, so every lane returns the row.
// Used for the few rows left after the last full round of a grid-stride loop,
// where one thread per row would leave the rest of the grid waiting on a single
// row's chain of field loads.  All 32 lanes must call it together.
template <int DIM, int P, typename T, bool MASS, int R, class Load>
__device__ __forceinline__ void stencil_row_warp(const T* __restrict__ F, long long pitch, const Load& ld, int i, int N,
                                                 int m, int lane, T* acc, T* own) {
    constexpr int NF = StencilShape<DIM, P>::T0;
#pragma unroll
    for (int r = 0; r < R; ++r) own[r] = ld(r, i);
    if (MASS) {
        const T d = lane == 0 ? __ldg(F + i) : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = d * own[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = T(0);
    }
    const T* Foff = MASS ? F + pitch : F;
    for (int u = lane; u < NF; u += 32) {
        const int dl = field_delta<DIM, P>(u, m);
        const T* Fu = Foff + (size_t)u * pitch;
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
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
}

// Interior rows (Delta_max <= i < N - Delta_max): every neighbour is inside
// [0, N), so no clamping or masking is needed.  Offsets come from the shared
// table sdl[u] = Delta_u (one broadcast load per field); per field and RHS the
// row costs 4 loads, 2 subtractions (difference form) and 2 FMAs.
template <int DIM, int P, typename T, bool MASS, int R, int UNR, class Load, bool NA = false>
__device__ __forceinline__ void stencil_row_interior(const T* __restrict__ F, long long pitch, const Load& ld, int i,
                                                     const int* sdl, T* acc, T* own) {
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
    const T* Fi = (MASS ? F + pitch : F) + i;
#pragma unroll UNR
    for (int u = 0; u < NF; ++u) {
        const int dl = sdl[u];
        const T* Fu = Fi + (size_t)u * pitch;
        const T s = ld_field<NA>(Fu);
        const T sm = ld_field<NA>(Fu - dl);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T xp = ld(r, i + dl);
            const T xm = ld(r, i - dl);
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

// ---------------------------------------------------------------------------
// FP32 path, four consecutive rows per thread (i0 = 4k).
//
// The own field values of rows i0..i0+3 are one aligned float4.  The mirrored
// values F_u[i0-Delta .. i0-Delta+3] and the neighbour vector values start at
// an offset that is the same for every thread of the warp (Delta mod 4), so
// they are read as two aligned float4 and the four wanted lanes selected
// without divergence.  Offsets come from a shared table sdl[u] = Delta_u.
// Only "interior" groups use this path: every index read, including the
// second aligned float4, lies in [0, N):  i0 >= Delta_max and
// i0 + 7 + Delta_max <= N - 1.  Other groups take the scalar path per row.
namespace iga {

__device__ __forceinline__ float4 f4_fma(float4 a, float4 b, float4 c) {
    return make_float4(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y), fmaf(a.z, b.z, c.z), fmaf(a.w, b.w, c.w));
}
__device__ __forceinline__ float4 f4_sub(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 f4_mul(float4 a, float4 b) {
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
// lanes off..off+3 of the 8 consecutive values (v0, v1)
__device__ __forceinline__ float4 f4_window(float4 v0, float4 v1, int off) {
    switch (off) {
        case 0: return v0;
        case 1: return make_float4(v0.y, v0.z, v0.w, v1.x);
        case 2: return make_float4(v0.z, v0.w, v1.x, v1.y);
        default: return make_float4(v0.w, v1.x, v1.y, v1.z);
    }
}
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
// four values base[j..j+3] for an arbitrary j >= 0 (warp-uniform j mod 4)
__device__ __forceinline__ float4 ldg4u(const float* base, int j) {
    const int off = j & 3;
    const float* a = base + (j - off);
    const float4 v0 = ldg4(a);
    if (off == 0) return v0;
    return f4_window(v0, ldg4(a + 4), off);
}

// Read-only vectors [R][ld] (ld a multiple of 4, base 16-byte aligned).
struct LdgLoad4 {
    const float* x;
    long long ld;
    __device__ __forceinline__ float load1(int r, int idx) const { return __ldg(x + r * ld + idx); }
    __device__ __forceinline__ float4 load4(int r, int idx) const { return ldg4(x + r * ld + idx); }
    __device__ __forceinline__ float4 load4u(int r, int j) const { return ldg4u(x + r * ld, j); }
};

template <int DIM, int P, bool MASS, int R, int UNR, class L>
__device__ __forceinline__ void stencil_row4(const float* __restrict__ F, long long pitch, const L& ld, int i0,
                                             const int* sdl, float4* acc, float4* own) {
    constexpr int NF = StencilShape<DIM, P>::T0;
#pragma unroll
    for (int r = 0; r < R; ++r) own[r] = ld.load4(r, i0);
    if (MASS) {
        const float4 d = ldg4(F + i0);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = f4_mul(d, own[r]);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float* Foff = MASS ? F + pitch : F;
#pragma unroll UNR
    for (int u = 0; u < NF; ++u) {
        const int dl = sdl[u];
        const float* Fu = Foff + (size_t)u * pitch;
        const float4 s = ldg4(Fu + i0);
        const float4 sm = ldg4u(Fu, i0 - dl);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 xp = ld.load4u(r, i0 + dl);
            const float4 xm = ld.load4u(r, i0 - dl);
            if (MASS) {
                acc[r] = f4_fma(s, xp, acc[r]);
                acc[r] = f4_fma(sm, xm, acc[r]);
            } else {
                acc[r] = f4_fma(s, f4_sub(xp, own[r]), acc[r]);
                acc[r] = f4_fma(sm, f4_sub(xm, own[r]), acc[r]);
            }
        }
    }
}

// Delta table of the off-diagonal fields in shared memory (call with all threads).
template <int DIM, int P>
__device__ __forceinline__ void fill_delta_table(int* sdl, int m) {
    for (int u = threadIdx.x; u < StencilShape<DIM, P>::T0; u += blockDim.x) sdl[u] = field_delta<DIM, P>(u, m);
    __syncthreads();
}

template <int DIM, int P>
__host__ __device__ __forceinline__ int max_delta(int m) {
    return field_delta<DIM, P>(StencilShape<DIM, P>::T0 - 1, m);
}

}  // namespace iga
