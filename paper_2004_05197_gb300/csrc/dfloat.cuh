// Double-float arithmetic: a value carried as the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits), after Dekker (1971) and Knuth's
// error-free transformations: TwoSum for sums, an FMA for the exact product of
// the high parts.  On GB300 the FP64 pipe issues about 1.9 operations per clock
// and SM against 128 FP32 FMAs, so a contraction done in these pairs costs far
// less issue time than the same contraction in FP64 while keeping close to FP64
// accuracy (each operation is exact up to about 2^-47 relative).  The round-to-
// nearest intrinsics keep the compiler from contracting the error terms.
#pragma once

namespace iga {

struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 df_from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_value(f2 a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (s, e) with |e| small against s: the pair renormalised
__device__ __forceinline__ f2 df_renorm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);   // a.hi b.hi = p + e exactly
    e = __fadd_rn(e, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
    return df_renorm(p, e);
}

// acc += a b
__device__ __forceinline__ void df_mac(f2& acc, f2 a, f2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = __fadd_rn(e, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
    float s, t;
    df_two_sum(acc.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(acc.lo, e));
    acc = df_renorm(s, t);
}

}  // namespace iga
