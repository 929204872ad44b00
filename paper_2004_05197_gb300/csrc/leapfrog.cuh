// Leapfrog update of an FP32 state kept as an unevaluated sum hi + lo of two
// FP32 numbers.  The step u^{n+1} = 2u^n - u^{n-1} + dt^2 a^n adds an increment
// several orders of magnitude smaller than u, so a plain FP32 update drops the
// increment's low bits every step and the loss accumulates over the run; here
// the rounding error of each step is captured exactly (Knuth's TwoSum, written
// with round-to-nearest intrinsics so that no FMA contraction alters it) and
// carried in lo.  The stencil apply reads hi only; receivers read hi + lo.
#pragma once

namespace iga {

__device__ __forceinline__ float two_sum(float a, float b, float& err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// (hn, ln) = 2 (hc + lc) - (hp + lp) + inc, or (hc + lc) + inc on the first step.
__device__ __forceinline__ void leapfrog_comp(float hc, float lc, float hp, float lp, float inc, bool first,
                                              float& hn, float& ln) {
    float s, t;
    if (first) {
        s = hc;
        t = __fadd_rn(lc, inc);
    } else {
        float e;
        s = two_sum(__fmul_rn(2.f, hc), -hp, e);                          // 2 hc is exact
        t = __fadd_rn(__fadd_rn(__fsub_rn(__fmul_rn(2.f, lc), lp), inc), e);
    }
    hn = two_sum(s, t, ln);
}

}  // namespace iga
