// Vectors of the FP32-form solves as pairs of floats (hi, lo), hi + lo the
// FP64 value to about 2^-48: products with an FP32 entry by TwoProduct (fmaf)
// plus the small entry-times-lo term, sums compensated (TwoSum; the scheme of
// Ogita, Rump and Oishi's Dot2).  Shared by the solves and by the forward
// substitution fused into the factor.
#pragma once
#include "common.cuh"

namespace kc {

// (s, c) += w (hi + lo): TwoProduct of w hi, TwoSum into s, small terms into c.
// The _rn intrinsics keep every rounding where the error-free steps need it.
__device__ __forceinline__ void pair_add(float& s, float& c, float w, float hi, float lo) {
    const float p = __fmul_rn(w, hi);
    const float e = fmaf(w, hi, -p);
    const float ns = __fadd_rn(s, p);
    const float z = __fsub_rn(ns, s);
    const float er = __fadd_rn(__fsub_rn(s, __fsub_rn(ns, z)), __fsub_rn(p, z));
    s = ns;
    c = fmaf(w, lo, __fadd_rn(c, __fadd_rn(er, e)));
}
__device__ __forceinline__ void pair_merge(float& s, float& c, float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float z = __fsub_rn(t, s);
    const float er = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, er));
}
__device__ __forceinline__ float2 pair_of(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ double value_of(float2 p) { return (double)p.x + (double)p.y; }

}  // namespace kc
