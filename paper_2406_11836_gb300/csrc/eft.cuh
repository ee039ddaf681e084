// Error-free transformations of float arithmetic (Knuth's two-sum, Dekker's fast two-sum,
// the fma two-product) and a compensated dot product in the style of Ogita, Rump and
// Oishi's Dot2: sums and products carried as an unevaluated pair hi + lo of floats, so that
// depths and order keys keep about twice the float precision.
#pragma once

namespace rgs {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// a0*b0 + a1*b1 + a2*b2 + c as hi + lo (Ogita-Rump-Oishi Dot2 style)
__device__ __forceinline__ void dot3_plus(float a0, float b0, float a1, float b1, float a2, float b2, float c,
                                          float& hi, float& lo) {
    float s, e, p, q, t;
    two_prod(a0, b0, s, e);
    two_prod(a1, b1, p, q);
    two_sum(s, p, s, t);
    e = __fadd_rn(e, __fadd_rn(q, t));
    two_prod(a2, b2, p, q);
    two_sum(s, p, s, t);
    e = __fadd_rn(e, __fadd_rn(q, t));
    two_sum(s, c, s, t);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, hi, lo);
}

}  // namespace rgs
