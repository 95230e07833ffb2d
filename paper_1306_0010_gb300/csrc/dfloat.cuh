// dfloat.cuh -- double-float arithmetic on the FP32 pipe, for the split path's stiff sources.
//
// A double-float is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48
// significant bits.  The building blocks are the error-free transforms of Knuth (TwoSum: a + b = s + e
// exactly), Dekker 1971 (Fast2Sum, for |a| >= |b|) and the FMA product (TwoProd: a b = p + e exactly,
// e = fma(a, b, -p)); the compound operations follow Joldes, Muller & Popescu, "Tight and rigorous error
// bounds for basic building blocks of double-word arithmetic" (ACM TOMS 44(2), 2017), whose relative
// error bounds are small multiples of u^2 (u = 2^-24) for normal operands.  The intrinsics with explicit
// rounding keep the compiler from contracting additions into FMAs or reassociating, which would break
// the transforms.  Values must stay inside the FP32 normal range (the callers check the results).
#pragma once
#include <cuda_runtime.h>

#include "fp_convert.cuh"

namespace rhd {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfl dneg(dfl x) { return {-x.hi, -x.lo}; }

// x + y, y an FP32 number (error <= 2 u^2)
__device__ __forceinline__ dfl dadd(dfl x, float y)
{
    const dfl s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}
// x + y for operands of any signs, accurate under cancellation (error <= 3 u^2 / (1 - 4u))
__device__ __forceinline__ dfl dadd(dfl x, dfl y)
{
    const dfl s = two_sum(x.hi, y.hi);
    const dfl t = two_sum(x.lo, y.lo);
    const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
// x + y for operands of the same sign (no cancellation): the cheaper sum
__device__ __forceinline__ dfl dadd_same(dfl x, dfl y)
{
    const dfl s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
// x y, y an FP32 number (error <= 2 u^2)
__device__ __forceinline__ dfl dmul(dfl x, float y)
{
    const dfl c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}
// x y (error <= 5 u^2)
__device__ __forceinline__ dfl dmul(dfl x, dfl y)
{
    const dfl c = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
    return fast_two_sum(c.hi, __fadd_rn(c.lo, __fmaf_rn(x.lo, y.hi, t)));
}
__device__ __forceinline__ dfl dsqr(dfl x)
{
    const dfl c = two_prod(x.hi, x.hi);
    return fast_two_sum(c.hi, __fmaf_rn(2.0f * x.hi, x.lo, c.lo));
}
// 1/x for x >= 1: the hardware FP32 reciprocal, one FP32 Newton-Raphson step, then the remaining
// residual e = 1 - x r (its high part exact by the FMA) as the low word r e
__device__ __forceinline__ dfl drcp(dfl x)
{
    float r = rcp(x.hi);
    r = __fmaf_rn(r, __fmaf_rn(-x.hi, r, 1.0f), r);
    const float e = __fmaf_rn(-x.lo, r, __fmaf_rn(-x.hi, r, 1.0f));
    return fast_two_sum(r, __fmul_rn(r, e));
}

// FP64 -> double-float by integer bit operations (no FP64-pipe conversion): round to nearest even of
// the 29 discarded mantissa bits; normal FP32 range (below: zero, beyond: infinity)
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u, a = hi & 0x7fffffffu;
    unsigned r = ((__funnelshift_l(lo, hi, 3) & 0x7fffffffu) ^ 0x40000000u);
    const unsigned rem = lo & 0x1fffffffu;
    r += (rem > 0x10000000u) || (rem == 0x10000000u && (r & 1u));  // a carry moves into the exponent
    r |= sign;
    r = a < 0x38100000u ? sign : r;
    r = a >= 0x47f00000u ? (sign | 0x7f800000u) : r;
    return __uint_as_float(r);
}
// x as a double-float (one FP64 subtraction, exact: x - hi is representable); relative error u^2
__device__ __forceinline__ dfl d2df(double x)
{
    const float h = d2f_rn(x);
    return {h, d2f_rn(x - f2d_exact(h))};
}
// x as an unnormalised double-float for the FP32 normal range, cheaply: hi is x truncated toward zero
// (its FP64 value is x with the 29 low mantissa bits cleared, one logic operation), lo = x - hi rounded
// to nearest (the subtraction is exact); relative error below 2^-47 (|lo| < ulp(hi)).  Values below the
// FP32 normal range become (0, 0).  The callers pass it to a double-float sum, which renormalises.
__device__ __forceinline__ dfl d2df_fast(double x)
{
    const float h = d2f_trunc(x);
    const double h64 = h != 0.0f ? __hiloint2double(__double2hiint(x), __double2loint(x) & (int)0xe0000000) : 0.0;
    return {h, d2f_rn(x - h64)};
}
// a double-float of a host-side FP64 constant (per thread, outside the loops)
__device__ __forceinline__ dfl dconst(double x) { return d2df(x); }
// hi + lo in FP64 (one FP64 addition)
__device__ __forceinline__ double df2d(dfl x) { return f2d_exact(x.hi) + f2d_exact(x.lo); }

}  // namespace rhd
