// fp_convert.cuh -- FP64 <-> FP32 conversions by integer bit operations, and the square roots and
// reciprocals of the kernels (shared by the kernel translation units).
#pragma once
#include <cuda_runtime.h>

namespace rhd {

// FP64 <-> FP32 conversions without the FP64 pipe (which runs at a small fraction of the FP32 rate
// on this part): truncation of the FP64 value to FP32 (normal range; underflow to 0, overflow to
// inf), and the exact widening of an FP32 value (denormals flushed), by integer bit operations.
__device__ __forceinline__ float d2f_trunc(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u, a = hi & 0x7fffffffu;
    // (hi:lo) << 3 puts the exponent's low 8 bits above the 23 leading mantissa bits; in the FP32
    // normal range the rebias (exponent - 896) mod 256 is those 8 bits with the top one flipped
    unsigned r = ((__funnelshift_l(lo, hi, 3) & 0x7fffffffu) ^ 0x40000000u) | sign;
    r = a < 0x38100000u ? sign : r;                   // below the FP32 normal range: signed zero
    r = a >= 0x47f00000u ? (sign | 0x7f800000u) : r;  // beyond it: signed infinity
    return __uint_as_float(r);
}
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, a = b & 0x7fffffffu;
    // exponent and mantissa shifted into place with the exponent rebiased by 896 (1023 - 127)
    unsigned hi = ((a >> 3) + 0x38000000u) | sign, lo = b << 29;
    hi = a < 0x00800000u ? sign : hi;  // zero and denormals: signed zero
    lo = a < 0x00800000u ? 0u : lo;
    hi = a >= 0x7f800000u ? ((a >> 3) | 0x7ff00000u | sign) : hi;
    return __hiloint2double((int)hi, (int)lo);
}

// Square root and reciprocal.  Split path: the hardware approximations (MUFU, about 1-2 ulp), well
// inside the FP32 error budget of the fluxes.  FP64 path: IEEE square root; the reciprocal is the
// hardware FP64 approximation refined by two Newton-Raphson steps r <- r + r (1 - x r), each of which
// squares the relative error (from below 2^-20 to below 2^-40, then to rounding): within an ulp or
// two of 1/x, not the correctly rounded quotient, which the FP64 path does not need (its bound
// against the oracle is 1e-12) and which costs several more FP64 operations.  x = 0, +-inf and FP64
// denormals (flushed) give NaN.
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
// 1/sqrt(x) for normal x > 0, FP64: the hardware approximation refined by two Newton-Raphson steps for
// f(y) = y^-2 - x, y <- y + (y/2)(1 - x y^2), each of which squares the relative error (within an ulp or
// two of 1/sqrt(x); tested against CUDA's 1/sqrt).  x sqrt(x)^-1 is then the square root as well.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double r = __fma_rn(-__dmul_rn(x, y), y, 1.0);
    y = __fma_rn(__dmul_rn(0.5, y), r, y);
    r = __fma_rn(-__dmul_rn(x, y), y, 1.0);
    return __fma_rn(__dmul_rn(0.5, y), r, y);
}
__device__ __forceinline__ float rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Explicitly rounded arithmetic: never contracted into FMAs or reassociated by the compiler, so every
// inlined copy of an expression written with these rounds the same way.  Quantities that two tiles (or a
// tile's own cells and its halo) compute separately use them, so that both copies get the same bits
// (a face flux shared by two tiles, a uniform state that must stay uniform).
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }

}  // namespace rhd
