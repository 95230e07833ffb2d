// fp_convert.cuh -- FP64 <-> FP32 conversions by integer bit operations (shared by the kernel
// translation units).
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

}  // namespace rhd
