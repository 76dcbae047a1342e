// Double-FP32 ("double-float") arithmetic: an FP64 operand carried as the
// unevaluated sum v = hi + lo of two FP32 numbers (hi = fp32(v),
// lo = fp32(v - hi)), 48 significand bits in the 8 bytes of an FP64 value.
// A product is formed without rounding error in its leading part (Dekker's
// product through a fused multiply-add: hi*hi exactly as p + e), the cross
// terms hi*lo + lo*hi are added to e, and the sum into the accumulator uses
// Knuth's TwoSum (Knuth, TAOCP vol. 2, 4.2.2; Ogita, Rump & Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 2005), so the accumulated error
// stays at a few units of 2^-48 relative to sum |h x|. Valid while the
// operands stay inside the FP32 exponent range (about 1e-30 .. 1e38 in
// magnitude for full accuracy).
#pragma once

#include <cuda_runtime.h>

namespace vbcsr {

struct DF {
    float hi, lo;
    __device__ __forceinline__ DF() {}
    __device__ __forceinline__ DF(int z) : hi((float)z), lo(0.f) {}
    __device__ __forceinline__ DF(float h) : hi(h), lo(0.f) {}
    __device__ __forceinline__ DF(float2 v) : hi(v.x), lo(v.y) {}
    __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ operator double() const { return (double)hi + (double)lo; }
};

// The _rn intrinsics below are never contracted into fused multiply-adds,
// which would break the exactness of the error-free transformations.

// a + b with the rounding error of the leading parts kept (TwoSum)
__device__ __forceinline__ DF operator+(DF a, DF b) {
    const float t = __fadd_rn(a.hi, b.hi);
    const float z = __fsub_rn(t, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, z)), __fsub_rn(b.hi, z));
    return DF(t, __fadd_rn(__fadd_rn(a.lo, b.lo), err));
}

__device__ __forceinline__ DF &operator+=(DF &a, DF b) {
    a = a + b;
    return a;
}

// keep the built-in overloads visible next to the DF one inside the namespace
using ::__shfl_xor_sync;

__device__ __forceinline__ DF __shfl_xor_sync(unsigned mask, DF v, int m) {
    return DF(::__shfl_xor_sync(mask, v.hi, m), ::__shfl_xor_sync(mask, v.lo, m));
}

// acc + a * x
__device__ __forceinline__ DF fmat(DF a, DF x, DF acc) {
    const float p = __fmul_rn(a.hi, x.hi);
    float e = __fmaf_rn(a.hi, x.hi, -p);     // exact: a.hi * x.hi = p + e
    e = __fmaf_rn(a.hi, x.lo, e);
    e = __fmaf_rn(a.lo, x.hi, e);
    const float t = __fadd_rn(acc.hi, p);    // TwoSum(acc.hi, p)
    const float z = __fsub_rn(t, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    return DF(t, __fadd_rn(acc.lo, __fadd_rn(e, err)));
}

}  // namespace vbcsr
