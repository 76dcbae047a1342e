// CUDA-core form of the tensor-core precision modes (TF32, TF32X3, BF16X2),
// for products too thin to fill an MMA tile (a matrix-vector product, or a
// scalar operator whose rows are single rows): the operands are cut into the
// same pieces the tensor-core kernel feeds its MMAs (hi = the value rounded to
// the piece format, lo = the rounded remainder), the same piece products are
// formed (hi*hi, hi*lo, lo*hi; hi*hi alone for TF32) - each exact in FP32,
// since a piece has at most 11 significand bits - and they are accumulated in
// FP32, one rounding per product.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.cuh"

namespace vbcsr {

__device__ __forceinline__ float round_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// The operand pieces of the BF16X2 mode as one 32-bit word, formed once per
// value as the kernels would form them: FP32 value v, hi = bf16_rn(v) in the
// low half, lo = bf16_rn(v - hi) in the high half. Used by the one-pass split
// of values and X and by the tensor-core epilogue that writes the next
// Chebyshev vector in this form.
__device__ __forceinline__ uint32_t bf16_pieces(double x) {
    const float v = (float)x;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    return (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(l) << 16);
}

// An operand as its pieces, or (hi only) an FP32 accumulator.
template <int MODE>
struct SplitF {
    float hi, lo;
    __device__ __forceinline__ SplitF() {}
    __device__ __forceinline__ SplitF(int z) : hi((float)z), lo(0.f) {}
    __device__ __forceinline__ explicit SplitF(float v) {
        if (MODE == kBF16X2Presplit) {
            // v carries a packed word split earlier: hi bf16 in the low half, lo in the high
            const uint32_t w = __float_as_uint(v);
            hi = __uint_as_float(w << 16);
            lo = __uint_as_float(w & 0xffff0000u);
        } else if (MODE == kBF16X2) {
            hi = round_bf16(v);
            lo = round_bf16(v - hi);
        } else {
            hi = round_tf32(v);
            lo = MODE == kTF32X3 ? round_tf32(v - hi) : 0.f;
        }
    }
    __device__ __forceinline__ operator double() const { return (double)hi; }
};

// accumulators
template <int MODE>
__device__ __forceinline__ SplitF<MODE> operator+(SplitF<MODE> a, SplitF<MODE> b) {
    SplitF<MODE> r(0);
    r.hi = a.hi + b.hi;
    return r;
}

template <int MODE>
__device__ __forceinline__ SplitF<MODE> &operator+=(SplitF<MODE> &a, SplitF<MODE> b) {
    a.hi += b.hi;
    return a;
}

using ::__shfl_xor_sync;

template <int MODE>
__device__ __forceinline__ SplitF<MODE> __shfl_xor_sync(unsigned mask, SplitF<MODE> v, int m) {
    SplitF<MODE> r(0);
    r.hi = ::__shfl_xor_sync(mask, v.hi, m);
    return r;
}

// acc + a * x over the piece products
template <int MODE>
__device__ __forceinline__ SplitF<MODE> fmat(SplitF<MODE> a, SplitF<MODE> x, SplitF<MODE> acc) {
    float s = fmaf(a.hi, x.hi, acc.hi);
    if (MODE != kTF32) {
        s = fmaf(a.hi, x.lo, s);
        s = fmaf(a.lo, x.hi, s);
    }
    SplitF<MODE> r(0);
    r.hi = s;
    return r;
}

}  // namespace vbcsr
