// FP64-accurate block products in double-FP32 ("double-float") arithmetic.
//
// GB300 executes FP32 FMAs about 60 times faster than FP64 FMAs, so FP64
// operands are carried as unevaluated sums v = hi + lo of two FP32 numbers
// (hi = fp32(v), lo = fp32(v - hi)): 48 significand bits, the same 8 bytes per
// value as FP64. A product is formed without rounding error in its leading
// part (Dekker's product through a fused multiply-add: hi*hi exactly as
// p + e), the cross terms hi*lo + lo*hi are added to e, and the sum into the
// accumulator uses Knuth's TwoSum (Knuth, TAOCP vol. 2, 4.2.2; Ogita, Rump &
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005), so the
// accumulated error stays at a few units of 2^-48 relative to sum |h x|. The
// epilogue adds hi and lo in FP64. Valid while the operands stay inside the
// FP32 exponent range (about 1e-30 .. 1e38 in magnitude for full accuracy).
#include "fma_kernel.cuh"

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

cudaError_t launch_fma_df(int B, bool trans, const ProdArgs &a, cudaStream_t s) {
    return launch_fma_family<float2, DF, double, float2>(B, trans, a, s);
}

const void *fma_df_kernel(bool trans, bool persistent) {
    return fma_kernel_ptr<float2, DF, double, float2>(trans, persistent);
}

// hi/lo split of FP64 values into FP32 pairs
__global__ void split_df_kernel(const double *in, int64_t ld, int64_t rows, int64_t k, float2 *out) {
    const int64_t n = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - r * k;
        const double v = in[r * ld + c];
        const float hi = (float)v;
        out[e] = make_float2(hi, (float)(v - (double)hi));
    }
}

cudaError_t launch_split_df(int64_t rows, int64_t k, const double *in, int64_t ld, float2 *out, cudaStream_t s) {
    const int64_t need = (rows * k + 255) / 256;
    if (need == 0) return cudaSuccess;
    split_df_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(in, ld, rows, k, out);
    return cudaGetLastError();
}

}  // namespace vbcsr
