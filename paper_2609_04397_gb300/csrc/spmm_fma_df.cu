// FP64-accurate block products in double-FP32 arithmetic (df.cuh).
//
// GB300 executes FP32 FMAs about 60 times faster than FP64 FMAs, so the FP64
// operands are carried as hi/lo FP32 pairs: values from a split copy of the
// value pages, X split once per call. The epilogue adds hi and lo in FP64.
#include "df.cuh"
#include "fma_kernel.cuh"

namespace vbcsr {

cudaError_t launch_fma_df(int B, bool trans, const ProdArgs &a, cudaStream_t s, bool narrow) {
    return launch_fma_family<float2, DF, double, float2>(B, trans, a, s, narrow);
}

const void *fma_df_kernel(bool trans, bool persistent, int B, bool narrow, bool ring) {
    return fma_kernel_ptr<float2, DF, double, float2>(trans, persistent, B, narrow, ring);
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
