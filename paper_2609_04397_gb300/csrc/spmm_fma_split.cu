// Forward products of an FP64 operator in the tensor-core precision modes on
// the CUDA cores (split.cuh), for panels of k <= kSplitFmaMaxK columns: one
// persistent launch over every item, FP32 value copy (BF16X2: the packed
// (hi, lo) bf16 words, split once per value update), X converted once per
// call, FP64 epilogue.
#include "split.cuh"
#include "fma_kernel.cuh"

namespace vbcsr {

namespace {

template <int MODE>
cudaError_t launch_mode(const ProdArgs &a, cudaStream_t s) {
    const size_t smem = fma_smem_bytes(false, a.warps);
    cudaError_t e = launch_smem_opt_in(fma_persistent_kernel<false, float, SplitF<MODE>, double, float>, smem);
    if (e != cudaSuccess) return e;
    fma_persistent_kernel<false, float, SplitF<MODE>, double, float><<<a.grid, a.warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fma_split(int mode, const ProdArgs &a, cudaStream_t s) {
    switch (mode) {
        case kTF32: return launch_mode<kTF32>(a, s);
        case kTF32X3: return launch_mode<kTF32X3>(a, s);
        case kBF16X2: return launch_mode<kBF16X2>(a, s);
        case kBF16X2Presplit: return launch_mode<kBF16X2Presplit>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

const void *fma_split_kernel(int mode) {
    switch (mode) {
        case kTF32: return (const void *)fma_persistent_kernel<false, float, SplitF<kTF32>, double, float>;
        case kTF32X3: return (const void *)fma_persistent_kernel<false, float, SplitF<kTF32X3>, double, float>;
        case kBF16X2: return (const void *)fma_persistent_kernel<false, float, SplitF<kBF16X2>, double, float>;
        case kBF16X2Presplit:
            return (const void *)fma_persistent_kernel<false, float, SplitF<kBF16X2Presplit>, double, float>;
        default: return nullptr;
    }
}

}  // namespace vbcsr
