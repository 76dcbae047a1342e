// FP32 CUDA-core block products: an FP32 operator on FP32 panels, and FP32
// arithmetic on the FP32 value copy of an FP64 operator (X converted to FP32
// once per call before the launch, FP64 epilogue into the FP64 Y).
#include "fma_kernel.cuh"

namespace vbcsr {

cudaError_t launch_fma_f32(int B, bool trans, const ProdArgs &a, cudaStream_t s) {
    return launch_fma_family<float, float, float, float>(B, trans, a, s);
}

cudaError_t launch_fma_f32_on_f64(int B, bool trans, const ProdArgs &a, cudaStream_t s) {
    return launch_fma_family<float, float, double, float>(B, trans, a, s);
}

const void *fma_f32_kernel(bool trans, bool persistent, int B, bool ring) {
    return fma_kernel_ptr<float, float, float, float>(trans, persistent, B, false, ring);
}
const void *fma_f32_on_f64_kernel(bool trans, bool persistent, int B, bool ring) {
    return fma_kernel_ptr<float, float, double, float>(trans, persistent, B, false, ring);
}

}  // namespace vbcsr
