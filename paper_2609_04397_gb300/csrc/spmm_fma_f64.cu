// FP64 CUDA-core block product (values, accumulation and panels in FP64).
#include "fma_kernel.cuh"

namespace vbcsr {

cudaError_t launch_fma_f64(int B, bool trans, const ProdArgs &a, cudaStream_t s) {
    return launch_fma_family<double, double, double, double>(B, trans, a, s);
}

const void *fma_f64_kernel(bool trans, bool persistent, int B) {
    return fma_kernel_ptr<double, double, double, double>(trans, persistent, B);
}

}  // namespace vbcsr
