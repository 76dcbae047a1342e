// Complex FP64 block products (VBCSR_C128 operators, cplx.cuh) on the CUDA
// cores: the forward and adjoint kernels of fma_kernel.cuh with complex values,
// X and Y.
#include "cplx.cuh"
#include "fma_kernel.cuh"

namespace vbcsr {

cudaError_t launch_fma_c128(int B, bool trans, const ProdArgs &a, cudaStream_t s) {
    return launch_fma_family<double2, Cplx, double2, double2>(B, trans, a, s);
}

const void *fma_c128_kernel(bool trans, bool persistent, int B) {
    return fma_kernel_ptr<double2, Cplx, double2, double2>(trans, persistent, B);
}

}  // namespace vbcsr
