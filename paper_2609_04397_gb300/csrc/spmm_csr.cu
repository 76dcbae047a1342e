// Scalar (CSR) operators: every block is 1 x 1, so a block row is one scalar
// row and the panel path would spend a whole warp on each row. Here L lanes
// share a row (32 / L rows per warp): each lane walks the row's entries with
// stride L, reads the column from the plan's block list and the X row
// segment of CW output columns (CW = 1, 4 or 8, chosen from k so that no
// masked FP64 instruction is issued: GB300's FP64 pipe charges a warp
// instruction whatever its mask), and the L lanes finish the sums with a
// butterfly. Every output entry is written once.
//
// The arithmetic kinds share the code (value type TV, accumulator TA, X type
// TXI, Y type TX): FP64, FP32, FP32 products of an FP64 operator (FP32 value
// copy, X converted once per call), double-FP32 (hi/lo value copy and X) and
// the piece products of the tensor-core modes (split.cuh) - a scalar row has
// one row, too thin for an MMA tile.
#include <type_traits>

#include "df.cuh"
#include "split.cuh"
#include "fma_kernel.cuh"

namespace vbcsr {

template <typename TV, typename TA, typename TX, typename TXI, int L, int CW>
__global__ void __launch_bounds__(256) csr_kernel(ProdArgs a) {
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / L, lr = lane % L;
    constexpr int RPW = 32 / L;   // rows per warp
    const TV *__restrict__ vals = static_cast<const TV *>(a.values);
    const TXI *__restrict__ X = static_cast<const TXI *>(a.X);
    TX *__restrict__ Y = static_cast<TX *>(a.Y);
    const EpiScalars<TX> sc = epi_scalars<TX>(a);
    const TX alpha = sc.alpha, beta = sc.beta, gamma = sc.gamma;
    const bool do_prod = a.alpha != 0.0;
    double dot = 0.0;
    for (int64_t base = ((int64_t)blockIdx.x * warps + warp) * RPW; base < a.n_items;
         base += (int64_t)gridDim.x * warps * RPW) {
        const int64_t it = base + sub;
        const bool valid = it < a.n_items;
        WorkItem w;
        w.K = 0;
        if (valid) w = a.items[it];
        for (int64_t c0 = 0; c0 < a.k; c0 += CW) {
            const int nc = (int)min((int64_t)CW, a.k - c0);   // columns of this tile (uniform)
            TA acc[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) acc[j] = TA(0);
            if (do_prod) {
                for (int e = lr; e < w.K; e += L) {
                    const TA v = TA(__ldg(vals + w.vbase + e));
                    const TXI *xp = X + (int64_t)__ldg(a.fl.xrow + w.lbegin + e) * a.ldx + c0;
                    if (nc == CW) {
#pragma unroll
                        for (int j = 0; j < CW; ++j) acc[j] = fmat(v, TA(__ldg(xp + j)), acc[j]);
                    } else {
#pragma unroll
                        for (int j = 0; j < CW; ++j)
                            if (j < nc) acc[j] = fmat(v, TA(__ldg(xp + j)), acc[j]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                if (j >= nc) break;   // uniform across the warp
#pragma unroll
                for (int m = L / 2; m > 0; m >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], m);
            }
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                if (valid && lr == (j % L) && c0 + j < a.k) {
                    const int64_t row = w.yrow, c = c0 + j;
                    TX r = alpha * (TX)acc[j];
                    if (a.beta_nz) r += beta * Y[row * a.ldy + c];
                    if (a.gamma_nz) r += gamma * static_cast<const TX *>(a.Z)[row * a.ldz + c];
                    Y[row * a.ldy + c] = r;
                    if (a.partials) dot += (double)static_cast<const TX *>(a.R)[row * a.ldr + c] * (double)r;
                }
            }
        }
    }
    if (a.partials) {
        for (int m = 16; m > 0; m >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, m);
        __shared__ double s_dot[32];
        __syncthreads();
        if (lane == 0) s_dot[warp] = dot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < warps; ++i) s += s_dot[i];
            a.partials[blockIdx.x] = s;
        }
    }
}

namespace {

int csr_cw(int64_t k) { return k == 1 ? 1 : (k <= 4 ? 4 : 8); }

// Kernel of lane count L and column tile CW for arithmetic kind <TV, TA, TX, TXI>.
// FP64 and double-FP32 rows use 2, 4 or 8 lanes (an FP64 instruction, or the
// dozen FP32 instructions of a double-FP32 step, is dear: few lanes keep the
// finishing butterfly short); the FP32 kinds use 4, 8, 16 or 32.
template <typename TV, typename TA, typename TX, typename TXI, int CW>
const void *ptr_l(int L) {
    if constexpr (std::is_same<TA, double>::value || std::is_same<TA, DF>::value) {
        switch (L) {
            case 2: return (const void *)csr_kernel<TV, TA, TX, TXI, 2, CW>;
            case 4: return (const void *)csr_kernel<TV, TA, TX, TXI, 4, CW>;
            case 8: return (const void *)csr_kernel<TV, TA, TX, TXI, 8, CW>;
            default: return nullptr;
        }
    } else {
        switch (L) {
            case 4: return (const void *)csr_kernel<TV, TA, TX, TXI, 4, CW>;
            case 8: return (const void *)csr_kernel<TV, TA, TX, TXI, 8, CW>;
            case 16: return (const void *)csr_kernel<TV, TA, TX, TXI, 16, CW>;
            case 32: return (const void *)csr_kernel<TV, TA, TX, TXI, 32, CW>;
            default: return nullptr;
        }
    }
}

template <typename TV, typename TA, typename TX, typename TXI>
const void *ptr_k(int L, int64_t k) {
    const int cw = csr_cw(k);
    return cw == 1 ? ptr_l<TV, TA, TX, TXI, 1>(L)
                   : (cw == 4 ? ptr_l<TV, TA, TX, TXI, 4>(L) : ptr_l<TV, TA, TX, TXI, 8>(L));
}

}  // namespace

int csr_lane_class(int kind) { return (kind == kCsrF64 || kind == kCsrDF) ? 0 : 1; }

const void *csr_kernel_ptr(int kind, int L, int64_t k) {
    switch (kind) {
        case kCsrF64: return ptr_k<double, double, double, double>(L, k);
        case kCsrF32: return ptr_k<float, float, float, float>(L, k);
        case kCsrF32OnF64: return ptr_k<float, float, double, float>(L, k);
        case kCsrDF: return ptr_k<float2, DF, double, float2>(L, k);
        case kCsrSplitTF32: return ptr_k<float, SplitF<kTF32>, double, float>(L, k);
        case kCsrSplitTF32X3: return ptr_k<float, SplitF<kTF32X3>, double, float>(L, k);
        case kCsrSplitBF16X2: return ptr_k<float, SplitF<kBF16X2>, double, float>(L, k);
        default: return nullptr;
    }
}

cudaError_t launch_csr(int kind, int L, const ProdArgs &a, cudaStream_t s) {
    const void *kern = csr_kernel_ptr(kind, L, a.k);
    if (!kern) return cudaErrorInvalidValue;
    void *args[] = {const_cast<ProdArgs *>(&a)};
    return cudaLaunchKernel(kern, dim3(a.grid), dim3(a.warps * 32), args, 0, s);
}

}  // namespace vbcsr
