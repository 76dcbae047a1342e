// CUDA-core (FMA) forward and adjoint block product.
//
// One warp owns one work item: B consecutive output rows of a block row
// (forward) or of a block column (adjoint). The item's "virtual columns" are
// staged in shared memory:
//   forward  virtual column t of block row i is panel column t; its X row is
//            c_j + q for the block j and offset q that the column belongs to,
//            and output row p reads P_i[p, t] (stride Kp between rows);
//   adjoint  virtual column u of block column j is (i, p) for every block
//            (i, j) and p < b_i; its X row is r_i + p and output row q reads
//            H_ij[p, q0 + q], contiguous in q (Eq. 1).
// Lanes split as (tg, c): c = lane % KC picks an output column of the pass,
// tg = lane / KC strides the virtual columns. Each lane keeps B partial sums
// in registers; a butterfly over the tg lanes finishes them, and each output
// entry is written once by one lane (no atomics). The epilogue applies
// alpha, beta, gamma * Z and accumulates the optional FP64 dot with R.
#pragma once

#include "internal.cuh"

namespace vbcsr {

template <typename T>
__device__ __forceinline__ T ld_ro(const T *p) { return __ldg(p); }

__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

template <int B, bool TRANS, typename TV, typename TA, typename TX>
__global__ void __launch_bounds__(256, 2) fma_product_kernel(ProdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw) + warp * kKMax;
    int64_t *s_a = reinterpret_cast<int64_t *>(smem_raw + (size_t)warps * kKMax * sizeof(int32_t)) +
                   warp * kKMax;

    const int KC = a.kc;
    const int TG = 32 / KC;
    const int cl = lane % KC;
    const int tg = lane / KC;
    const TV *__restrict__ vals = static_cast<const TV *>(a.values);
    const TX *__restrict__ X = static_cast<const TX *>(a.X);
    TX *__restrict__ Y = static_cast<TX *>(a.Y);
    const TX *__restrict__ Z = static_cast<const TX *>(a.Z);
    const TX *__restrict__ R = static_cast<const TX *>(a.R);
    const TX alpha = (TX)a.alpha, beta = (TX)a.beta, gamma = (TX)a.gamma;
    const bool do_prod = a.alpha != 0.0;
    double dot = 0.0;

    for (int64_t it = (int64_t)blockIdx.x * warps + warp; it < a.n_items;
         it += (int64_t)gridDim.x * warps) {
        const WorkItem w = a.items[it];
        for (int64_t c0 = 0; c0 < a.k; c0 += KC) {
            const int64_t c = c0 + cl;
            const bool cv = c < a.k;
            TA acc[B];
#pragma unroll
            for (int p = 0; p < B; ++p) acc[p] = (TA)0;

            if (do_prod) {
                for (int t0 = 0; t0 < w.K; t0 += kKMax) {
                    const int tn = min(kKMax, w.K - t0);
                    if (c0 == 0 || w.K > kKMax) {
                        __syncwarp();
                        for (int e = lane; e < w.nlist; e += 32) {
                            const int64_t l = w.lbegin + e;
                            if (!TRANS) {
                                const int xr = a.fl.xrow[l], pc = a.fl.pcol[l], wd = a.fl.w[l];
                                const int lo = max(pc, t0), hi = min(pc + wd, t0 + tn);
                                for (int t = lo; t < hi; ++t) s_x[t - t0] = xr + (t - pc);
                            } else {
                                const int64_t pb = a.tl.pbase[l];
                                const int kp = a.tl.kp[l], bi = a.tl.bi[l];
                                const int xr = a.tl.xrow[l], vc = a.tl.vcol[l];
                                const int lo = max(vc, t0), hi = min(vc + bi, t0 + tn);
                                for (int t = lo; t < hi; ++t) {
                                    s_x[t - t0] = xr + (t - vc);
                                    s_a[t - t0] = pb + (int64_t)(t - vc) * kp + w.Kp;
                                }
                            }
                        }
                        __syncwarp();
                    }
                    for (int t = tg; t < tn; t += TG) {
                        const int xr = s_x[t];
                        if (a.debug_checks && (xr < 0 || xr >= a.x_rows)) {
                            atomicExch(a.err, 1);
                            continue;
                        }
                        const TA x = cv ? (TA)ld_ro(X + (int64_t)xr * a.ldx + c) : (TA)0;
                        if (!TRANS) {
                            const TV *v = vals + w.vbase + t0 + t;
                            const int64_t kp = w.Kp;
#pragma unroll
                            for (int p = 0; p < B; ++p) acc[p] = fmat((TA)ld_ro(v + p * kp), x, acc[p]);
                        } else {
                            const TV *v = vals + s_a[t];
#pragma unroll
                            for (int p = 0; p < B; ++p) acc[p] = fmat((TA)ld_ro(v + p), x, acc[p]);
                        }
                    }
                }
            }
            // finish the partial sums over the tg lanes that share column c
            for (int m = KC; m < 32; m <<= 1) {
#pragma unroll
                for (int p = 0; p < B; ++p) acc[p] += __shfl_xor_sync(0xffffffffu, acc[p], m);
            }
#pragma unroll
            for (int p = 0; p < B; ++p) {
                if ((p % TG) == tg && cv) {
                    const int64_t row = w.yrow + p;
                    TX *yp = Y + row * a.ldy + c;
                    TX r = alpha * (TX)acc[p];
                    if (a.beta != 0.0) r += beta * *yp;
                    if (a.gamma != 0.0) r += gamma * Z[row * a.ldz + c];
                    *yp = r;
                    if (a.partials) dot += (double)R[row * a.ldr + c] * (double)r;
                }
            }
        }
    }

    if (a.partials) {
        // fixed-order CTA reduction of the dot partials
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

template <typename TV, typename TA, typename TX>
cudaError_t launch_fma_family(int B, bool trans, const ProdArgs &a, cudaStream_t s) {
    const int threads = a.warps * 32;
    const size_t smem = fma_smem_bytes(trans, a.warps);
#define VBCSR_FMA_CASE(NB)                                                                        \
    case NB:                                                                                      \
        if (trans) fma_product_kernel<NB, true, TV, TA, TX><<<a.grid, threads, smem, s>>>(a);    \
        else fma_product_kernel<NB, false, TV, TA, TX><<<a.grid, threads, smem, s>>>(a);         \
        break;
    switch (B) {
        VBCSR_FMA_CASE(1) VBCSR_FMA_CASE(2) VBCSR_FMA_CASE(3) VBCSR_FMA_CASE(4)
        VBCSR_FMA_CASE(5) VBCSR_FMA_CASE(6) VBCSR_FMA_CASE(7) VBCSR_FMA_CASE(8)
        VBCSR_FMA_CASE(9) VBCSR_FMA_CASE(10) VBCSR_FMA_CASE(11) VBCSR_FMA_CASE(12)
        VBCSR_FMA_CASE(13) VBCSR_FMA_CASE(14) VBCSR_FMA_CASE(15) VBCSR_FMA_CASE(16)
        default: return cudaErrorInvalidValue;
    }
#undef VBCSR_FMA_CASE
    return cudaGetLastError();
}

template <typename TV, typename TA, typename TX>
const void *fma_kernel_ptr(bool trans) {
    // B = 16 is the largest register footprint; used for the occupancy cap
    return trans ? (const void *)fma_product_kernel<16, true, TV, TA, TX>
                 : (const void *)fma_product_kernel<16, false, TV, TA, TX>;
}

}  // namespace vbcsr
