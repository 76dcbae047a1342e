// Tensor-core block products for the mixed-precision modes (TF32, TF32X3,
// BF16X2) on the FP32 copy of the values, with FP32 accumulation and the
// epilogue (alpha, beta, gamma * Z, dot with R) in the panel dtype.
//
// Work decomposition is that of the CUDA-core kernel (one warp per work item
// of up to 16 output rows; virtual columns staged in shared memory). The item
// is a 16-row MMA tile: rows >= B are zero. Each step consumes 16 virtual
// columns; lane (g = lane / 4, t = lane % 4) holds output rows g and g + 8 and
// the virtual columns 4t .. 4t+3 of the step, loaded as one float4 per row in
// the forward direction. Because the order of the reduction index is free,
// those four columns are assigned to the k-slots of the fragments so that A
// and B use the same columns:
//   m16n8k8  (TF32): MMA 0 slots (t, t+4) <- columns (4t, 4t+1),
//                    MMA 1 slots (t, t+4) <- columns (4t+2, 4t+3);
//   m16n8k16 (BF16): slots (2t, 2t+1, 2t+8, 2t+9) <- columns 4t .. 4t+3.
// Split modes: v = hi + lo, hi = rn(v), lo = rn(v - hi) in the piece format;
// the products hi*hi + hi*lo + lo*hi accumulate in the same FP32 registers.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace vbcsr {

namespace {

constexpr int kTF32 = 2, kTF32X3 = 3, kBF16X2 = 4;

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo_k, hi_k);   // .x (low half) = lower k index
    return *reinterpret_cast<uint32_t *>(&h);
}

// Pieces of four consecutive virtual columns c0..c3 of one fragment row.
struct Pieces {
    uint32_t hi[4], lo[4];   // TF32 modes: one tf32 per column
    uint32_t bh[2], bl[2];   // BF16X2: packed pairs (c0,c1), (c2,c3)
};

template <int MODE>
__device__ __forceinline__ void split4(const float (&v)[4], Pieces &p) {
    if (MODE == kBF16X2) {
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            h[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
            l[j] = v[j] - h[j];
        }
        p.bh[0] = pack_bf16(h[0], h[1]);
        p.bh[1] = pack_bf16(h[2], h[3]);
        p.bl[0] = pack_bf16(l[0], l[1]);
        p.bl[1] = pack_bf16(l[2], l[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            p.hi[j] = to_tf32(v[j]);
            if (MODE == kTF32X3) p.lo[j] = to_tf32(v[j] - __uint_as_float(p.hi[j]));
        }
    }
}

// acc += A(rows g, g+8; 16 columns) * B(16 columns; 8 output columns)
template <int MODE>
__device__ __forceinline__ void step(float (&acc)[4], const Pieces &ag, const Pieces &ag8, const Pieces &b) {
    if (MODE == kBF16X2) {
        mma_bf16(acc, ag.bh[0], ag8.bh[0], ag.bh[1], ag8.bh[1], b.bh[0], b.bh[1]);
        mma_bf16(acc, ag.bh[0], ag8.bh[0], ag.bh[1], ag8.bh[1], b.bl[0], b.bl[1]);
        mma_bf16(acc, ag.bl[0], ag8.bl[0], ag.bl[1], ag8.bl[1], b.bh[0], b.bh[1]);
    } else {
        mma_tf32(acc, ag.hi[0], ag8.hi[0], ag.hi[1], ag8.hi[1], b.hi[0], b.hi[1]);
        mma_tf32(acc, ag.hi[2], ag8.hi[2], ag.hi[3], ag8.hi[3], b.hi[2], b.hi[3]);
        if (MODE == kTF32X3) {
            mma_tf32(acc, ag.hi[0], ag8.hi[0], ag.hi[1], ag8.hi[1], b.lo[0], b.lo[1]);
            mma_tf32(acc, ag.hi[2], ag8.hi[2], ag.hi[3], ag8.hi[3], b.lo[2], b.lo[3]);
            mma_tf32(acc, ag.lo[0], ag8.lo[0], ag.lo[1], ag8.lo[1], b.hi[0], b.hi[1]);
            mma_tf32(acc, ag.lo[2], ag8.lo[2], ag.lo[3], ag8.lo[3], b.hi[2], b.hi[3]);
        }
    }
}

template <int MODE, bool TRANS, typename TX, int NT>
__global__ void __launch_bounds__(128, 4) mma_product_kernel(ProdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw) + warp * kKMax;
    int64_t *s_a = reinterpret_cast<int64_t *>(smem_raw + (size_t)warps * kKMax * sizeof(int32_t)) +
                   warp * kKMax;
    const float *__restrict__ vals = static_cast<const float *>(a.values);
    const TX *__restrict__ X = static_cast<const TX *>(a.X);
    TX *__restrict__ Y = static_cast<TX *>(a.Y);
    const TX *__restrict__ Z = static_cast<const TX *>(a.Z);
    const TX *__restrict__ R = static_cast<const TX *>(a.R);
    const TX alpha = (TX)a.alpha, beta = (TX)a.beta, gamma = (TX)a.gamma;
    const bool do_prod = a.alpha != 0.0;
    double dot = 0.0;

    for (int64_t it = (int64_t)blockIdx.x * warps + warp; it < a.n_items; it += (int64_t)gridDim.x * warps) {
        const WorkItem w = a.items[it];
        for (int64_t n0 = 0; n0 < a.k; n0 += 8 * NT) {
            float acc[NT][4];
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[n][j] = 0.f;

            if (do_prod) {
                for (int t0 = 0; t0 < w.K; t0 += kKMax) {
                    const int tn = min(kKMax, w.K - t0);
                    if (n0 == 0 || w.K > kKMax) {
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
                    for (int c16 = 0; c16 < tn; c16 += 16) {
                        const int cl = c16 + 4 * t4;   // first of this lane's 4 columns, window-relative
                        float va[4] = {0.f, 0.f, 0.f, 0.f}, vb[4] = {0.f, 0.f, 0.f, 0.f};
                        if (!TRANS) {
                            const int64_t col = (int64_t)t0 + cl;
                            if (col < w.Kp) {   // Kp is a multiple of 4: the float4 is inside the row
                                if (g < w.B) {
                                    const float4 q = __ldg(reinterpret_cast<const float4 *>(
                                        vals + w.vbase + (int64_t)g * w.Kp + col));
                                    va[0] = q.x; va[1] = q.y; va[2] = q.z; va[3] = q.w;
                                }
                                if (g + 8 < w.B) {
                                    const float4 q = __ldg(reinterpret_cast<const float4 *>(
                                        vals + w.vbase + (int64_t)(g + 8) * w.Kp + col));
                                    vb[0] = q.x; vb[1] = q.y; vb[2] = q.z; vb[3] = q.w;
                                }
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (cl + j < tn) {
                                    const float *base = vals + s_a[cl + j];
                                    if (g < w.B) va[j] = __ldg(base + g);
                                    if (g + 8 < w.B) vb[j] = __ldg(base + g + 8);
                                }
                            }
                        }
                        Pieces pa, pb;
                        split4<MODE>(va, pa);
                        split4<MODE>(vb, pb);
                        int xr[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) xr[j] = (cl + j < tn) ? s_x[cl + j] : -1;
#pragma unroll
                        for (int n = 0; n < NT; ++n) {
                            const int64_t col = n0 + n * 8 + g;
                            float xv[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                xv[j] = (xr[j] >= 0 && col < a.k) ? (float)__ldg(X + (int64_t)xr[j] * a.ldx + col)
                                                                 : 0.f;
                            Pieces px;
                            split4<MODE>(xv, px);
                            step<MODE>(acc[n], pa, pb, px);
                        }
                    }
                }
            }
            // epilogue: acc[n] = {(g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)} of tile n
#pragma unroll
            for (int n = 0; n < NT; ++n) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = g + ((j >> 1) << 3);
                    const int64_t col = n0 + n * 8 + 2 * t4 + (j & 1);
                    if (r < w.B && col < a.k) {
                        const int64_t row = w.yrow + r;
                        TX *yp = Y + row * a.ldy + col;
                        TX v = alpha * (TX)acc[n][j];
                        if (a.beta != 0.0) v += beta * *yp;
                        if (a.gamma != 0.0) v += gamma * Z[row * a.ldz + col];
                        *yp = v;
                        if (a.partials) dot += (double)R[row * a.ldr + col] * (double)v;
                    }
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

template <int MODE, bool TRANS, typename TX>
cudaError_t launch_nt(const ProdArgs &a, cudaStream_t s) {
    const size_t smem = mma_smem_bytes(TRANS, a.warps);
    const int threads = a.warps * 32;
    if (a.k <= 8) mma_product_kernel<MODE, TRANS, TX, 1><<<a.grid, threads, smem, s>>>(a);
    else if (a.k <= 16) mma_product_kernel<MODE, TRANS, TX, 2><<<a.grid, threads, smem, s>>>(a);
    else mma_product_kernel<MODE, TRANS, TX, 4><<<a.grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(bool xdouble, bool trans, const ProdArgs &a, cudaStream_t s) {
    if (xdouble) return trans ? launch_nt<MODE, true, double>(a, s) : launch_nt<MODE, false, double>(a, s);
    return trans ? launch_nt<MODE, true, float>(a, s) : launch_nt<MODE, false, float>(a, s);
}

}  // namespace

size_t mma_smem_bytes(bool trans, int warps) {
    return (size_t)warps * kKMax * (sizeof(int32_t) + (trans ? sizeof(int64_t) : 0));
}

const void *mma_kernel_ptr(int mode, bool xdouble, bool trans) {
#define VBCSR_PTR(M)                                                                                  \
    if (mode == M) {                                                                                  \
        if (xdouble) return trans ? (const void *)mma_product_kernel<M, true, double, 4>              \
                                  : (const void *)mma_product_kernel<M, false, double, 4>;            \
        return trans ? (const void *)mma_product_kernel<M, true, float, 4>                            \
                     : (const void *)mma_product_kernel<M, false, float, 4>;                          \
    }
    VBCSR_PTR(kTF32)
    VBCSR_PTR(kTF32X3)
    VBCSR_PTR(kBF16X2)
#undef VBCSR_PTR
    return nullptr;
}

cudaError_t launch_mma(int mode, bool xdouble, bool trans, const ProdArgs &a, cudaStream_t s) {
    switch (mode) {
        case kTF32: return launch_mode<kTF32>(xdouble, trans, a, s);
        case kTF32X3: return launch_mode<kTF32X3>(xdouble, trans, a, s);
        case kBF16X2: return launch_mode<kBF16X2>(xdouble, trans, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vbcsr
