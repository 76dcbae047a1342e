// Tensor-core block products for the mixed-precision modes (TF32, TF32X3,
// BF16X2) on the FP32 copy of the values, with FP32 accumulation and the
// epilogue (alpha, beta, gamma * Z, dot with R) in the panel dtype. X is read
// as FP32: an FP64 X is converted once per call before the launch.
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
#include "split.cuh"

namespace vbcsr {

namespace {


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
    if (MODE == kBF16X2Presplit) {
        // operands already split into words (hi bf16 low half, lo bf16 high half):
        // pair the halves of columns (c0, c1) and (c2, c3)
        const uint32_t w0 = __float_as_uint(v[0]), w1 = __float_as_uint(v[1]);
        const uint32_t w2 = __float_as_uint(v[2]), w3 = __float_as_uint(v[3]);
        p.bh[0] = __byte_perm(w0, w1, 0x5410);
        p.bh[1] = __byte_perm(w2, w3, 0x5410);
        p.bl[0] = __byte_perm(w0, w1, 0x7632);
        p.bl[1] = __byte_perm(w2, w3, 0x7632);
    } else if (MODE == kBF16X2) {
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
    if (MODE == kBF16X2 || MODE == kBF16X2Presplit) {
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

// The output element as the forward kernel reads X (FP32, or the packed bf16
// pieces of BF16X2), written by the epilogue for the next Chebyshev step.
template <int MODE, typename TX>
__device__ __forceinline__ float xs_form(TX v) {
    if (MODE == kBF16X2Presplit) return __uint_as_float(bf16_pieces((double)v));
    return (float)v;
}

// Resident CTAs (of 4 warps) per SM and the forward kernel's step group U, per
// mode and column-tile count. Measured on GB300 (50k-atom zinc-blende operator,
// one GPU, variants side by side): the pre-split BF16X2 kernel at NT = 4 runs
// 6.6 % faster at 5 CTAs (96 registers, no spills) than at 4, at NT = 1 4 % faster
// at 7 than at 6; TF32X3 at NT = 2 2.4 % faster with U = 2 at 5 CTAs; the
// in-kernel BF16X2 and TF32X3 splits at NT = 4 would spill at 5 CTAs and stay at
// 4. Everything else kept what ran best before: NT = 1 U = 2 at 6 CTAs, NT = 2
// U = 4 at 4 CTAs, NT = 4 U = 2.
template <int MODE, int NT>
struct MmaShape {
    static constexpr int CTAS = NT == 1 ? (MODE == kBF16X2Presplit ? 7 : 6)
                              : NT == 2 ? (MODE == kTF32X3 ? 5 : 4)
                                        : ((MODE == kTF32X3 || MODE == kBF16X2) ? 4 : 5);
    static constexpr int U = NT == 2 && MODE != kTF32X3 ? 4 : 2;
};

template <int MODE, bool TRANS, typename TX, int NT>
__global__ void __launch_bounds__(128, MmaShape<MODE, NT>::CTAS) mma_product_kernel(ProdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw) + warp * kKMax;
    int64_t *s_a = reinterpret_cast<int64_t *>(smem_raw + (size_t)warps * kKMax * sizeof(int32_t)) +
                   warp * kKMax;
    const float *__restrict__ vals = static_cast<const float *>(a.values);
    const float *__restrict__ X = static_cast<const float *>(a.X);   // FP32 (converted before the launch)
    TX *__restrict__ Y = static_cast<TX *>(a.Y);
    const TX *__restrict__ Z = static_cast<const TX *>(a.Z);
    const TX *__restrict__ R = static_cast<const TX *>(a.R);
    float *__restrict__ XS = static_cast<float *>(a.xs_out);
    const EpiScalars<TX> sc = epi_scalars<TX>(a);
    const TX alpha = sc.alpha, beta = sc.beta, gamma = sc.gamma;
    const bool do_prod = a.alpha != 0.0;
    double dot = 0.0;

    // items (in descending cost) come from the device counter a.queue when given,
    // else round-robin
    int64_t it = (int64_t)blockIdx.x * warps + warp;
    for (;;) {
        if (a.queue) {
            unsigned long long q = 0;
            if (lane == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(a.queue), 1ull);
            it = (int64_t)__shfl_sync(0xffffffffu, q, 0);
        }
        if (it >= a.n_items) break;
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
                    if (!TRANS) {
                        // forward: groups of U steps (MmaShape); all value and X loads of a
                        // group are issued before its MMAs, so each warp has U steps of loads
                        // in flight. A window holds kKMax = 512 columns, a multiple of 16 U,
                        // so a group never straddles two windows.
                        constexpr int U = MmaShape<MODE, NT>::U;
                        for (int cg = 0; cg < tn; cg += 16 * U) {
                            float4 qa[U], qb[U];
                            float xv[U][NT][4];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const int64_t col = (int64_t)t0 + cg + 16 * u + 4 * t4;
                                qa[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                                qb[u] = qa[u];
                                if (col < w.Kp) {   // Kp is a multiple of 4: the float4 is inside the row
                                    if (g < w.B)
                                        qa[u] = __ldg(reinterpret_cast<const float4 *>(vals + w.vbase +
                                                                                      (int64_t)g * w.Kp + col));
                                    if (g + 8 < w.B)
                                        qb[u] = __ldg(reinterpret_cast<const float4 *>(
                                            vals + w.vbase + (int64_t)(g + 8) * w.Kp + col));
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const int cl = cg + 16 * u + 4 * t4;
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const int xr = (cl + j < tn) ? s_x[cl + j] : -1;
#pragma unroll
                                    for (int n = 0; n < NT; ++n) {
                                        const int64_t col = n0 + n * 8 + g;
                                        xv[u][n][j] = (xr >= 0 && col < a.k) ? __ldg(X + (int64_t)xr * a.ldx + col)
                                                                             : 0.f;
                                    }
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const float va[4] = {qa[u].x, qa[u].y, qa[u].z, qa[u].w};
                                const float vb[4] = {qb[u].x, qb[u].y, qb[u].z, qb[u].w};
                                Pieces pa, pb;
                                split4<MODE>(va, pa);
                                split4<MODE>(vb, pb);
#pragma unroll
                                for (int n = 0; n < NT; ++n) {
                                    Pieces px;
                                    split4<MODE>(xv[u][n], px);
                                    step<MODE>(acc[n], pa, pb, px);
                                }
                            }
                        }
                        continue;
                    }
                    for (int c16 = 0; c16 < tn; c16 += 16) {
                        const int cl = c16 + 4 * t4;   // first of this lane's 4 columns, window-relative
                        float va[4] = {0.f, 0.f, 0.f, 0.f}, vb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (cl + j < tn) {
                                const float *base = vals + s_a[cl + j];
                                if (g < w.B) va[j] = __ldg(base + g);
                                if (g + 8 < w.B) vb[j] = __ldg(base + g + 8);
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
                                xv[j] = (xr[j] >= 0 && col < a.k) ? __ldg(X + (int64_t)xr[j] * a.ldx + col)
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
                        if (a.beta_nz) v += beta * *yp;
                        if (a.gamma_nz) v += gamma * Z[row * a.ldz + col];
                        *yp = v;
                        if (a.partials || a.item_partials) dot += (double)R[row * a.ldr + col] * (double)v;
                        if (!TRANS && XS) XS[row * a.k + col] = xs_form<MODE, TX>(v);
                    }
                }
            }
        }
        if (a.item_partials) {
            // the item's share of the fused dot at the item's index (summed in a fixed
            // order afterwards, whichever warp took the item)
            for (int m = 16; m > 0; m >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, m);
            if (lane == 0) a.item_partials[it] = dot;
            dot = 0.0;
        }
        if (!a.queue) it += (int64_t)gridDim.x * warps;
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


// ---------------------------------------------------------------------------
// Forward product with the value panel staged in shared memory.
//
// The plain kernel above keeps about one 16-column step of loads in flight per
// warp, which leaves the HBM pipe mostly idle. Here each warp copies its
// item's panel in chunks of kStageCols columns (B row segments of up to
// 512 bytes) into shared memory with bulk asynchronous copies that complete
// on an mbarrier, two buffers deep: while one chunk feeds the tensor cores
// the next chunk (of the same item, the next column pass, or the warp's next
// item) is already on its way. Panel rows start 32-byte aligned and chunk
// widths are multiples of 8 columns, so every copy is a multiple of 16 bytes
// from a 16-byte aligned address. Waits are bounded: on timeout the kernel
// records error code 2 in the handle's error word and the warp stops.

constexpr int kStageCols = 64;
constexpr int kStageLd = kStageCols + 16;      // padded row: rows g and g+1 fall on disjoint bank halves
constexpr int kStageBuf = 16 * kStageLd;       // floats per buffer
constexpr long long kWaitLimit = 1ll << 26;    // try_wait polls before a wait is declared failed

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <int MODE, typename TX, int NT>
__global__ void __launch_bounds__(128, 4) mma_staged_kernel(ProdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    float *bufs = reinterpret_cast<float *>(smem_raw) + (size_t)warp * 2 * kStageBuf;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw + (size_t)warps * 2 * kStageBuf * sizeof(float)) +
                   warp * kKMax;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)warps * 2 * kStageBuf * sizeof(float) +
                                                  (size_t)warps * kKMax * sizeof(int32_t)) +
                     warp * 2;
    const float *__restrict__ vals = static_cast<const float *>(a.values);
    const float *__restrict__ X = static_cast<const float *>(a.X);
    TX *__restrict__ Y = static_cast<TX *>(a.Y);
    const TX *__restrict__ Z = static_cast<const TX *>(a.Z);
    const TX *__restrict__ R = static_cast<const TX *>(a.R);
    const EpiScalars<TX> sc = epi_scalars<TX>(a);
    const TX alpha = sc.alpha, beta = sc.beta, gamma = sc.gamma;
    const bool do_prod = a.alpha != 0.0;
    const int64_t stride = (int64_t)gridDim.x * warps;
    const int64_t npass = (a.k + 8 * NT - 1) / (8 * NT);
    double dot = 0.0;

    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // a stage is (item, column pass, chunk); the warp walks its stages in order
    struct Stage {
        int64_t it, pass;
        int c;
    };
    auto nchunks = [](const WorkItem &w) { return w.Kp > 0 ? (w.Kp + kStageCols - 1) / kStageCols : 1; };
    auto issue = [&](const Stage &st, const WorkItem &w, int b) {
        const int col0 = st.c * kStageCols;
        const int ncol = max(0, min(kStageCols, w.Kp - col0));
        float *dst = bufs + b * kStageBuf;
        if (lane == 0) {
            if (ncol > 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect(&bars[b], (uint32_t)(w.B * ncol * sizeof(float)));
            } else {
                mbar_arrive(&bars[b]);
            }
        }
        __syncwarp();
        if (ncol > 0 && lane < w.B)
            bulk_copy_g2s(dst + lane * kStageLd, vals + w.vbase + (int64_t)lane * w.Kp + col0,
                          (uint32_t)(ncol * sizeof(float)), &bars[b]);
    };

    uint32_t phase[2] = {0u, 0u};
    Stage cur{(int64_t)blockIdx.x * warps + warp, 0, 0};
    if (!do_prod) {
        // alpha == 0: no product, only Y = beta Y (+ gamma Z)
        for (int64_t it = cur.it; it < a.n_items; it += stride) {
            const WorkItem w = a.items[it];
            for (int64_t col = lane; col < (int64_t)w.B * a.k; col += 32) {
                const int64_t row = w.yrow + col / a.k, c = col % a.k;
                TX v = (TX)0;
                if (a.beta_nz) v += beta * Y[row * a.ldy + c];
                if (a.gamma_nz) v += gamma * Z[row * a.ldz + c];
                Y[row * a.ldy + c] = v;
                if (a.partials) dot += (double)R[row * a.ldr + c] * (double)v;
            }
        }
    } else if (cur.it < a.n_items) {
        WorkItem wc = a.items[cur.it];
        int b = 0;
        issue(cur, wc, b);
        float acc[NT][4];
        bool failed = false;
        for (;;) {
            // successor stage
            Stage nx = cur;
            WorkItem wn = wc;
            bool have_next = true;
            if (cur.c + 1 < nchunks(wc)) {
                nx.c = cur.c + 1;
            } else if (cur.pass + 1 < npass) {
                nx.pass = cur.pass + 1;
                nx.c = 0;
            } else {
                nx.it = cur.it + stride;
                nx.pass = 0;
                nx.c = 0;
                have_next = nx.it < a.n_items;
                if (have_next) wn = a.items[nx.it];
            }
            if (have_next) issue(nx, wn, b ^ 1);

            // consume the current stage
            const int col0 = cur.c * kStageCols;
            const int ncol = max(0, min(kStageCols, wc.Kp - col0));
            const int64_t n0 = cur.pass * 8 * NT;
            if (cur.c == 0) {
#pragma unroll
                for (int n = 0; n < NT; ++n)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[n][j] = 0.f;
            }
            // X rows of this chunk's columns: staged per kKMax window
            const int win0 = (col0 / kKMax) * kKMax;
            const int wn_cols = min(kKMax, wc.K - win0);
            if (col0 % kKMax == 0 && wn_cols > 0) {
                __syncwarp();
                for (int e = lane; e < wc.nlist; e += 32) {
                    const int64_t l = wc.lbegin + e;
                    const int xr = a.fl.xrow[l], pc = a.fl.pcol[l], wd = a.fl.w[l];
                    const int lo = max(pc, win0), hi = min(pc + wd, win0 + wn_cols);
                    for (int t = lo; t < hi; ++t) s_x[t - win0] = xr + (t - pc);
                }
                __syncwarp();
            }
            if (!mbar_wait(&bars[b], phase[b])) {
                failed = true;
                break;
            }
            phase[b] ^= 1u;
            const float *buf = bufs + b * kStageBuf;
            // X values of a 16-column step: lane holds columns 4t..4t+3 of the step for
            // output columns n0 + 8n + g; the next step's are loaded before this step's MMAs
            auto load_x = [&](int c16, float (&xv)[NT][4]) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int cl = c16 + 4 * t4 + j;
                    const int t = col0 + cl;
                    const int xr = (cl < ncol && t < wc.K) ? s_x[t - win0] : -1;
#pragma unroll
                    for (int n = 0; n < NT; ++n) {
                        const int64_t col = n0 + n * 8 + g;
                        xv[n][j] = (xr >= 0 && col < a.k) ? __ldg(X + (int64_t)xr * a.ldx + col) : 0.f;
                    }
                }
            };
            float xnext[NT][4];
            if (ncol > 0) load_x(0, xnext);
            for (int c16 = 0; c16 < ncol; c16 += 16) {
                float xcur[NT][4];
#pragma unroll
                for (int n = 0; n < NT; ++n)
#pragma unroll
                    for (int j = 0; j < 4; ++j) xcur[n][j] = xnext[n][j];
                if (c16 + 16 < ncol) load_x(c16 + 16, xnext);
                const int cl = c16 + 4 * t4;                 // chunk-relative first column of this lane
                float va[4] = {0.f, 0.f, 0.f, 0.f}, vb[4] = {0.f, 0.f, 0.f, 0.f};
                if (cl < ncol) {                              // ncol is a multiple of 4: all four are inside
                    if (g < wc.B) {
                        const float4 q = *reinterpret_cast<const float4 *>(buf + g * kStageLd + cl);
                        va[0] = q.x; va[1] = q.y; va[2] = q.z; va[3] = q.w;
                    }
                    if (g + 8 < wc.B) {
                        const float4 q = *reinterpret_cast<const float4 *>(buf + (g + 8) * kStageLd + cl);
                        vb[0] = q.x; vb[1] = q.y; vb[2] = q.z; vb[3] = q.w;
                    }
                }
                Pieces pa, pb;
                split4<MODE>(va, pa);
                split4<MODE>(vb, pb);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    Pieces px;
                    split4<MODE>(xcur[n], px);
                    step<MODE>(acc[n], pa, pb, px);
                }
            }
            __syncwarp();   // every lane is done with buffer b before it is refilled

            if (cur.c + 1 == nchunks(wc)) {
                // epilogue of (item, pass): acc[n] = {(g,2t),(g,2t+1),(g+8,2t),(g+8,2t+1)} of tile n
#pragma unroll
                for (int n = 0; n < NT; ++n) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int r = g + ((j >> 1) << 3);
                        const int64_t col = n0 + n * 8 + 2 * t4 + (j & 1);
                        if (r < wc.B && col < a.k) {
                            const int64_t row = wc.yrow + r;
                            TX *yp = Y + row * a.ldy + col;
                            TX v = alpha * (TX)acc[n][j];
                            if (a.beta_nz) v += beta * *yp;
                            if (a.gamma_nz) v += gamma * Z[row * a.ldz + col];
                            *yp = v;
                            if (a.partials) dot += (double)R[row * a.ldr + col] * (double)v;
                        }
                    }
                }
            }
            if (!have_next) break;
            cur = nx;
            wc = wn;
            b ^= 1;
        }
        if (failed) {
            if (lane == 0) atomicExch(a.err, 2);
            // let copies already issued into either buffer land before the CTA exits
            mbar_wait(&bars[0], phase[0]);
            mbar_wait(&bars[1], phase[1]);
        }
    }

    if (a.partials) {
        for (int m = 16; m > 0; m >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, m);
        __shared__ double s_dot[32];
        __syncthreads();
        if (lane == 0) s_dot[warp] = dot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int i = 0; i < warps; ++i) sum += s_dot[i];
            a.partials[blockIdx.x] = sum;
        }
    }
}

size_t staged_smem_bytes(int warps) {
    return (size_t)warps * (2 * kStageBuf * sizeof(float) + kKMax * sizeof(int32_t) + 2 * sizeof(uint64_t));
}

template <typename K>
cudaError_t staged_launch(K kernel, const ProdArgs &a, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<a.grid, a.warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MODE, bool TRANS, typename TX>
cudaError_t launch_nt(const ProdArgs &a, cudaStream_t s) {
    if (!TRANS && a.mma_staged) {
        const size_t smem = staged_smem_bytes(a.warps);
        if (a.k <= 8) return staged_launch(mma_staged_kernel<MODE, TX, 1>, a, smem, s);
        if (a.k <= 16) return staged_launch(mma_staged_kernel<MODE, TX, 2>, a, smem, s);
        return staged_launch(mma_staged_kernel<MODE, TX, 4>, a, smem, s);
    }
    const size_t smem = mma_smem_bytes(TRANS, false, a.warps);
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

size_t mma_smem_bytes(bool trans, bool staged, int warps) {
    if (!trans && staged) return staged_smem_bytes(warps);
    return (size_t)warps * kKMax * (sizeof(int32_t) + (trans ? sizeof(int64_t) : 0));
}

// The kernel a launch of (mode, X/Y type, direction, variant, k) runs; used to size its grid.
const void *mma_kernel_ptr(int mode, bool xdouble, bool trans, bool staged, int64_t k) {
    const int nt = k <= 8 ? 1 : (k <= 16 ? 2 : 4);
#define VBCSR_PTR_NT(M, TX, NT)                                                                   \
    if (nt == NT) {                                                                               \
        if (trans) return (const void *)mma_product_kernel<M, true, TX, NT>;                      \
        if (staged) return (const void *)mma_staged_kernel<M, TX, NT>;                            \
        return (const void *)mma_product_kernel<M, false, TX, NT>;                                \
    }
#define VBCSR_PTR(M)                                                                              \
    if (mode == M) {                                                                              \
        if (xdouble) {                                                                            \
            VBCSR_PTR_NT(M, double, 1) VBCSR_PTR_NT(M, double, 2) VBCSR_PTR_NT(M, double, 4)      \
        } else {                                                                                  \
            VBCSR_PTR_NT(M, float, 1) VBCSR_PTR_NT(M, float, 2) VBCSR_PTR_NT(M, float, 4)         \
        }                                                                                         \
    }
    VBCSR_PTR(kTF32)
    VBCSR_PTR(kTF32X3)
    VBCSR_PTR(kBF16X2)
#undef VBCSR_PTR
#undef VBCSR_PTR_NT
    if (mode == kBF16X2Presplit && xdouble && !trans && !staged) {
        if (nt == 1) return (const void *)mma_product_kernel<kBF16X2Presplit, false, double, 1>;
        if (nt == 2) return (const void *)mma_product_kernel<kBF16X2Presplit, false, double, 2>;
        return (const void *)mma_product_kernel<kBF16X2Presplit, false, double, 4>;
    }
    return nullptr;
}

cudaError_t launch_mma(int mode, bool xdouble, bool trans, const ProdArgs &a, cudaStream_t s) {
    switch (mode) {
        case kTF32: return launch_mode<kTF32>(xdouble, trans, a, s);
        case kTF32X3: return launch_mode<kTF32X3>(xdouble, trans, a, s);
        case kBF16X2: return launch_mode<kBF16X2>(xdouble, trans, a, s);
        case kBF16X2Presplit:
            // forward, plain kernel, FP64 X / Y only (the split copies belong to FP64 operators)
            if (!xdouble || trans || a.mma_staged) return cudaErrorInvalidValue;
            return launch_nt<kBF16X2Presplit, false, double>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vbcsr
