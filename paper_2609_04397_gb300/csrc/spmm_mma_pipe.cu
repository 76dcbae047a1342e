// BF16X2 forward product of an FP64 operator on the tensor cores, pipelined
// through shared memory (the default forward kernel of the BF16X2 mode for
// k >= 3).
//
// Operands are split once into bf16 pieces v = hi + lo (hi = bf16_rn(v),
// lo = bf16_rn(v - hi), v rounded to FP32 first) and kept as two planes of
// the same shape: the values as planes of the value pages (panel layout), X
// as planes [rows, ldp] with ldp a multiple of the pass width. Products
// hi*hi + hi*lo + lo*hi accumulate in FP32 (m16n8k16, FP32 accumulators);
// the epilogue (alpha, beta, gamma * Z, the dot with R) is FP64.
//
// One warp owns one work item (up to 16 output rows of a block row) and
// walks its virtual columns in steps of 16. Each step's operands, 16 rows x
// 16 columns of both value planes and the 16 gathered X rows x 8 NT columns
// of both X planes, are copied into a ring of S shared-memory stages by
// asynchronous 16-byte copies, S - 1 steps ahead of the tensor cores. The
// copies of columns beyond the panel row or beyond the item's last virtual
// column are zero-filled, so the tail steps add nothing; value rows >= B are
// not copied (whatever the stage holds there reaches only output rows that
// are not written). Fragments come from the stages with ldmatrix (the
// transposing form for the X tile, whose 16 rows are virtual columns); the
// 16-byte chunks of a stage row are XOR-swizzled by the row so that the eight
// rows of each ldmatrix matrix fall on distinct banks.
//
// The loads in flight per warp are the ring's, not registers, and the bf16
// planes feed the MMA fragments directly (no byte permutes).
#include <cuda_bf16.h>

#include "internal.cuh"
#include "split.cuh"

namespace vbcsr {

namespace {

constexpr int kPipeStages = 4;   // ring depth (stages of 16 virtual columns)

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// 16 bytes global -> shared, asynchronously; zero-filled when !valid (src is then not read)
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t (&r)[2]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(addr));
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage layout (bytes), per warp and stage: value plane hi, value plane lo
// (16 rows x 32 B each), X plane hi, X plane lo (16 rows x 16 NT B each).
template <int NT>
struct PipeStage {
    static constexpr int kVPlane = 16 * 32;
    static constexpr int kXRow = 16 * NT;
    static constexpr int kXPlane = 16 * kXRow;
    static constexpr int kBytes = 2 * kVPlane + 2 * kXPlane;
};

// byte offset of 16-byte chunk c of row r in a value plane (two chunks per row)
__device__ __forceinline__ int v_off(int r, int c) { return r * 32 + 16 * (c ^ ((r >> 2) & 1)); }

// byte offset of chunk c of row r in an X plane (NT chunks per row)
template <int NT>
__device__ __forceinline__ int x_off(int r, int c) {
    const int sw = NT == 4 ? ((r >> 1) & 3) : NT == 2 ? ((r >> 2) & 1) : 0;
    return r * (16 * NT) + 16 * (c ^ sw);
}

// packed bf16 hi / lo pieces of two FP64 values (lower column in the low half)
__device__ __forceinline__ void pieces2(double v0, double v1, uint32_t &hi, uint32_t &lo) {
    const uint32_t w0 = bf16_pieces(v0), w1 = bf16_pieces(v1);
    hi = (w0 & 0xffffu) | (w1 << 16);
    lo = (w0 >> 16) | (w1 & 0xffff0000u);
}

template <int NT>
__global__ void __launch_bounds__(128, 4) mma_bf16_pipe_kernel(ProdArgs a) {
    constexpr int S = kPipeStages;
    using St = PipeStage<NT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    unsigned char *ring = smem_raw + (size_t)warp * S * St::kBytes;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw + (size_t)warps * S * St::kBytes) + warp * kKMax;
    const uint32_t ring_s = smem_addr(ring);

    const __nv_bfloat16 *__restrict__ vhi = static_cast<const __nv_bfloat16 *>(a.values);
    const __nv_bfloat16 *__restrict__ xhi = static_cast<const __nv_bfloat16 *>(a.X);
    double *__restrict__ Y = static_cast<double *>(a.Y);
    const double *__restrict__ Z = static_cast<const double *>(a.Z);
    const double *__restrict__ R = static_cast<const double *>(a.R);
    uint32_t *__restrict__ XS = static_cast<uint32_t *>(a.xs_out);   // hi plane; lo plane at + a.xs_plane / 2
    const int64_t ldp = a.ldx;
    const bool do_prod = a.alpha != 0.0;
    const bool want_dot = a.partials || a.item_partials;
    double dot = 0.0;

    // this lane's value copies: chunk (row vr, half vh) of both planes
    const int vr = (lane >> 1) & 15, vh = lane & 1;
    const uint32_t v_dst = (uint32_t)v_off(vr, vh);
    // X offsets in 32-bit arithmetic when the planes are small enough (64-bit
    // integer arithmetic is slow on this chip); row indices are staged as int32
    const bool x32 = (uint64_t)a.x_plane < (1ull << 31);

    int64_t it = (int64_t)blockIdx.x * warps + warp;
    for (;;) {
        if (a.queue) {
            unsigned long long q = 0;
            if (lane == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(a.queue), 1ull);
            it = (int64_t)__shfl_sync(0xffffffffu, q, 0);
        }
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        // this lane's value row of the item in the hi plane (the lo plane is v_plane further)
        const __nv_bfloat16 *vrow = vhi + (w.vbase + (int64_t)min(vr, w.B - 1) * w.Kp);
        for (int64_t n0 = 0; n0 < a.k; n0 += 8 * NT) {
            float acc[NT][4];
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[n][j] = 0.f;

            if (do_prod) {
                for (int t0 = 0; t0 < w.K; t0 += kKMax) {
                    const int tn = min(kKMax, w.K - t0);
                    const int nsteps = (tn + 15) >> 4;
                    if (n0 == 0 || w.K > kKMax) {
                        __syncwarp();
                        for (int e = lane; e < w.nlist; e += 32) {
                            const int64_t l = w.lbegin + e;
                            const int xr = a.fl.xrow[l], pc = a.fl.pcol[l], wd = a.fl.w[l];
                            const int lo = max(pc, t0), hi = min(pc + wd, t0 + tn);
                            for (int t = lo; t < hi; ++t) s_x[t - t0] = xr + (t - pc);
                        }
                        __syncwarp();
                    }
                    // copies of step s into ring slot s % S (an empty group past the last step)
                    auto issue = [&](int s) {
                        if (s < nsteps) {
                            const uint32_t st = ring_s + (uint32_t)((s % S) * St::kBytes);
                            if (vr < w.B) {
                                const int col = t0 + 16 * s + 8 * vh;
                                const bool ok = col < w.Kp;   // Kp is a multiple of 8: a chunk is in or out
                                const __nv_bfloat16 *src = vrow + (ok ? col : 0);
                                cp16(st + v_dst, src, ok);
                                cp16(st + St::kVPlane + v_dst, src + a.v_plane, ok);
                            }
                            // the X tile: 16 rows x NT chunks per plane; lane handles (row, chunk)
                            // pairs lane, lane + 32, ... below 16 NT, in both planes
                            for (int idx = lane; idx < 16 * NT; idx += 32) {
                                const int v = idx / NT, c = idx % NT;
                                const int t = 16 * s + v;
                                const bool ok = t < tn;
                                const int xr = ok ? s_x[t] : 0;
                                const __nv_bfloat16 *src =
                                    x32 ? xhi + ((uint32_t)xr * (uint32_t)ldp + (uint32_t)n0 + 8u * c)
                                        : xhi + ((int64_t)xr * ldp + n0 + 8 * c);
                                cp16(st + 2 * St::kVPlane + x_off<NT>(v, c), src, ok);
                                cp16(st + 2 * St::kVPlane + St::kXPlane + x_off<NT>(v, c), src + a.x_plane, ok);
                            }
                        }
                        cp_commit();
                    };
#pragma unroll
                    for (int s = 0; s < S - 1; ++s) issue(s);
                    for (int s = 0; s < nsteps; ++s) {
                        cp_wait<S - 2>();
                        __syncwarp();
                        const uint32_t st = ring_s + (uint32_t)((s % S) * St::kBytes);
                        // A fragments: matrices (rows 0-7 | 8-15) x (columns 0-7 | 8-15)
                        const int am = lane >> 3, ar = (lane & 7) + 8 * (am & 1), ac = am >> 1;
                        uint32_t ahi[4], alo[4];
                        ldsm_x4(st + v_off(ar, ac), ahi);
                        ldsm_x4(st + St::kVPlane + v_off(ar, ac), alo);
                        // B fragments: the X tile's rows are the step's virtual columns
                        const uint32_t xs0 = st + 2 * St::kVPlane;
                        if constexpr (NT == 1) {
                            const int br = lane & 15;
                            uint32_t bh[2], bl[2];
                            ldsm_x2_t(xs0 + x_off<NT>(br, 0), bh);
                            ldsm_x2_t(xs0 + St::kXPlane + x_off<NT>(br, 0), bl);
                            mma16816(acc[0], ahi, bh[0], bh[1]);
                            mma16816(acc[0], ahi, bl[0], bl[1]);
                            mma16816(acc[0], alo, bh[0], bh[1]);
                        } else {
#pragma unroll
                            for (int n = 0; n < NT; n += 2) {
                                const int bm = lane >> 3, br = (lane & 7) + 8 * (bm & 1), bc = n + (bm >> 1);
                                uint32_t bh[4], bl[4];
                                ldsm_x4_t(xs0 + x_off<NT>(br, bc), bh);
                                ldsm_x4_t(xs0 + St::kXPlane + x_off<NT>(br, bc), bl);
                                mma16816(acc[n], ahi, bh[0], bh[1]);
                                mma16816(acc[n], ahi, bl[0], bl[1]);
                                mma16816(acc[n], alo, bh[0], bh[1]);
                                mma16816(acc[n + 1], ahi, bh[2], bh[3]);
                                mma16816(acc[n + 1], ahi, bl[2], bl[3]);
                                mma16816(acc[n + 1], alo, bh[2], bh[3]);
                            }
                        }
                        issue(s + S - 1);
                    }
                    cp_wait_all();
                    __syncwarp();
                }
            }
            // epilogue: acc[n] = {(g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)} of tile n
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                if (r >= w.B) continue;
                const int64_t row = w.yrow + r;
                double *yrow = Y + row * a.ldy + n0;
                const double *zrow = Z + row * a.ldz + n0;
                const double *rrow = R + row * a.ldr + n0;
                uint32_t *xsrow = XS + ((row * ldp + n0) >> 1);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const int cl = n * 8 + 2 * t4;   // column relative to n0
                    if (n0 + cl >= a.k) continue;
                    const bool pair = n0 + cl + 1 < a.k;
                    double v[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (e == 1 && !pair) break;
                        double o = a.alpha * (double)acc[n][2 * h + e];
                        if (a.beta != 0.0) o += a.beta * yrow[cl + e];
                        if (a.gamma != 0.0) o += a.gamma * zrow[cl + e];
                        yrow[cl + e] = o;
                        if (want_dot) dot += rrow[cl + e] * o;
                        v[e] = o;
                    }
                    if (XS) {
                        uint32_t hi, lo;
                        pieces2(v[0], pair ? v[1] : 0.0, hi, lo);
                        // the column is even and the plane stride ldp even: a 4-byte aligned pair
                        xsrow[cl >> 1] = hi;
                        xsrow[(cl >> 1) + (a.xs_plane >> 1)] = lo;
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
            double sum = 0.0;
            for (int i = 0; i < warps; ++i) sum += s_dot[i];
            a.partials[blockIdx.x] = sum;
        }
    }
}

template <int NT>
size_t pipe_smem(int warps) {
    return (size_t)warps * ((size_t)kPipeStages * PipeStage<NT>::kBytes + kKMax * sizeof(int32_t));
}

template <int NT>
cudaError_t pipe_launch(const ProdArgs &a, cudaStream_t s) {
    const size_t smem = pipe_smem<NT>(a.warps);
    cudaError_t e = cudaFuncSetAttribute((const void *)mma_bf16_pipe_kernel<NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mma_bf16_pipe_kernel<NT><<<a.grid, a.warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// TF32 / TF32X3 forward product of an FP64 operator pipelined the same way:
// the FP32 copy of the values and X as FP32 rows of ldp elements stream
// through the per-warp ring (16 virtual columns per stage). The value tile
// is read by ldmatrix (a 16 x 8 FP32 tile viewed as four 8 x 8 b16 matrices
// lands in exactly the m16n8k8 TF32 A-fragment layout), the X tile by 32-bit
// shared loads; each operand is cut into tf32 pieces in registers (hi =
// rna(v), lo = rna(v - hi)), and TF32 multiplies hi*hi, TF32X3 adds hi*lo +
// lo*hi, all accumulated in FP32 (m16n8k8); the epilogue is FP64 and writes
// the output also as FP32 rows of ldp elements when the next product of a
// recurrence reads it.

template <int NT>
struct TfStage {
    static constexpr int kV = 16 * 64;         // values: 16 rows x 16 FP32
    static constexpr int kXRow = 32 * NT;      // X: 16 rows x 8 NT FP32
    static constexpr int kBytes = kV + 16 * kXRow;
};

// byte offset of 16-byte chunk c (4 FP32) of value row r: XOR-swizzled so that
// the eight rows of each ldmatrix matrix fall on distinct banks
__device__ __forceinline__ int tv_off(int r, int c) { return r * 64 + 16 * (c ^ ((r >> 1) & 3)); }

// physical chunk of chunk c of X row r: swizzled so that the four rows t, or
// t + 4, of one B-fragment load fall on distinct banks
template <int NT>
__device__ __forceinline__ int tx_chunk(int r, int c) {
    return NT == 4 ? (c ^ (2 * (r & 3))) : NT == 2 ? (c ^ (2 * ((r >> 1) & 1))) : c;
}

__device__ __forceinline__ uint32_t tf32_bits(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ void mma1688(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int NT, int MODE>
__global__ void __launch_bounds__(128, 4) mma_tf32_pipe_kernel(ProdArgs a) {
    constexpr int S = kPipeStages;
    using St = TfStage<NT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    unsigned char *ring = smem_raw + (size_t)warp * S * St::kBytes;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw + (size_t)warps * S * St::kBytes) + warp * kKMax;
    const uint32_t ring_s = smem_addr(ring);

    const float *__restrict__ vals = static_cast<const float *>(a.values);
    const float *__restrict__ X = static_cast<const float *>(a.X);
    double *__restrict__ Y = static_cast<double *>(a.Y);
    const double *__restrict__ Z = static_cast<const double *>(a.Z);
    const double *__restrict__ R = static_cast<const double *>(a.R);
    float *__restrict__ XS = static_cast<float *>(a.xs_out);   // [rows, ldp], or NULL
    const int64_t ldp = a.ldx;
    const bool do_prod = a.alpha != 0.0;
    const bool want_dot = a.partials || a.item_partials;
    double dot = 0.0;

    // this lane's value copies: row vr, chunks vc, vc + 1 (columns 8 (lane & 1) .. + 7)
    const int vr = lane >> 1, vc = 2 * (lane & 1);
    const bool x32 = (uint64_t)a.x_rows * (uint64_t)ldp < (1ull << 31);
    // A fragments: lane supplies row ar of matrix lane / 8 (chunk ac of a substep)
    const int ar = ((lane >> 3) & 1) * 8 + (lane & 7), ac = lane >> 4;

    int64_t it = (int64_t)blockIdx.x * warps + warp;
    for (;;) {
        if (a.queue) {
            unsigned long long q = 0;
            if (lane == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(a.queue), 1ull);
            it = (int64_t)__shfl_sync(0xffffffffu, q, 0);
        }
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        const float *vrow = vals + (w.vbase + (int64_t)min(vr, w.B - 1) * w.Kp);
        for (int64_t n0 = 0; n0 < a.k; n0 += 8 * NT) {
            float acc[NT][4];
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[n][j] = 0.f;

            if (do_prod) {
                for (int t0 = 0; t0 < w.K; t0 += kKMax) {
                    const int tn = min(kKMax, w.K - t0);
                    const int nsteps = (tn + 15) >> 4;
                    if (n0 == 0 || w.K > kKMax) {
                        __syncwarp();
                        for (int e = lane; e < w.nlist; e += 32) {
                            const int64_t l = w.lbegin + e;
                            const int xr = a.fl.xrow[l], pc = a.fl.pcol[l], wd = a.fl.w[l];
                            const int lo = max(pc, t0), hi = min(pc + wd, t0 + tn);
                            for (int t = lo; t < hi; ++t) s_x[t - t0] = xr + (t - pc);
                        }
                        __syncwarp();
                    }
                    auto issue = [&](int s) {
                        if (s < nsteps) {
                            const uint32_t st = ring_s + (uint32_t)((s % S) * St::kBytes);
                            if (vr < w.B) {
#pragma unroll
                                for (int c = vc; c < vc + 2; ++c) {
                                    const int col = t0 + 16 * s + 4 * c;
                                    const bool ok = col < w.Kp;   // Kp is a multiple of 8
                                    cp16(st + tv_off(vr, c), vrow + (ok ? col : 0), ok);
                                }
                            }
                            // the X tile: 16 rows x 2 NT chunks; lane takes (row, chunk) pairs
                            // lane, lane + 32, ... below 32 NT
#pragma unroll
                            for (int i = 0; i < NT; ++i) {
                                const int idx = lane + 32 * i;
                                const int v = idx / (2 * NT), c = idx % (2 * NT);
                                const int t = 16 * s + v;
                                const bool ok = t < tn;
                                const int xr = ok ? s_x[t] : 0;
                                const float *src = x32 ? X + ((uint32_t)xr * (uint32_t)ldp + (uint32_t)n0 + 4u * c)
                                                       : X + ((int64_t)xr * ldp + n0 + 4 * c);
                                cp16(st + St::kV + v * St::kXRow + 16 * tx_chunk<NT>(v, c), src, ok);
                            }
                        }
                        cp_commit();
                    };
#pragma unroll
                    for (int s = 0; s < S - 1; ++s) issue(s);
                    for (int s = 0; s < nsteps; ++s) {
                        cp_wait<S - 2>();
                        __syncwarp();
                        issue(s + S - 1);
                        const uint32_t st = ring_s + (uint32_t)((s % S) * St::kBytes);
                        const unsigned char *stp = ring + (s % S) * St::kBytes;
#pragma unroll
                        for (int j = 0; j < 2; ++j) {   // two k8 substeps per stage
                            uint32_t av[4], ahi[4], alo[4];
                            ldsm_x4(st + tv_off(ar, 2 * j + ac), av);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                ahi[q] = tf32_bits(__uint_as_float(av[q]));
                                if (MODE == kTF32X3)
                                    alo[q] = tf32_bits(__uint_as_float(av[q]) - __uint_as_float(ahi[q]));
                            }
                            const int r0 = 8 * j + t4, r1 = r0 + 4;
#pragma unroll
                            for (int n = 0; n < NT; ++n) {
                                const int col = 8 * n + g;
                                const float b0 = *reinterpret_cast<const float *>(
                                    stp + St::kV + r0 * St::kXRow + 16 * tx_chunk<NT>(r0, col >> 2) + 4 * (col & 3));
                                const float b1 = *reinterpret_cast<const float *>(
                                    stp + St::kV + r1 * St::kXRow + 16 * tx_chunk<NT>(r1, col >> 2) + 4 * (col & 3));
                                const uint32_t bh0 = tf32_bits(b0), bh1 = tf32_bits(b1);
                                mma1688(acc[n], ahi, bh0, bh1);
                                if (MODE == kTF32X3) {
                                    const uint32_t bl0 = tf32_bits(b0 - __uint_as_float(bh0));
                                    const uint32_t bl1 = tf32_bits(b1 - __uint_as_float(bh1));
                                    mma1688(acc[n], ahi, bl0, bl1);
                                    mma1688(acc[n], alo, bh0, bh1);
                                }
                            }
                        }
                    }
                    cp_wait_all();
                    __syncwarp();
                }
            }
            // epilogue: acc[n] = {(g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)} of tile n
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g + 8 * h;
                if (r >= w.B) continue;
                const int64_t row = w.yrow + r;
                double *yrow = Y + row * a.ldy + n0;
                const double *zrow = Z + row * a.ldz + n0;
                const double *rrow = R + row * a.ldr + n0;
                float *xsrow = XS + (row * ldp + n0);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const int cl = n * 8 + 2 * t4;   // column relative to n0
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (n0 + cl + e >= a.k) break;
                        double o = a.alpha * (double)acc[n][2 * h + e];
                        if (a.beta != 0.0) o += a.beta * yrow[cl + e];
                        if (a.gamma != 0.0) o += a.gamma * zrow[cl + e];
                        yrow[cl + e] = o;
                        if (want_dot) dot += rrow[cl + e] * o;
                        if (XS) xsrow[cl + e] = (float)o;
                    }
                }
            }
        }
        if (a.item_partials) {
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
            double sum = 0.0;
            for (int i = 0; i < warps; ++i) sum += s_dot[i];
            a.partials[blockIdx.x] = sum;
        }
    }
}

template <int NT>
size_t tf_smem(int warps) {
    return (size_t)warps * ((size_t)kPipeStages * TfStage<NT>::kBytes + kKMax * sizeof(int32_t));
}

template <int NT, int MODE>
cudaError_t tf_launch(const ProdArgs &a, cudaStream_t s) {
    const size_t smem = tf_smem<NT>(a.warps);
    cudaError_t e = cudaFuncSetAttribute((const void *)mma_tf32_pipe_kernel<NT, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mma_tf32_pipe_kernel<NT, MODE><<<a.grid, a.warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32-value forward product on the CUDA cores, pipelined the same way: FP32
// values (an FP32 operator, or the FP32 copy of an FP64 operator in the F32
// mode) and the gathered FP32 X tile stream through a ring of shared-memory
// stages of 16 virtual columns; each lane accumulates a register tile of 4
// rows x CPL output columns in FP32 from the stage (per 4 virtual columns:
// four 16-byte loads of values, four of X, 16 CPL multiply-adds). Lanes: rg =
// lane & 3 picks rows rg, rg + 4, rg + 8, rg + 12, cg the column group; for
// 8-column passes (NT = 1) the two halves of the lanes (vg) take alternate
// chunks of 4 virtual columns of each stage and are added at the end of the
// item. Value rows >= B are not copied (their outputs are not written);
// columns past the row or past the item's last virtual column are
// zero-filled. Value stage rows are 64 bytes with chunk c of row r at chunk
// c ^ (2 ((r >> 1) & 1)), so the rows 4i .. 4i + 3 that one load reads (and
// the two chunks the lane halves read) fall on distinct banks; X rows of an
// 8-column pass are padded to 48 bytes for the same reason.

template <int NT>
struct F32Pipe {
    static constexpr int CPL = NT == 4 ? 4 : 2;           // output columns per lane
    static constexpr int PW = 8 * NT;                     // output columns per pass
    static constexpr int CG = PW / CPL;                   // column groups
    static constexpr int V = 32 / (4 * CG);               // virtual-column groups (1 or 2)
    static constexpr int kVBytes = 16 * 64;               // values: 16 rows x 16 columns x 4 B
    static constexpr int kXRow = NT == 1 ? 48 : PW * 4;   // X row stride (bytes)
    static constexpr int kXBytes = 16 * kXRow;            // X: 16 rows x PW columns
    static constexpr int kBytes = kVBytes + kXBytes;
    static constexpr int S = NT == 4 ? 3 : NT == 1 ? 5 : 4;   // ring depth: as deep as 5 CTAs per SM allow
};

__device__ __forceinline__ int f_off(int r, int c) { return r * 64 + 16 * (c ^ (2 * ((r >> 1) & 1))); }

// One stage of the FP32 pipelined kernel: NI row groups (rows rg + 4 i, i < NI)
// of this lane's tile, from the stage at st.
template <int NT, int NI>
__device__ __forceinline__ void f32_stage(const unsigned char *st, int rg, int cg, int vg,
                                          float (&acc)[4][F32Pipe<NT>::CPL]) {
    using P = F32Pipe<NT>;
#pragma unroll
    for (int q = 0; q < 4 / P::V; ++q) {   // this lane's chunks of 4 virtual columns
        const int c = P::V == 2 ? 2 * q + vg : q;
        float4 vv[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) vv[i] = *reinterpret_cast<const float4 *>(st + f_off(rg + 4 * i, c));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned char *xp = st + P::kVBytes + (4 * c + u) * P::kXRow + 4 * cg * P::CPL;
            float xv[P::CPL];
            if constexpr (P::CPL == 4) {
                const float4 x4 = *reinterpret_cast<const float4 *>(xp);
                xv[0] = x4.x;
                xv[1] = x4.y;
                xv[2] = x4.z;
                xv[3] = x4.w;
            } else {
                const float2 x2 = *reinterpret_cast<const float2 *>(xp);
                xv[0] = x2.x;
                xv[1] = x2.y;
            }
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                const float vi = u == 0 ? vv[i].x : u == 1 ? vv[i].y : u == 2 ? vv[i].z : vv[i].w;
#pragma unroll
                for (int j = 0; j < P::CPL; ++j) acc[i][j] = fmaf(vi, xv[j], acc[i][j]);
            }
        }
    }
}

template <int NT, typename TX>
__global__ void __launch_bounds__(128, NT <= 2 ? 5 : 4) fma32_pipe_kernel(ProdArgs a) {
    constexpr int S = F32Pipe<NT>::S;
    using P = F32Pipe<NT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    unsigned char *ring = smem_raw + (size_t)warp * S * P::kBytes;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw + (size_t)warps * S * P::kBytes) + warp * kKMax;
    const uint32_t ring_s = smem_addr(ring);
    const float *__restrict__ vals = static_cast<const float *>(a.values);
    const float *__restrict__ X = static_cast<const float *>(a.X);
    TX *__restrict__ Y = static_cast<TX *>(a.Y);
    const TX *__restrict__ Z = static_cast<const TX *>(a.Z);
    const TX *__restrict__ R = static_cast<const TX *>(a.R);
    const int64_t ldx = a.ldx;
    const bool do_prod = a.alpha != 0.0;
    const bool want_dot = a.partials || a.item_partials;
    const EpiScalars<TX> sc = epi_scalars<TX>(a);
    double dot = 0.0;
    const int rg = lane & 3, cg = (lane >> 2) % P::CG, vg = lane / (4 * P::CG);
    // this lane's copies: value chunk (row vrow_, chunk vc_) x 2; X chunks below
    const int vrow_ = lane >> 1, vc0 = 2 * (lane & 1);   // rows 0..15, chunks {0,1} or {2,3}

    int64_t it = (int64_t)blockIdx.x * warps + warp;
    for (;;) {
        if (a.queue) {
            unsigned long long q = 0;
            if (lane == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(a.queue), 1ull);
            it = (int64_t)__shfl_sync(0xffffffffu, q, 0);
        }
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        const float *vrowp = vals + (w.vbase + (int64_t)min(vrow_, w.B - 1) * w.Kp);
        for (int64_t n0 = 0; n0 < a.k; n0 += P::PW) {
            float acc[4][P::CPL];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < P::CPL; ++j) acc[i][j] = 0.f;
            if (do_prod) {
                for (int t0 = 0; t0 < w.K; t0 += kKMax) {
                    const int tn = min(kKMax, w.K - t0);
                    const int nsteps = (tn + 15) >> 4;
                    if (n0 == 0 || w.K > kKMax) {
                        __syncwarp();
                        for (int e = lane; e < w.nlist; e += 32) {
                            const int64_t l = w.lbegin + e;
                            const int xr = a.fl.xrow[l], pc = a.fl.pcol[l], wd = a.fl.w[l];
                            const int lo = max(pc, t0), hi = min(pc + wd, t0 + tn);
                            for (int t = lo; t < hi; ++t) s_x[t - t0] = xr + (t - pc);
                        }
                        __syncwarp();
                    }
                    auto issue = [&](int s) {
                        if (s < nsteps) {
                            const uint32_t st = ring_s + (uint32_t)((s % S) * P::kBytes);
                            if (vrow_ < w.B) {
#pragma unroll
                                for (int c = vc0; c < vc0 + 2; ++c) {
                                    const int col = t0 + 16 * s + 4 * c;
                                    const bool ok = col < w.Kp;   // Kp is a multiple of 4
                                    cp16(st + f_off(vrow_, c), vrowp + (ok ? col : 0), ok);
                                }
                            }
                            // X tile: 16 rows x (PW / 4) chunks
                            for (int idx = lane; idx < 16 * (P::PW / 4); idx += 32) {
                                const int v = idx / (P::PW / 4), c = idx % (P::PW / 4);
                                const int t = 16 * s + v;
                                const int64_t col = n0 + 4 * c;
                                const bool ok = t < tn && col + 4 <= ldx;
                                const float *src = X + (ok ? (int64_t)s_x[t] * ldx + col : 0);
                                cp16(st + P::kVBytes + v * P::kXRow + 16 * c, src, ok);
                            }
                        }
                        cp_commit();
                    };
#pragma unroll
                    for (int s = 0; s < S - 1; ++s) issue(s);
                    const int ni = (w.B + 3) >> 2;   // row groups of the item: rows rg + 4 i, i < ni
                    for (int s = 0; s < nsteps; ++s) {
                        cp_wait<S - 2>();
                        __syncwarp();
                        issue(s + S - 1);
                        const unsigned char *st = ring + (s % S) * P::kBytes;
                        // only the row groups the item has (a 4-row item computes a quarter)
                        switch (ni) {
                            case 1: f32_stage<NT, 1>(st, rg, cg, vg, acc); break;
                            case 2: f32_stage<NT, 2>(st, rg, cg, vg, acc); break;
                            case 3: f32_stage<NT, 3>(st, rg, cg, vg, acc); break;
                            default: f32_stage<NT, 4>(st, rg, cg, vg, acc); break;
                        }
                    }
                    cp_wait_all();
                    __syncwarp();
                }
            }
            if (P::V == 2) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < P::CPL; ++j) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], 16);
            }
            // epilogue: rows rg + 4 i, columns n0 + cg CPL + j (the first half of the lanes
            // when the virtual columns were split)
            if (vg == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = rg + 4 * i;
                    if (r >= w.B) continue;
                    const int64_t row = w.yrow + r;
#pragma unroll
                    for (int j = 0; j < P::CPL; ++j) {
                        const int64_t col = n0 + cg * P::CPL + j;
                        if (col >= a.k) continue;
                        TX *yp = Y + row * a.ldy + col;
                        TX o = sc.alpha * (TX)acc[i][j];
                        if (a.beta_nz) o += sc.beta * *yp;
                        if (a.gamma_nz) o += sc.gamma * Z[row * a.ldz + col];
                        *yp = o;
                        if (want_dot) dot += (double)R[row * a.ldr + col] * (double)o;
                    }
                }
            }
        }
        if (a.item_partials) {
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
            double sum = 0.0;
            for (int i = 0; i < warps; ++i) sum += s_dot[i];
            a.partials[blockIdx.x] = sum;
        }
    }
}

template <int NT>
size_t fpipe_smem(int warps) {
    return (size_t)warps * ((size_t)F32Pipe<NT>::S * F32Pipe<NT>::kBytes + kKMax * sizeof(int32_t));
}

template <int NT, typename TX>
cudaError_t fpipe_launch(const ProdArgs &a, cudaStream_t s) {
    const size_t smem = fpipe_smem<NT>(a.warps);
    cudaError_t e = cudaFuncSetAttribute((const void *)fma32_pipe_kernel<NT, TX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fma32_pipe_kernel<NT, TX><<<a.grid, a.warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int pipe_nt(int64_t k) { return k <= 8 ? 1 : (k <= 16 ? 2 : 4); }

int64_t pipe_ldp(int64_t k) {
    const int64_t w = 8 * pipe_nt(k);
    return (k + w - 1) / w * w;
}

size_t mma_pipe_smem_bytes(int mode, int64_t k, int warps) {
    const int nt = pipe_nt(k);
    if (mode != kBF16X2) return nt == 1 ? tf_smem<1>(warps) : nt == 2 ? tf_smem<2>(warps) : tf_smem<4>(warps);
    return nt == 1 ? pipe_smem<1>(warps) : nt == 2 ? pipe_smem<2>(warps) : pipe_smem<4>(warps);
}

const void *mma_pipe_kernel_ptr(int mode, int64_t k) {
    const int nt = pipe_nt(k);
    if (mode == kTF32)
        return nt == 1 ? (const void *)mma_tf32_pipe_kernel<1, kTF32>
                       : nt == 2 ? (const void *)mma_tf32_pipe_kernel<2, kTF32>
                                 : (const void *)mma_tf32_pipe_kernel<4, kTF32>;
    if (mode == kTF32X3)
        return nt == 1 ? (const void *)mma_tf32_pipe_kernel<1, kTF32X3>
                       : nt == 2 ? (const void *)mma_tf32_pipe_kernel<2, kTF32X3>
                                 : (const void *)mma_tf32_pipe_kernel<4, kTF32X3>;
    return nt == 1 ? (const void *)mma_bf16_pipe_kernel<1>
                   : nt == 2 ? (const void *)mma_bf16_pipe_kernel<2> : (const void *)mma_bf16_pipe_kernel<4>;
}

cudaError_t launch_mma_pipe(int mode, const ProdArgs &a, cudaStream_t s) {
    const int nt = pipe_nt(a.k);
    if (mode == kTF32) return nt == 1 ? tf_launch<1, kTF32>(a, s) : nt == 2 ? tf_launch<2, kTF32>(a, s)
                                                                           : tf_launch<4, kTF32>(a, s);
    if (mode == kTF32X3) return nt == 1 ? tf_launch<1, kTF32X3>(a, s) : nt == 2 ? tf_launch<2, kTF32X3>(a, s)
                                                                               : tf_launch<4, kTF32X3>(a, s);
    if (nt == 1) return pipe_launch<1>(a, s);
    if (nt == 2) return pipe_launch<2>(a, s);
    return pipe_launch<4>(a, s);
}

size_t fma32_pipe_smem_bytes(int64_t k, int warps) {
    const int nt = pipe_nt(k);
    return nt == 1 ? fpipe_smem<1>(warps) : nt == 2 ? fpipe_smem<2>(warps) : fpipe_smem<4>(warps);
}

const void *fma32_pipe_kernel_ptr(int64_t k, bool ydouble) {
    const int nt = pipe_nt(k);
    if (ydouble)
        return nt == 1 ? (const void *)fma32_pipe_kernel<1, double>
                       : nt == 2 ? (const void *)fma32_pipe_kernel<2, double> : (const void *)fma32_pipe_kernel<4, double>;
    return nt == 1 ? (const void *)fma32_pipe_kernel<1, float>
                   : nt == 2 ? (const void *)fma32_pipe_kernel<2, float> : (const void *)fma32_pipe_kernel<4, float>;
}

cudaError_t launch_fma32_pipe(bool ydouble, const ProdArgs &a, cudaStream_t s) {
    const int nt = pipe_nt(a.k);
    if (ydouble) return nt == 1 ? fpipe_launch<1, double>(a, s) : nt == 2 ? fpipe_launch<2, double>(a, s)
                                                                          : fpipe_launch<4, double>(a, s);
    return nt == 1 ? fpipe_launch<1, float>(a, s) : nt == 2 ? fpipe_launch<2, float>(a, s)
                                                            : fpipe_launch<4, float>(a, s);
}

}  // namespace vbcsr
