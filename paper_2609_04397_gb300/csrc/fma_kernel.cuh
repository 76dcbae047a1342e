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
// in registers; the tg lanes of a column then combine them (a reduce-scatter
// when KC = 1, a butterfly otherwise), and each output entry is written once
// by one lane (no atomics). The epilogue applies alpha, beta, gamma * Z and
// accumulates the optional FP64 dot with R.
//
// Two launch shapes share the per-item code: one launch per row count B over
// the items of that count, and one persistent launch over all items (a switch
// on B per item) that takes items from a work queue in descending-cost order.
// Kernel forms (template flags): WIDE (double-FP32 pairs read four columns per
// lane for items of up to 13 rows, else two) and RING (FP32 values and
// double-FP32 pairs streamed through a ring of shared-memory stages filled by
// asynchronous copies, for wide column tiles); the host picks them from the
// operator's row counts and k.
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace vbcsr {

template <typename T>
__device__ __forceinline__ T ld_ro(const T *p) { return __ldg(p); }

// 16 bytes from global to shared memory, asynchronously (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

// The value as the adjoint product uses it: itself for real types (complex
// types overload this with the conjugate).
template <typename T>
__device__ __forceinline__ T adj_val(T v) { return v; }

// Stage the X row (and, for the adjoint, the value address) of virtual
// columns [t0, t0 + tn) of item w in shared memory.
template <bool TRANS>
__device__ __forceinline__ void stage_columns(const ProdArgs &a, const WorkItem &w, int t0, int tn,
                                              int32_t *s_x, int64_t *s_a, int lane) {
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

template <typename TX>
__device__ __forceinline__ void write_out(const ProdArgs &a, int64_t row, int64_t c, TX acc, double &dot) {
    TX *Y = static_cast<TX *>(a.Y);
    TX *yp = Y + row * a.ldy + c;
    const EpiScalars<TX> sc = epi_scalars<TX>(a);
    TX r = sc.alpha * acc;
    if (a.beta_nz) r += sc.beta * *yp;
    if (a.gamma_nz) r += sc.gamma * static_cast<const TX *>(a.Z)[row * a.ldz + c];
    *yp = r;
    if (a.partials || a.item_partials) dot += (double)static_cast<const TX *>(a.R)[row * a.ldr + c] * (double)r;
}

// complex Y (interleaved re, im): real alpha, beta, gamma; the dot is the real
// part of sum(conj(R) .* Y)
template <>
__device__ __forceinline__ void write_out<double2>(const ProdArgs &a, int64_t row, int64_t c, double2 acc,
                                                   double &dot) {
    double2 *yp = static_cast<double2 *>(a.Y) + row * a.ldy + c;
    double2 r = make_double2(a.alpha * acc.x, a.alpha * acc.y);
    if (a.beta_nz) {
        const double2 y = *yp;
        r.x += a.beta * y.x;
        r.y += a.beta * y.y;
    }
    if (a.gamma_nz) {
        const double2 z = static_cast<const double2 *>(a.Z)[row * a.ldz + c];
        r.x += a.gamma * z.x;
        r.y += a.gamma * z.y;
    }
    *yp = r;
    if (a.partials || a.item_partials) {
        const double2 q = static_cast<const double2 *>(a.R)[row * a.ldr + c];
        dot += q.x * r.x + q.y * r.y;
    }
}

// Reduce-scatter of B (<= 16) per-lane partial sums over all 32 lanes, sized
// to NV = the next power of two >= B: halving steps over the lane bits 16, 8,
// 4, 2 while more than one value remains, plain butterfly steps for the rest.
// Afterwards the lanes whose bits select row rs_row<NV>(lane) hold that row's
// full sum. It costs (NV - 1) + (5 - log2 NV) adds per lane (5 for B <= 2,
// 16 for B > 8) instead of 5 * B; FP64 adds are issued per warp instruction
// on GB300's narrow FP64 pipe, so this matters for small rows.
template <int B>
struct RsShape {
    static constexpr int NV = B <= 1 ? 1 : B <= 2 ? 2 : B <= 4 ? 4 : B <= 8 ? 8 : 16;
    static constexpr int LOG = NV == 1 ? 0 : NV == 2 ? 1 : NV == 4 ? 2 : NV == 8 ? 3 : 4;
};

template <int NV>
__device__ __forceinline__ int rs_row(int lane) {
    // the halving steps use lane bits 16, 8, 4, 2 in that order
    int r = 0;
    if (NV >= 2) r += ((lane >> 4) & 1) * (NV / 2);
    if (NV >= 4) r += ((lane >> 3) & 1) * (NV / 4);
    if (NV >= 8) r += ((lane >> 2) & 1) * (NV / 8);
    if (NV >= 16) r += ((lane >> 1) & 1);
    return r;
}

template <int B, typename TA>
__device__ __forceinline__ TA reduce_scatter32(const TA (&acc)[B], int lane) {
    constexpr int NV = RsShape<B>::NV;
    TA v[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = (j < B) ? acc[j] : (TA)0;
    // halving steps: keep the half selected by the lane bit, receive the partner's copy of it
#pragma unroll
    for (int h = NV / 2, bit = 16; h >= 1; h >>= 1, bit >>= 1) {
        const bool up = lane & bit;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const TA keep = up ? v[j + h] : v[j], send = up ? v[j] : v[j + h];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    // one value left; add over the lane bits not used above
    TA r = v[0];
#pragma unroll
    for (int bit = 16 >> RsShape<B>::LOG; bit >= 1; bit >>= 1) r += __shfl_xor_sync(0xffffffffu, r, bit);
    return r;
}

template <int B, bool TRANS, typename TV, typename TA, typename TX, typename TXI, bool WIDE = true, bool RING = false>
__device__ __forceinline__ void process_item(const ProdArgs &a, const WorkItem &w, int KC, int32_t *s_x,
                                             int64_t *s_a, float *s_ring, int lane, double &dot) {
    const int TG = 32 / KC;
    const int cl = lane % KC;
    const int tg = lane / KC;
    const TV *__restrict__ vals = static_cast<const TV *>(a.values);
    const TXI *__restrict__ X = static_cast<const TXI *>(a.X);
    const bool do_prod = a.alpha != 0.0;

    for (int64_t c0 = 0; c0 < a.k; c0 += KC) {
        const int64_t c = c0 + cl;
        const bool cv = c < a.k;
        TA acc[B];
#pragma unroll
        for (int p = 0; p < B; ++p) acc[p] = (TA)0;

        if (do_prod) {
            for (int t0 = 0; t0 < w.K; t0 += kKMax) {
                const int tn = min(kKMax, w.K - t0);
                if (c0 == 0 || w.K > kKMax) stage_columns<TRANS>(a, w, t0, tn, s_x, s_a, lane);
                if constexpr (!TRANS && sizeof(TV) == 4 && RING) {
                    if (KC >= 4) {
                        // FP32 values through a ring of kRingStages stages of kRingCols
                        // panel columns in shared memory, filled by asynchronous 16-byte
                        // copies two stages ahead: with wide column tiles (the host picks
                        // this form for k >= 8) each step covers few panel columns, and
                        // loading the values in the step left too few bytes in flight to
                        // cover the DRAM latency. Lanes read their four columns of every
                        // row from the stage (lanes of one column group share the address).
                        const int ncs = (tn + kRingCols - 1) / kRingCols;
                        auto issue = [&](int si) {
                            if (si < ncs) {
                                float *dst = s_ring + (si % kRingStages) * (16 * kRingCols);
                                for (int q = lane; q < B * (kRingCols / 4); q += 32) {
                                    const int p = q / (kRingCols / 4), col = si * kRingCols + (q % (kRingCols / 4)) * 4;
                                    float *d = dst + p * kRingCols + (col - si * kRingCols);
                                    if (t0 + col < w.Kp)   // Kp is a multiple of 4: the chunk is inside the row
                                        cp_async16(d, vals + w.vbase + (int64_t)p * w.Kp + t0 + col);
                                    else
                                        *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
                                }
                            }
                            asm volatile("cp.async.commit_group;" ::: "memory");
                        };
                        // X of the lane's next four columns is loaded before the current
                        // columns' multiply-adds (one group ahead, in registers)
                        auto load_x = [&](int t, TA (&x)[4]) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int xr = (t + j < tn) ? s_x[t + j] : -1;
                                x[j] = (cv && xr >= 0) ? (TA)ld_ro(X + (int64_t)xr * a.ldx + c) : (TA)0;
                            }
                        };
                        __syncwarp();
                        issue(0);
                        issue(1);
                        TA x[4];
                        load_x(4 * tg, x);
                        for (int si = 0; si < ncs; ++si) {
                            issue(si + 2);
                            asm volatile("cp.async.wait_group 2;" ::: "memory");
                            __syncwarp();
                            const float *st = s_ring + (si % kRingStages) * (16 * kRingCols);
                            for (int tt = 4 * tg; tt < kRingCols; tt += 4 * TG) {
                                const int t = si * kRingCols + tt;
                                TA xn[4];
                                load_x(t + 4 * TG, xn);
#pragma unroll
                                for (int p = 0; p < B; ++p) {
                                    const float4 q = *reinterpret_cast<const float4 *>(st + p * kRingCols + tt);
                                    acc[p] = fmat((TA)q.x, x[0], acc[p]);
                                    acc[p] = fmat((TA)q.y, x[1], acc[p]);
                                    acc[p] = fmat((TA)q.z, x[2], acc[p]);
                                    acc[p] = fmat((TA)q.w, x[3], acc[p]);
                                }
#pragma unroll
                                for (int j = 0; j < 4; ++j) x[j] = xn[j];
                            }
                            __syncwarp();
                        }
                        asm volatile("cp.async.wait_all;" ::: "memory");
                        __syncwarp();
                        continue;
                    }
                }
                if (!TRANS && sizeof(TV) == 4) {
                    // FP32 values: four consecutive panel columns per lane and step, one
                    // 16-byte load per row (rows start 16-byte aligned; Kp is a multiple
                    // of 4, so the four columns never leave the row)
                    for (int t = 4 * tg; t < tn; t += 4 * TG) {
                        TA x[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int xr = (t + j < tn) ? s_x[t + j] : -1;
                            x[j] = (cv && xr >= 0) ? (TA)ld_ro(X + (int64_t)xr * a.ldx + c) : (TA)0;
                        }
                        const TV *v = vals + w.vbase + t0 + t;
                        const int64_t kp = w.Kp;
#pragma unroll
                        for (int p = 0; p < B; ++p) {
                            const float4 q = __ldg(reinterpret_cast<const float4 *>(v + p * kp));
                            acc[p] = fmat((TA)q.x, x[0], acc[p]);
                            acc[p] = fmat((TA)q.y, x[1], acc[p]);
                            acc[p] = fmat((TA)q.z, x[2], acc[p]);
                            acc[p] = fmat((TA)q.w, x[3], acc[p]);
                        }
                    }
                    continue;
                }
                if constexpr (!TRANS && sizeof(TV) == 8 && RING) {
                    if (KC >= 4) {
                        // double-FP32 pairs through the ring (as the FP32 values above:
                        // stages of kRingCols / 2 panel columns of 8-byte values filled
                        // by asynchronous 16-byte copies two stages ahead), CPL columns per
                        // lane as below, X one column group ahead
                        constexpr int RC = kRingCols / 2;
                        constexpr int CPL = (WIDE && B <= 13) ? 4 : 2;
                        TV *ring = reinterpret_cast<TV *>(s_ring);
                        const int ncs = (tn + RC - 1) / RC;
                        auto issue = [&](int si) {
                            if (si < ncs) {
                                TV *dst = ring + (si % kRingStages) * (16 * RC);
                                for (int q = lane; q < B * (RC / 2); q += 32) {
                                    const int p = q / (RC / 2), col = si * RC + (q % (RC / 2)) * 2;
                                    TV *d = dst + p * RC + (col - si * RC);
                                    if (t0 + col < w.Kp)   // Kp is even: the pair is inside the row
                                        cp_async16(d, vals + w.vbase + (int64_t)p * w.Kp + t0 + col);
                                    else
                                        *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
                                }
                            }
                            asm volatile("cp.async.commit_group;" ::: "memory");
                        };
                        auto load_x = [&](int t, TA (&x)[CPL]) {
#pragma unroll
                            for (int j = 0; j < CPL; ++j) {
                                const int xr = (t + j < tn) ? s_x[t + j] : -1;
                                x[j] = (cv && xr >= 0) ? (TA)ld_ro(X + (int64_t)xr * a.ldx + c) : (TA)0;
                            }
                        };
                        __syncwarp();
                        issue(0);
                        issue(1);
                        TA x[CPL];
                        load_x(CPL * tg, x);
                        for (int si = 0; si < ncs; ++si) {
                            issue(si + 2);
                            asm volatile("cp.async.wait_group 2;" ::: "memory");
                            __syncwarp();
                            const TV *st = ring + (si % kRingStages) * (16 * RC);
                            for (int tt = CPL * tg; tt < RC; tt += CPL * TG) {
                                const int t = si * RC + tt;
                                TA xn[CPL];
                                load_x(t + CPL * TG, xn);
#pragma unroll
                                for (int p = 0; p < B; ++p) {
#pragma unroll
                                    for (int h = 0; h < CPL; h += 2) {
                                        const uint4 q = *reinterpret_cast<const uint4 *>(st + p * RC + tt + h);
                                        TV v2[2];
                                        memcpy(v2, &q, sizeof(v2));
                                        acc[p] = fmat((TA)v2[0], x[h], acc[p]);
                                        acc[p] = fmat((TA)v2[1], x[h + 1], acc[p]);
                                    }
                                }
#pragma unroll
                                for (int j = 0; j < CPL; ++j) x[j] = xn[j];
                            }
                            __syncwarp();
                        }
                        asm volatile("cp.async.wait_all;" ::: "memory");
                        __syncwarp();
                        continue;
                    }
                }
                if (!TRANS && sizeof(TV) == 8) {
                    // 8-byte values (FP64, double-FP32 pairs): CPL consecutive panel columns
                    // per lane and step, 16-byte loads (rows start 32-byte aligned and Kp is
                    // a multiple of 4, so the columns never leave the row): more bytes per
                    // load instruction and more independent multiply-adds in flight. FP64
                    // takes 2. The FP32-pipe double-FP32 arithmetic takes 4 for items of up
                    // to 13 rows when WIDE, else 2: the wide form is twice the code per row
                    // count, and a persistent launch that runs many row counts at once
                    // (measured: nine on a variable-block operator with b in [9, 20]) ran
                    // 1.4x slower with it, while one or two row counts ran 3-10 % faster.
                    constexpr int CPL = sizeof(TA) == 8 && alignof(TA) == 8 ? 2 : (WIDE && B <= 13 ? 4 : 2);
                    for (int t = CPL * tg; t < tn; t += CPL * TG) {
                        TA x[CPL];
#pragma unroll
                        for (int j = 0; j < CPL; ++j) {
                            const int xr = (t + j < tn) ? s_x[t + j] : -1;
                            x[j] = (cv && xr >= 0) ? (TA)ld_ro(X + (int64_t)xr * a.ldx + c) : (TA)0;
                        }
                        const TV *v = vals + w.vbase + t0 + t;
                        const int64_t kp = w.Kp;
#pragma unroll
                        for (int p = 0; p < B; ++p) {
#pragma unroll
                            for (int h = 0; h < CPL; h += 2) {
                                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(v + p * kp + h));
                                TV v2[2];
                                memcpy(v2, &q, sizeof(v2));
                                acc[p] = fmat((TA)v2[0], x[h], acc[p]);
                                acc[p] = fmat((TA)v2[1], x[h + 1], acc[p]);
                            }
                        }
                    }
                    continue;
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
                    } else if constexpr (sizeof(TV) == 8) {
                        // 8-byte values: the B values of the column (contiguous, any
                        // parity) come from the aligned 16-byte pairs that cover them, half
                        // the load requests of one load per value; a select picks each
                        // value by the start's parity (the pages carry two elements of
                        // slack after their end for the last pair)
                        const TV *v = vals + s_a[t];
                        const bool odd = (reinterpret_cast<uintptr_t>(v) & 15) != 0;
                        const uint4 *vp = reinterpret_cast<const uint4 *>(reinterpret_cast<uintptr_t>(v) &
                                                                          ~static_cast<uintptr_t>(15));
                        constexpr int NP = B / 2 + 1;
                        TV e[2 * NP];
#pragma unroll
                        for (int m = 0; m < NP; ++m) {
                            const uint4 q = __ldg(vp + m);
                            memcpy(&e[2 * m], &q, sizeof(q));
                        }
#pragma unroll
                        for (int p = 0; p < B; ++p) acc[p] = fmat(adj_val((TA)(odd ? e[p + 1] : e[p])), x, acc[p]);
                    } else {
                        const TV *v = vals + s_a[t];
#pragma unroll
                        for (int p = 0; p < B; ++p) acc[p] = fmat(adj_val((TA)ld_ro(v + p)), x, acc[p]);
                    }
                }
            }
        }
        if (KC == 1) {
            // every lane worked on column c0; one reduce-scatter finishes all rows.
            // Lanes agreeing in the bits the halving steps used hold the same row:
            // the one with the unused low bits clear writes it.
            constexpr int NV = RsShape<B>::NV, LOG = RsShape<B>::LOG;
            const TA v = reduce_scatter32<B>(acc, lane);
            const int p = rs_row<NV>(lane);
            const int owner_mask = (16 >> LOG) * 2 - 1;   // lane bits below the last halving bit
            if ((lane & owner_mask) == 0 && p < B && cv) write_out<TX>(a, w.yrow + p, c, (TX)v, dot);
        } else {
            for (int m = KC; m < 32; m <<= 1) {
#pragma unroll
                for (int p = 0; p < B; ++p) acc[p] += __shfl_xor_sync(0xffffffffu, acc[p], m);
            }
            // every lane of column c now holds all B sums; lane group tg writes rows
            // tg, tg + TG, ...: each epilogue step stores TG rows with the whole warp
            // (the epilogue's FP64 instructions are charged per warp instruction)
            for (int p0 = 0; p0 < B; p0 += TG) {
                const int p = p0 + tg;
                TA v = acc[0];
#pragma unroll
                for (int q = 1; q < B; ++q)
                    if (q == p) v = acc[q];
                if (p < B && cv) write_out<TX>(a, w.yrow + p, c, (TX)v, dot);
            }
        }
    }
}

__device__ __forceinline__ void finish_dot(const ProdArgs &a, double dot, int warp, int lane, int warps) {
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

template <int B, bool TRANS, typename TV, typename TA, typename TX, typename TXI, bool RING = false>
__global__ void __launch_bounds__(256, 2) fma_product_kernel(ProdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw) + warp * kKMax;
    int64_t *s_a = reinterpret_cast<int64_t *>(smem_raw + (size_t)warps * kKMax * sizeof(int32_t)) +
                   warp * kKMax;
    float *s_ring = reinterpret_cast<float *>(smem_raw + (size_t)warps * kKMax * sizeof(int32_t)) +
                    (size_t)warp * (kRingBytes / sizeof(float));   // forward launches with RING only
    double dot = 0.0;
    for (int64_t it = (int64_t)blockIdx.x * warps + warp; it < a.n_items; it += (int64_t)gridDim.x * warps) {
        const WorkItem w = a.items[it];
        process_item<B, TRANS, TV, TA, TX, TXI, true, RING>(a, w, a.kc, s_x, s_a, s_ring, lane, dot);
    }
    if (a.partials) finish_dot(a, dot, warp, lane, warps);
}

// One launch over items of every row count. Items come from a.items in
// order (the planner sorts them by descending cost); warps take the next
// item from a device counter (a.queue, zeroed before the launch) or, without
// a queue, round-robin. a.kc_of(B) is the column tile of row count B.
template <bool TRANS, typename TV, typename TA, typename TX, typename TXI, bool WIDE = true, bool RING = false>
__global__ void __launch_bounds__(256, 2) fma_persistent_kernel(ProdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = a.warps;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw) + warp * kKMax;
    int64_t *s_a = reinterpret_cast<int64_t *>(smem_raw + (size_t)warps * kKMax * sizeof(int32_t)) +
                   warp * kKMax;
    float *s_ring = reinterpret_cast<float *>(smem_raw + (size_t)warps * kKMax * sizeof(int32_t)) +
                    (size_t)warp * (kRingBytes / sizeof(float));   // forward launches with RING only
    double dot = 0.0;
    int64_t it = (int64_t)blockIdx.x * warps + warp;
    for (;;) {
        if (a.queue) {
            unsigned long long q = 0;
            if (lane == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(a.queue), 1ull);
            it = (int64_t)__shfl_sync(0xffffffffu, q, 0);
        }
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
        const int kc = a.kc_of(w.B);
#define VBCSR_ITEM_CASE(NB) \
    case NB: process_item<NB, TRANS, TV, TA, TX, TXI, WIDE, RING>(a, w, kc, s_x, s_a, s_ring, lane, dot); break;
        switch (w.B) {
            VBCSR_ITEM_CASE(1) VBCSR_ITEM_CASE(2) VBCSR_ITEM_CASE(3) VBCSR_ITEM_CASE(4)
            VBCSR_ITEM_CASE(5) VBCSR_ITEM_CASE(6) VBCSR_ITEM_CASE(7) VBCSR_ITEM_CASE(8)
            VBCSR_ITEM_CASE(9) VBCSR_ITEM_CASE(10) VBCSR_ITEM_CASE(11) VBCSR_ITEM_CASE(12)
            VBCSR_ITEM_CASE(13) VBCSR_ITEM_CASE(14) VBCSR_ITEM_CASE(15) VBCSR_ITEM_CASE(16)
            default: break;
        }
#undef VBCSR_ITEM_CASE
        if (a.item_partials) {
            // the item's share of the fused dot, at the item's index: the sum over
            // items then runs in a fixed order, whichever warp took which item
            for (int m = 16; m > 0; m >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, m);
            if (lane == 0) a.item_partials[it] = dot;
            dot = 0.0;
        }
        if (!a.queue) it += (int64_t)gridDim.x * warps;
    }
    if (a.partials) finish_dot(a, dot, warp, lane, warps);
}

// Kernels whose dynamic shared memory plus the static dot buffer would pass
// the default 48 KB per CTA need the larger carve-out requested first.
template <typename K>
inline cudaError_t launch_smem_opt_in(K kernel, size_t smem) {
    if (smem + 1024 <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute((const void *)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem + 1024);
}

// Only the double-FP32 pairs (8-byte values, FP32-pipe arithmetic) have a
// narrow form distinct from the wide one.
template <typename TV, typename TA>
constexpr bool kHasNarrowForm = sizeof(TV) == 8 && !(sizeof(TA) == 8 && alignof(TA) == 8);
// FP32 values and double-FP32 pairs have a form that reads them through a
// shared-memory ring (FP64 is bound by its arithmetic, not by the loads)
template <typename TV>
constexpr bool kHasRingForm = sizeof(TV) == 4 || std::is_same<TV, float2>::value;

// narrow: the persistent forward kernel in its narrow form (process_item's
// WIDE = false), for operators with many row counts.
template <typename TV, typename TA, typename TX, typename TXI>
cudaError_t launch_fma_family(int B, bool trans, const ProdArgs &a, cudaStream_t s, bool narrow = false) {
    const int threads = a.warps * 32;
    const bool ring = !trans && a.value_ring && kHasRingForm<TV>;
    const size_t smem = fma_smem_bytes(trans, a.warps, ring);
    cudaError_t e;
    if (B == 0) {   // persistent launch over every row count
        if (trans) {
            if ((e = launch_smem_opt_in(fma_persistent_kernel<true, TV, TA, TX, TXI>, smem)) != cudaSuccess) return e;
            fma_persistent_kernel<true, TV, TA, TX, TXI><<<a.grid, threads, smem, s>>>(a);
        } else if (a.value_ring && kHasRingForm<TV>) {
            if constexpr (kHasRingForm<TV>) {
                auto k = fma_persistent_kernel<false, TV, TA, TX, TXI, true, true>;
                if constexpr (kHasNarrowForm<TV, TA>)
                    if (narrow) k = fma_persistent_kernel<false, TV, TA, TX, TXI, false, true>;
                if ((e = launch_smem_opt_in(k, smem)) != cudaSuccess) return e;
                k<<<a.grid, threads, smem, s>>>(a);
            }
        } else if (narrow && kHasNarrowForm<TV, TA>) {
            if constexpr (kHasNarrowForm<TV, TA>) {
                auto k = fma_persistent_kernel<false, TV, TA, TX, TXI, false>;
                if ((e = launch_smem_opt_in(k, smem)) != cudaSuccess) return e;
                k<<<a.grid, threads, smem, s>>>(a);
            }
        } else {
            if ((e = launch_smem_opt_in(fma_persistent_kernel<false, TV, TA, TX, TXI>, smem)) != cudaSuccess) return e;
            fma_persistent_kernel<false, TV, TA, TX, TXI><<<a.grid, threads, smem, s>>>(a);
        }
        return cudaGetLastError();
    }
#define VBCSR_FMA_CASE(NB)                                                                               \
    case NB:                                                                                             \
        if constexpr (kHasRingForm<TV>) {                                                                \
            if (ring) {                                                                                  \
                auto k = fma_product_kernel<NB, false, TV, TA, TX, TXI, true>;                           \
                if ((e = launch_smem_opt_in(k, smem)) != cudaSuccess) return e;                          \
                k<<<a.grid, threads, smem, s>>>(a);                                                      \
                break;                                                                                   \
            }                                                                                            \
        }                                                                                                \
        if (trans) {                                                                                     \
            if ((e = launch_smem_opt_in(fma_product_kernel<NB, true, TV, TA, TX, TXI>, smem)) != cudaSuccess) \
                return e;                                                                                \
            fma_product_kernel<NB, true, TV, TA, TX, TXI><<<a.grid, threads, smem, s>>>(a);                   \
        } else {                                                                                         \
            if ((e = launch_smem_opt_in(fma_product_kernel<NB, false, TV, TA, TX, TXI>, smem)) != cudaSuccess) \
                return e;                                                                                \
            fma_product_kernel<NB, false, TV, TA, TX, TXI><<<a.grid, threads, smem, s>>>(a);                  \
        }                                                                                                \
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

// The kernel a launch runs (persistent, or the bucket kernel of row count B),
// for its occupancy-derived grid size.
template <typename TV, typename TA, typename TX, typename TXI>
const void *fma_kernel_ptr(bool trans, bool persistent, int B, bool narrow = false, bool ring = false) {
    if (persistent) {
        if (trans) return (const void *)fma_persistent_kernel<true, TV, TA, TX, TXI>;
        if constexpr (kHasRingForm<TV>)
            if (ring) {
                if constexpr (kHasNarrowForm<TV, TA>)
                    if (narrow) return (const void *)fma_persistent_kernel<false, TV, TA, TX, TXI, false, true>;
                return (const void *)fma_persistent_kernel<false, TV, TA, TX, TXI, true, true>;
            }
        if constexpr (kHasNarrowForm<TV, TA>)
            if (narrow) return (const void *)fma_persistent_kernel<false, TV, TA, TX, TXI, false>;
        return (const void *)fma_persistent_kernel<false, TV, TA, TX, TXI>;
    }
#define VBCSR_PTR_CASE(NB)                                                                 \
    case NB:                                                                               \
        if constexpr (kHasRingForm<TV>)                                                    \
            if (ring && !trans) return (const void *)fma_product_kernel<NB, false, TV, TA, TX, TXI, true>; \
        return trans ? (const void *)fma_product_kernel<NB, true, TV, TA, TX, TXI>         \
                     : (const void *)fma_product_kernel<NB, false, TV, TA, TX, TXI>;
    switch (B) {
        VBCSR_PTR_CASE(1) VBCSR_PTR_CASE(2) VBCSR_PTR_CASE(3) VBCSR_PTR_CASE(4)
        VBCSR_PTR_CASE(5) VBCSR_PTR_CASE(6) VBCSR_PTR_CASE(7) VBCSR_PTR_CASE(8)
        VBCSR_PTR_CASE(9) VBCSR_PTR_CASE(10) VBCSR_PTR_CASE(11) VBCSR_PTR_CASE(12)
        VBCSR_PTR_CASE(13) VBCSR_PTR_CASE(14) VBCSR_PTR_CASE(15) VBCSR_PTR_CASE(16)
        default: return nullptr;
    }
#undef VBCSR_PTR_CASE
}

}  // namespace vbcsr
