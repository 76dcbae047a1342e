// Pattern-sampled product (SDDMM), value permutation between packed order and
// panels, and the fixed-order FP64 reductions used by the Chebyshev moments.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "split.cuh"

namespace vbcsr {

size_t fma_smem_bytes(bool trans, int warps, bool ring) {
    return (size_t)warps * kKMax * (sizeof(int32_t) + (trans ? sizeof(int64_t) : 0)) +
           (ring ? (size_t)warps * kRingBytes : 0);
}

int max_resident_ctas(const void *kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    if (smem + 1024 > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem + 1024) != cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) return -1;
    return sms * (per_sm < 1 ? 1 : per_sm);
}

// ---------------------------------------------------------------------------
// SDDMM: D_ij[p, q] = alpha * <A[r_i + p, :], B[c_j + q, :]> + beta * D_ij[p, q].
//
// The forward product's work decomposition read the other way round: one warp
// per work item (B <= 16 rows of a block row, taken in descending cost from a
// device counter); its virtual columns t (the stored blocks' columns c_j + q
// side by side) are staged in shared memory with the packed-order address of
// (row r0 + p, column q) of their block. Lane t keeps the B sums of column t
// in registers, reads its own row of B (contiguous in c) and the item's rows
// of A from shared memory (a broadcast; alpha folded in when they are staged),
// kSdCK columns of c at a time: B FMAs per value read from B, the packed
// output written once per entry.

constexpr int kSdCK = 32;   // columns c of A staged per chunk

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <int B, typename T>
__device__ __forceinline__ void sddmm_item(const SddmmArgs &a, const WorkItem &w, int32_t *s_x, int64_t *s_u,
                                           int32_t *s_w, T *s_a, int lane) {
    const T *__restrict__ A = static_cast<const T *>(a.A);
    const T *__restrict__ Bm = static_cast<const T *>(a.B);
    T *__restrict__ D = static_cast<T *>(a.D);
    const T alpha = (T)a.alpha, beta = (T)a.beta;
    if (w.nlist == 0) return;
    // the item's first row inside its block row (items split rows taller than 16)
    const int64_t r0 = (w.vbase - a.fl_pbase[w.lbegin]) / w.Kp;
    const int nck = (int)((a.k + kSdCK - 1) / kSdCK);
    for (int t0 = 0; t0 < w.K; t0 += kKMax) {
        const int tn = min(kKMax, w.K - t0);
        __syncwarp();
        for (int e = lane; e < w.nlist; e += 32) {
            const int64_t l = w.lbegin + e;
            const int xr = a.fl_xrow[l], pc = a.fl_pcol[l], wd = a.fl_w[l];
            const int64_t u = a.fl_uoff[l] + r0 * wd;
            const int lo = max(pc, t0), hi = min(pc + wd, t0 + tn);
            for (int t = lo; t < hi; ++t) {
                s_x[t - t0] = xr + (t - pc);
                s_u[t - t0] = u + (t - pc);
                s_w[t - t0] = wd;
            }
        }
        __syncwarp();
        for (int tb = 0; tb < tn; tb += 32) {
            const int t = tb + lane;
            const bool tv = t < tn;
            T acc[B];
#pragma unroll
            for (int p = 0; p < B; ++p) acc[p] = (T)0;
            for (int ck = 0; ck < nck; ++ck) {
                const int64_t c0 = (int64_t)ck * kSdCK;
                const int cn = (int)min((int64_t)kSdCK, a.k - c0);
                if (nck > 1 || tb == 0) {   // alpha times the item's rows of A, columns c0 .. c0 + cn
                    __syncwarp();
                    for (int e = lane; e < B * cn; e += 32) {
                        const int p = e / cn, c = e - p * cn;
                        const T v = __ldg(A + (w.yrow + p) * a.lda + c0 + c);
                        s_a[p * kSdCK + c] = a.alpha == 1.0 ? v : alpha * v;
                    }
                    __syncwarp();
                }
                if (tv) {
                    const T *br = Bm + (int64_t)s_x[t] * a.ldb + c0;
                    for (int c = 0; c < cn; ++c) {
                        const T b = __ldg(br + c);
#pragma unroll
                        for (int p = 0; p < B; ++p) acc[p] = fma_t(s_a[p * kSdCK + c], b, acc[p]);
                    }
                }
            }
            if (tv) {
                const int64_t u = s_u[t];
                const int wd = s_w[t];
#pragma unroll
                for (int p = 0; p < B; ++p) {
                    T *d = D + u + (int64_t)p * wd;
                    *d = a.beta != 0.0 ? fma_t(beta, *d, acc[p]) : acc[p];
                }
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(128) sddmm_kernel(SddmmArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *s_a = reinterpret_cast<T *>(smem_raw) + (size_t)warp * 16 * kSdCK;
    int64_t *s_u = reinterpret_cast<int64_t *>(smem_raw + (size_t)warps * 16 * kSdCK * sizeof(T)) + warp * kKMax;
    int32_t *s_x = reinterpret_cast<int32_t *>(smem_raw + (size_t)warps * (16 * kSdCK * sizeof(T) +
                                                                            kKMax * sizeof(int64_t))) +
                   warp * 2 * kKMax;
    int32_t *s_w = s_x + kKMax;
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(reinterpret_cast<unsigned long long *>(a.queue), 1ull);
        const int64_t it = (int64_t)__shfl_sync(0xffffffffu, q, 0);
        if (it >= a.n_items) break;
        const WorkItem w = a.items[it];
#define VBCSR_SDDMM_CASE(NB) \
    case NB: sddmm_item<NB, T>(a, w, s_x, s_u, s_w, s_a, lane); break;
        switch (w.B) {
            VBCSR_SDDMM_CASE(1) VBCSR_SDDMM_CASE(2) VBCSR_SDDMM_CASE(3) VBCSR_SDDMM_CASE(4)
            VBCSR_SDDMM_CASE(5) VBCSR_SDDMM_CASE(6) VBCSR_SDDMM_CASE(7) VBCSR_SDDMM_CASE(8)
            VBCSR_SDDMM_CASE(9) VBCSR_SDDMM_CASE(10) VBCSR_SDDMM_CASE(11) VBCSR_SDDMM_CASE(12)
            VBCSR_SDDMM_CASE(13) VBCSR_SDDMM_CASE(14) VBCSR_SDDMM_CASE(15) VBCSR_SDDMM_CASE(16)
            default: break;
        }
#undef VBCSR_SDDMM_CASE
    }
}

cudaError_t launch_sddmm(bool f64, const SddmmArgs &a, cudaStream_t s) {
    if (a.n_items == 0) return cudaSuccess;
    const int warps = 4, threads = warps * 32;
    const size_t esz = f64 ? sizeof(double) : sizeof(float);
    const size_t smem = (size_t)warps * (16 * kSdCK * esz + kKMax * (sizeof(int64_t) + 2 * sizeof(int32_t)));
    static int cap64 = 0, cap32 = 0;
    int &cap = f64 ? cap64 : cap32;
    const void *k = f64 ? (const void *)sddmm_kernel<double> : (const void *)sddmm_kernel<float>;
    if (!cap) {
        cap = max_resident_ctas(k, threads, smem);
        if (cap < 0) {
            cap = 0;
            return cudaGetLastError();
        }
    }
    if (smem + 1024 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem + 1024);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(long long), s);
    if (e != cudaSuccess) return e;
    const int64_t need = (a.n_items + warps - 1) / warps;
    const int grid = (int)(need < cap ? need : cap);
    if (f64) sddmm_kernel<double><<<grid, threads, smem, s>>>(a);
    else sddmm_kernel<float><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// packed order <-> panels (one warp per block)

template <typename T>
__global__ void permute_kernel(bool to_panel, int64_t nblk, const int64_t *uoff, const int64_t *pbase,
                               const int32_t *kp, const int32_t *bi, const int32_t *bj, const T *user,
                               T *panel, int warps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t l = (int64_t)blockIdx.x * warps + warp; l < nblk; l += (int64_t)gridDim.x * warps) {
        const int w = bj[l], h = bi[l];
        const int64_t u = uoff[l], pb = pbase[l], stride = kp[l];
        for (int e = lane; e < h * w; e += 32) {
            const int p = e / w, q = e - p * w;
            if (to_panel) panel[pb + p * stride + q] = user[u + e];
            else ((T *)user)[u + e] = panel[pb + p * stride + q];
        }
    }
}

cudaError_t launch_permute_values(int esize, bool to_panel, int64_t nblk, const int64_t *uoff,
                                  const int64_t *pbase, const int32_t *kp, const int32_t *bi,
                                  const int32_t *bj, const void *user, void *panel, cudaStream_t s) {
    if (nblk == 0) return cudaSuccess;
    const int warps = 8;
    int64_t need = (nblk + warps - 1) / warps;
    int grid = (int)(need < 65536 ? need : 65536);
    if (esize == 16)
        permute_kernel<double2><<<grid, warps * 32, 0, s>>>(to_panel, nblk, uoff, pbase, kp, bi, bj,
                                                            (const double2 *)user, (double2 *)panel, warps);
    else if (esize == 8)
        permute_kernel<double><<<grid, warps * 32, 0, s>>>(to_panel, nblk, uoff, pbase, kp, bi, bj,
                                                           (const double *)user, (double *)panel, warps);
    else if (esize == 4)
        permute_kernel<float><<<grid, warps * 32, 0, s>>>(to_panel, nblk, uoff, pbase, kp, bi, bj,
                                                          (const float *)user, (float *)panel, warps);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reciprocal-space sampling (Eq. 4). First the phase of every edge,
// exp(-2 pi i k . s_e) = cos(pi * 2 k.s_e) - i sin(pi * 2 k.s_e), s_e = R [+ tau_j -
// tau_i] (one FP64 sincospi per edge: GB300's FP64 pipe is narrow, so it is not
// repeated per entry); then block u of the union pattern sums its edges
// ks_ptr[u] .. ks_ptr[u+1] (real b_i x b_j image blocks at ks_voff) times their
// phases, written in packed order at uoff[u]: one warp per block, lanes over
// its entries.

__global__ void kphase_kernel(int64_t n_edges, const double *ks_shift, double k0, double k1, double k2,
                              double2 *phase) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += (int64_t)gridDim.x * blockDim.x) {
        const double ks = 2.0 * (k0 * ks_shift[3 * e] + k1 * ks_shift[3 * e + 1] + k2 * ks_shift[3 * e + 2]);
        double sn, cs;
        sincospi(ks, &sn, &cs);
        phase[e] = make_double2(cs, -sn);
    }
}

__global__ void ksample_kernel(int64_t nblk, const int64_t *ks_ptr, const double2 *phase, const int64_t *ks_voff,
                               const double *ks_vals, const int64_t *uoff, const int32_t *ub_n, double2 *out,
                               int warps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t u = (int64_t)blockIdx.x * warps + warp; u < nblk; u += (int64_t)gridDim.x * warps) {
        const int n = ub_n[u];
        const int64_t e0 = ks_ptr[u], e1 = ks_ptr[u + 1], o = uoff[u];
        for (int q = lane; q < n; q += 32) {
            double re = 0.0, im = 0.0;
            for (int64_t e = e0; e < e1; ++e) {
                const double2 ph = phase[e];
                const double v = ks_vals[ks_voff[e] + q];
                re = fma(v, ph.x, re);
                im = fma(v, ph.y, im);
            }
            out[o + q] = make_double2(re, im);
        }
    }
}

cudaError_t launch_ksample(int64_t nblk, int64_t n_edges, const int64_t *ks_ptr, const double *ks_shift,
                           const int64_t *ks_voff, const double *ks_vals, const int64_t *uoff, const int32_t *ub_n,
                           const double *kfrac, double2 *phase, double2 *out, cudaStream_t s) {
    if (n_edges > 0) {
        int64_t need = (n_edges + 255) / 256;
        kphase_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(n_edges, ks_shift, kfrac[0], kfrac[1],
                                                                         kfrac[2], phase);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nblk == 0) return cudaSuccess;
    const int warps = 8;
    int64_t need = (nblk + warps - 1) / warps;
    int grid = (int)(need < 65536 ? need : 65536);
    ksample_kernel<<<grid, warps * 32, 0, s>>>(nblk, ks_ptr, phase, ks_voff, ks_vals, uoff, ub_n, out, warps);
    return cudaGetLastError();
}

__global__ void convert_kernel(const double *in, float *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

cudaError_t launch_convert_f64_to_f32(const double *in, float *out, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int64_t need = (n + 255) / 256;
    convert_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

__global__ void split_bf16_kernel(const double *in, uint32_t *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = bf16_pieces(in[i]);
}

__global__ void split_bf16_panel_kernel(int64_t rows, int64_t k, const double *in, int64_t ld, uint32_t *out) {
    const int64_t n = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - r * k;
        out[e] = bf16_pieces(in[r * ld + c]);
    }
}

cudaError_t launch_split_bf16(const double *in, uint32_t *out, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int64_t need = (n + 255) / 256;
    split_bf16_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16_panel(int64_t rows, int64_t k, const double *in, int64_t ld, uint32_t *out,
                                    cudaStream_t s) {
    if (rows * k == 0) return cudaSuccess;
    int64_t need = (rows * k + 255) / 256;
    split_bf16_panel_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(rows, k, in, ld, out);
    return cudaGetLastError();
}

__global__ void split_planes_kernel(const double *in, uint16_t *hi, uint16_t *lo, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = bf16_pieces(in[i]);
        hi[i] = (uint16_t)(w & 0xffffu);
        lo[i] = (uint16_t)(w >> 16);
    }
}

__global__ void split_planes_panel_kernel(int64_t rows, int64_t k, const double *in, int64_t ld, uint16_t *hi,
                                          uint16_t *lo, int64_t ldp) {
    const int64_t n = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - r * k;
        const uint32_t w = bf16_pieces(in[r * ld + c]);
        hi[r * ldp + c] = (uint16_t)(w & 0xffffu);
        lo[r * ldp + c] = (uint16_t)(w >> 16);
    }
}

cudaError_t launch_split_bf16_planes(const double *in, uint16_t *hi, uint16_t *lo, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t need = (n + 255) / 256;
    split_planes_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(in, hi, lo, n);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16_planes_panel(int64_t rows, int64_t k, const double *in, int64_t ld, uint16_t *hi,
                                           uint16_t *lo, int64_t ldp, cudaStream_t s) {
    if (rows * k == 0) return cudaSuccess;
    const int64_t need = (rows * k + 255) / 256;
    split_planes_panel_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(rows, k, in, ld, hi, lo, ldp);
    return cudaGetLastError();
}

__global__ void convert_panel_kernel(int64_t rows, int64_t k, const double *in, int64_t ld, float *out,
                                     int64_t ldo) {
    const int64_t n = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - r * k;
        out[r * ldo + c] = (float)in[r * ld + c];
    }
}

cudaError_t launch_convert_panel_f64_to_f32(int64_t rows, int64_t k, const double *in, int64_t ld, float *out,
                                            int64_t ldo, cudaStream_t s) {
    const int64_t need = (rows * k + 255) / 256;
    if (need == 0) return cudaSuccess;
    convert_panel_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(rows, k, in, ld, out, ldo);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fixed-order reductions

__global__ void finalize_dot_kernel(const double *partials, int64_t n, double scale, double *out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int m = blockDim.x / 2; m > 0; m >>= 1) {
        if (threadIdx.x < m) sh[threadIdx.x] += sh[threadIdx.x + m];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = scale * sh[0];
}

// first stage of a long sum: CTA b adds the contiguous chunk [b * chunk, (b + 1) * chunk)
__global__ void chunk_sum_kernel(const double *partials, int64_t n, int64_t chunk, double *out) {
    __shared__ double sh[256];
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    double s = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += partials[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int m = blockDim.x / 2; m > 0; m >>= 1) {
        if (threadIdx.x < m) sh[threadIdx.x] += sh[threadIdx.x + m];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// Fixed-order sum: up to kDotOneStage partials in one CTA; beyond that, chunks of
// kDotChunk partials summed by one CTA each into `scratch` (kDotScratch doubles),
// then those by one CTA. The order depends only on n, so repeated calls give the
// same bits. (One CTA over a million per-item partials took 0.6 ms: one SM's
// bandwidth and a long dependent chain of FP64 adds per thread.)
cudaError_t launch_finalize_dot(const double *partials, int64_t n, double scale, double *out, double *scratch,
                                cudaStream_t s) {
    if (n <= kDotOneStage || scratch == nullptr) {
        finalize_dot_kernel<<<1, 256, 0, s>>>(partials, n, scale, out);
        return cudaGetLastError();
    }
    int64_t chunk = kDotChunk;
    while ((n + chunk - 1) / chunk > kDotScratch) chunk *= 2;
    const int64_t nb = (n + chunk - 1) / chunk;
    chunk_sum_kernel<<<(unsigned)nb, 256, 0, s>>>(partials, n, chunk, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finalize_dot_kernel<<<1, 256, 0, s>>>(scratch, nb, scale, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void dot_panels_kernel(int64_t rows, int64_t k, const T *A, int64_t lda, const T *B, int64_t ldb,
                                  double *partials) {
    __shared__ double sh[256];
    double s = 0.0;
    const int64_t n = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - r * k;
        s += (double)A[r * lda + c] * (double)B[r * ldb + c];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int m = blockDim.x / 2; m > 0; m >>= 1) {
        if (threadIdx.x < m) sh[threadIdx.x] += sh[threadIdx.x + m];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

cudaError_t launch_dot_panels(bool f64, int64_t rows, int64_t k, const void *A, int64_t lda, const void *B,
                              int64_t ldb, double *partials, int64_t cap, int64_t *n_used, cudaStream_t s) {
    int64_t need = (rows * k + 255) / 256;
    int grid = (int)(need < cap ? (need > 0 ? need : 1) : cap);
    if (grid > 4096) grid = 4096;
    if (f64)
        dot_panels_kernel<double><<<grid, 256, 0, s>>>(rows, k, (const double *)A, lda, (const double *)B, ldb,
                                                       partials);
    else
        dot_panels_kernel<float><<<grid, 256, 0, s>>>(rows, k, (const float *)A, lda, (const float *)B, ldb,
                                                      partials);
    *n_used = grid;
    return cudaGetLastError();
}

__global__ void copy_panel_kernel(int64_t rows, int64_t k, const double *src, int64_t lds, double *dst,
                                  int64_t ldd) {
    const int64_t n = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - r * k;
        dst[r * ldd + c] = src[r * lds + c];
    }
}

cudaError_t launch_copy_panel(int64_t rows, int64_t k, const double *src, int64_t lds, double *dst, int64_t ldd,
                              cudaStream_t s) {
    int64_t need = (rows * k + 255) / 256;
    if (need == 0) return cudaSuccess;
    copy_panel_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(rows, k, src, lds, dst, ldd);
    return cudaGetLastError();
}

__global__ void axpby_kernel(int64_t rows, int64_t k, double alpha, const double *X, int64_t ldx, double beta,
                             double *Y, int64_t ldy) {
    const int64_t n = rows * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e - r * k;
        double v = alpha * X[r * ldx + c];
        if (beta != 0.0) v += beta * Y[r * ldy + c];
        Y[r * ldy + c] = v;
    }
}

cudaError_t launch_axpby(int64_t rows, int64_t k, double alpha, const double *X, int64_t ldx, double beta,
                         double *Y, int64_t ldy, cudaStream_t s) {
    int64_t need = (rows * k + 255) / 256;
    if (need == 0) return cudaSuccess;
    axpby_kernel<<<(int)(need < 65536 ? need : 65536), 256, 0, s>>>(rows, k, alpha, X, ldx, beta, Y, ldy);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gershgorin bounds and the shift/scale of the Chebyshev recurrence, both
// walking the forward work items (every panel row exactly once). A panel
// column t of a row r is on the scalar diagonal when its X row equals r.

__device__ __forceinline__ void stage_x_rows(const WorkItem &w, const int32_t *xrow, const int32_t *pcol,
                                             const int32_t *wd, int t0, int tn, int32_t *s_x, int lane) {
    __syncwarp();
    for (int e = lane; e < w.nlist; e += 32) {
        const int64_t l = w.lbegin + e;
        const int xr = xrow[l], pc = pcol[l], bw = wd[l];
        const int lo = max(pc, t0), hi = min(pc + bw, t0 + tn);
        for (int t = lo; t < hi; ++t) s_x[t - t0] = xr + (t - pc);
    }
    __syncwarp();
}

// real and complex (Hermitian) operators: the diagonal's real part, entry moduli
__device__ __forceinline__ double re_part(double v) { return v; }
__device__ __forceinline__ double re_part(double2 v) { return v.x; }
__device__ __forceinline__ double modulus(double v) { return fabs(v); }
__device__ __forceinline__ double modulus(double2 v) { return hypot(v.x, v.y); }
__device__ __forceinline__ double shifted(double v, bool diag, double c, double d) { return (diag ? v - c : v) / d; }
__device__ __forceinline__ double2 shifted(double2 v, bool diag, double c, double d) {
    return make_double2((diag ? v.x - c : v.x) / d, v.y / d);
}

template <typename T>
__global__ void gershgorin_kernel(const WorkItem *items, int64_t n_items, const T *panel, const int32_t *xrow,
                                  const int32_t *pcol, const int32_t *wd, double *partials, int warps) {
    extern __shared__ int32_t s_mem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *s_x = s_mem + warp * kKMax;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t it = (int64_t)blockIdx.x * warps + warp; it < n_items; it += (int64_t)gridDim.x * warps) {
        const WorkItem w = items[it];
        for (int p = 0; p < w.B; ++p) {
            double off = 0.0, dg = 0.0;
            for (int t0 = 0; t0 < w.K; t0 += kKMax) {
                const int tn = min(kKMax, w.K - t0);
                if (p == 0 || w.K > kKMax) stage_x_rows(w, xrow, pcol, wd, t0, tn, s_x, lane);
                for (int t = lane; t < tn; t += 32) {
                    const T v = panel[w.vbase + (int64_t)p * w.Kp + t0 + t];
                    if (s_x[t] == w.yrow + p) dg += re_part(v);
                    else off += modulus(v);
                }
            }
            for (int m = 16; m > 0; m >>= 1) {
                off += __shfl_xor_sync(0xffffffffu, off, m);
                dg += __shfl_xor_sync(0xffffffffu, dg, m);
            }
            lo = fmin(lo, dg - off);
            hi = fmax(hi, dg + off);
        }
    }
    __shared__ double s_lo[32], s_hi[32];
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < warps; ++i) {
            lo = fmin(lo, s_lo[i]);
            hi = fmax(hi, s_hi[i]);
        }
        partials[2 * blockIdx.x] = lo;
        partials[2 * blockIdx.x + 1] = hi;
    }
}

__global__ void minmax_finalize_kernel(const double *partials, int n, double *out) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < n; ++i) {
        lo = fmin(lo, partials[2 * i]);
        hi = fmax(hi, partials[2 * i + 1]);
    }
    out[0] = lo;
    out[1] = hi;
}

cudaError_t launch_gershgorin(bool cplx, const WorkItem *items, int64_t n_items, const void *panel,
                              const int32_t *xrow, const int32_t *pcol, const int32_t *wd, double *partials,
                              int64_t cap, double *out, cudaStream_t s) {
    const int warps = 4;
    int64_t need = (n_items + warps - 1) / warps;
    int grid = (int)(need < cap / 2 ? (need > 0 ? need : 1) : cap / 2);
    if (grid > 2048) grid = 2048;
    const size_t smem = warps * kKMax * sizeof(int32_t);
    if (cplx)
        gershgorin_kernel<double2><<<grid, warps * 32, smem, s>>>(items, n_items, (const double2 *)panel, xrow,
                                                                  pcol, wd, partials, warps);
    else
        gershgorin_kernel<double><<<grid, warps * 32, smem, s>>>(items, n_items, (const double *)panel, xrow,
                                                                 pcol, wd, partials, warps);
    minmax_finalize_kernel<<<1, 1, 0, s>>>(partials, grid, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void shift_scale_kernel(const WorkItem *items, int64_t n_items, T *panel, const int32_t *xrow,
                                   const int32_t *pcol, const int32_t *wd, double c, double d, int warps) {
    extern __shared__ int32_t s_mem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *s_x = s_mem + warp * kKMax;
    for (int64_t it = (int64_t)blockIdx.x * warps + warp; it < n_items; it += (int64_t)gridDim.x * warps) {
        const WorkItem w = items[it];
        for (int t0 = 0; t0 < w.K; t0 += kKMax) {
            const int tn = min(kKMax, w.K - t0);
            stage_x_rows(w, xrow, pcol, wd, t0, tn, s_x, lane);
            for (int p = 0; p < w.B; ++p)
                for (int t = lane; t < tn; t += 32) {
                    T *v = panel + w.vbase + (int64_t)p * w.Kp + t0 + t;
                    *v = shifted(*v, s_x[t] == w.yrow + p, c, d);
                }
        }
    }
}

cudaError_t launch_shift_scale(bool cplx, const WorkItem *items, int64_t n_items, void *panel, const int32_t *xrow,
                               const int32_t *pcol, const int32_t *wd, double c, double d, cudaStream_t s) {
    const int warps = 4;
    int64_t need = (n_items + warps - 1) / warps;
    if (need == 0) return cudaSuccess;
    const int grid = (int)(need < 65536 ? need : 65536);
    const size_t smem = warps * kKMax * sizeof(int32_t);
    if (cplx)
        shift_scale_kernel<double2><<<grid, warps * 32, smem, s>>>(items, n_items, (double2 *)panel, xrow, pcol, wd,
                                                                   c, d, warps);
    else
        shift_scale_kernel<double><<<grid, warps * 32, smem, s>>>(items, n_items, (double *)panel, xrow, pcol, wd, c,
                                                                  d, warps);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// kernel polynomial method: doubling fix-up and DOS reconstruction

// raw[m] holds <t_a, t_b> / (N k) for m = 2n (a = b = n) and m = 2n+1 (a = n+1,
// b = n), m >= 2; turn them into moments: mu_m = 2 raw[m] - mu_(m mod 2).
__global__ void kpm_fixup_kernel(double *mu, int64_t M) {
    const double m0 = mu[0], m1 = M > 1 ? mu[1] : 0.0;
    for (int64_t m = 2 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x)
        mu[m] = 2.0 * mu[m] - ((m & 1) ? m1 : m0);
}

cudaError_t launch_kpm_fixup(double *mu, int64_t M, cudaStream_t s) {
    if (M <= 2) return cudaSuccess;
    kpm_fixup_kernel<<<1, 256, 0, s>>>(mu, M);
    return cudaGetLastError();
}

// rho(x) = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(x)] / (pi sqrt(1 - x^2)); g the Jackson
// factors (jackson != 0) or 1. Each CTA computes g_n mu_n for a chunk of n into shared
// memory; each thread runs T_n(x) = 2 x T_{n-1}(x) - T_{n-2}(x) for its own x.
__global__ void kpm_dos_kernel(const double *mu, int64_t M, int jackson, const double *x, int64_t nx, double *out) {
    constexpr int kChunk = 1024;
    __shared__ double s_c[kChunk];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double xi = i < nx ? x[i] : 0.0;
    const double q = 3.14159265358979323846 / (double)(M + 1);
    const double cotq = cos(q) / sin(q);
    double acc = 0.0, t_prev = 1.0, t_cur = xi;   // T_0, T_1
    for (int64_t n0 = 0; n0 < M; n0 += kChunk) {
        const int nc = (int)min((int64_t)kChunk, M - n0);
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += blockDim.x) {
            const int64_t n = n0 + j;
            double g = 1.0;
            if (jackson) g = ((double)(M - n + 1) * cos(q * n) + sin(q * n) * cotq) / (double)(M + 1);
            s_c[j] = (n == 0 ? 1.0 : 2.0) * g * mu[n];
        }
        __syncthreads();
        for (int j = 0; j < nc; ++j) {
            const int64_t n = n0 + j;
            double tn;
            if (n == 0) tn = 1.0;
            else if (n == 1) tn = xi;
            else {
                tn = 2.0 * xi * t_cur - t_prev;
                t_prev = t_cur;
                t_cur = tn;
            }
            acc += s_c[j] * tn;
        }
    }
    if (i < nx) out[i] = acc / (3.14159265358979323846 * sqrt(1.0 - xi * xi));
}

cudaError_t launch_kpm_dos(const double *mu, int64_t M, int jackson, const double *x, int64_t nx, double *out,
                           cudaStream_t s) {
    if (nx == 0) return cudaSuccess;
    const int64_t grid = (nx + 255) / 256;
    kpm_dos_kernel<<<(unsigned)grid, 256, 0, s>>>(mu, M, jackson, x, nx, out);
    return cudaGetLastError();
}

// Gap of a density of states on an energy grid around a reference energy: one
// CTA. (1) i0 = the grid point nearest the reference (smallest index on a
// tie); (2) the nearest points left and right of i0 whose DOS is not below
// the threshold (NaN counts as not below); the gap is the run between them.
__global__ void __launch_bounds__(1024) kpm_gap_kernel(const double *E, const double *D, int64_t n, double ref,
                                                        double thr, double *out) {
    __shared__ double s_d[32];
    __shared__ long long s_i[32];
    __shared__ long long s_lr[2][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double bd = INFINITY;
    long long bi = n;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
        const double dj = fabs(E[j] - ref);
        if (dj < bd) {          // j increases along the thread's loop: the first minimum is kept
            bd = dj;
            bi = j;
        }
    }
    for (int m = 16; m > 0; m >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, m);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, m);
        if (od < bd || (od == bd && oi < bi)) {
            bd = od;
            bi = oi;
        }
    }
    if (lane == 0) {
        s_d[warp] = bd;
        s_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            if (s_d[w] < s_d[0] || (s_d[w] == s_d[0] && s_i[w] < s_i[0])) {
                s_d[0] = s_d[w];
                s_i[0] = s_i[w];
            }
    }
    __syncthreads();
    const long long i0 = s_i[0];
    long long left = -1, right = n;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
        if (!(D[j] < thr)) {
            if (j < i0 && j > left) left = j;
            if (j > i0 && j < right) right = j;
        }
    }
    for (int m = 16; m > 0; m >>= 1) {
        left = max(left, (long long)__shfl_xor_sync(0xffffffffu, left, m));
        right = min(right, (long long)__shfl_xor_sync(0xffffffffu, right, m));
    }
    if (lane == 0) {
        s_lr[0][warp] = left;
        s_lr[1][warp] = right;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            left = max(left, s_lr[0][w]);
            right = min(right, s_lr[1][w]);
        }
        if (i0 >= n || !(D[i0] < thr)) {
            out[0] = NAN;
            out[1] = NAN;
        } else {
            out[0] = E[left + 1];
            out[1] = E[right - 1];
        }
    }
}

cudaError_t launch_kpm_gap(const double *E, const double *D, int64_t n, double ref, double thr, double *out,
                           cudaStream_t s) {
    kpm_gap_kernel<<<1, 1024, 0, s>>>(E, D, n, ref, thr, out);
    return cudaGetLastError();
}

}  // namespace vbcsr
