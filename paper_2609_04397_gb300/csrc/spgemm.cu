// Thresholded block sparse product C = A B (Eqs. 2-3): device kernels for the
// block norms, the numeric stage and the compaction after the final filter.
// The symbolic stage (candidate blocks, norm bounds, product lists grouped by
// shape) runs on the host in api.cu.
#include "internal.cuh"

namespace vbcsr {

// Frobenius norm of every plan block of an operator stored in panels.
template <typename T>
__global__ void block_norms_kernel(int64_t nblk, const T *panel, const int64_t *pbase, const int32_t *kp,
                                   const int32_t *bi, const int32_t *bj, double *out, int warps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t l = (int64_t)blockIdx.x * warps + warp; l < nblk; l += (int64_t)gridDim.x * warps) {
        const int h = bi[l], w = bj[l];
        const int64_t pb = pbase[l], s = kp[l];
        double acc = 0.0;
        for (int e = lane; e < h * w; e += 32) {
            const int p = e / w, q = e - p * w;
            const double v = (double)panel[pb + p * s + q];
            acc += v * v;
        }
        for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
        if (lane == 0) out[l] = sqrt(acc);
    }
}

cudaError_t launch_block_norms(bool f64, int64_t nblk, const void *panel, const int64_t *pbase, const int32_t *kp,
                               const int32_t *bi, const int32_t *bj, double *out, cudaStream_t s) {
    if (nblk == 0) return cudaSuccess;
    const int warps = 8;
    const int64_t need = (nblk + warps - 1) / warps;
    const int grid = (int)(need < 65536 ? need : 65536);
    if (f64)
        block_norms_kernel<double><<<grid, warps * 32, 0, s>>>(nblk, (const double *)panel, pbase, kp, bi, bj, out,
                                                               warps);
    else
        block_norms_kernel<float><<<grid, warps * 32, 0, s>>>(nblk, (const float *)panel, pbase, kp, bi, bj, out,
                                                              warps);
    return cudaGetLastError();
}

// One warp per output block: lanes own its entries (p, q) and sum
// A_ik[p, :] B_kj[:, q] over the block's product list; the result goes to
// the packed-order output at uoff[o]. The norm of the finished block is
// written to norms[o].
template <typename T>
__global__ void spgemm_numeric_kernel(SpgemmArgs g, int warps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ B = static_cast<const T *>(g.B);
    T *__restrict__ C = static_cast<T *>(g.C);
    for (int64_t o = (int64_t)blockIdx.x * warps + warp; o < g.n_out; o += (int64_t)gridDim.x * warps) {
        const int bi = g.out_bi[o], bj = g.out_bj[o];
        const int ne = bi * bj;
        const int64_t p0 = g.out_pbeg[o], p1 = g.out_pbeg[o + 1];
        double nrm = 0.0;
        for (int e0 = 0; e0 < ne; e0 += 32) {
            const int e = e0 + lane;
            const bool live = e < ne;
            const int p = live ? e / bj : 0, q = live ? e - (e / bj) * bj : 0;
            T acc = (T)0;
            if (live) {
                for (int64_t u = p0; u < p1; ++u) {
                    const T *ar = A + g.pa[u] + (int64_t)p * g.kpa[u];
                    const T *bc = B + g.pb[u] + q;
                    const int64_t sb = g.kpb[u];
                    const int bk = g.bk[u];
                    for (int kk = 0; kk < bk; ++kk) acc = fma(__ldg(ar + kk), __ldg(bc + kk * sb), acc);
                }
                C[g.out_uoff[o] + e] = acc;
                nrm += (double)acc * (double)acc;
            }
        }
        for (int m = 16; m > 0; m >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, m);
        if (lane == 0) g.norms[o] = sqrt(nrm);
    }
}

cudaError_t launch_spgemm_numeric(bool f64, const SpgemmArgs &g, cudaStream_t s) {
    if (g.n_out == 0) return cudaSuccess;
    const int warps = 8;
    const int64_t need = (g.n_out + warps - 1) / warps;
    const int grid = (int)(need < 65536 ? need : 65536);
    if (f64) spgemm_numeric_kernel<double><<<grid, warps * 32, 0, s>>>(g, warps);
    else spgemm_numeric_kernel<float><<<grid, warps * 32, 0, s>>>(g, warps);
    return cudaGetLastError();
}

// dst[new_off[o] ..] = src[old_off[keep[o]] ..] (size[o] elements) for the kept blocks.
template <typename T>
__global__ void compact_kernel(int64_t n, const int64_t *keep_src, const int64_t *dst_off, const int32_t *size,
                               const T *src, T *dst, int warps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t o = (int64_t)blockIdx.x * warps + warp; o < n; o += (int64_t)gridDim.x * warps)
        for (int e = lane; e < size[o]; e += 32) dst[dst_off[o] + e] = src[keep_src[o] + e];
}

cudaError_t launch_compact(bool f64, int64_t n, const int64_t *keep_src, const int64_t *dst_off, const int32_t *size,
                           const void *src, void *dst, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int warps = 8;
    const int64_t need = (n + warps - 1) / warps;
    const int grid = (int)(need < 65536 ? need : 65536);
    if (f64)
        compact_kernel<double><<<grid, warps * 32, 0, s>>>(n, keep_src, dst_off, size, (const double *)src,
                                                           (double *)dst, warps);
    else
        compact_kernel<float><<<grid, warps * 32, 0, s>>>(n, keep_src, dst_off, size, (const float *)src,
                                                          (float *)dst, warps);
    return cudaGetLastError();
}

}  // namespace vbcsr
