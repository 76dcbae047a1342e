// Thresholded block sparse product C = A B (Eqs. 2-3): device kernels for the
// block norms, the symbolic stage (candidate blocks, Eq. 3 norm bounds, kept
// pattern, product lists grouped by inner size), the numeric stage and the
// compaction after the final filter.
#include <climits>

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

namespace {

// A row's workspace: an open-addressing table from candidate block column j
// to its slot, the sorted candidates, their bounds, kept indices and cursors.
struct SymWs {
    double *bound;
    int32_t *keys, *pos, *list, *kidx, *cur;
    int h, cap;
};

__device__ __forceinline__ SymWs sym_ws(unsigned char *base, int h, int cap) {
    SymWs w;
    w.h = h;
    w.cap = cap;
    w.bound = reinterpret_cast<double *>(base);
    w.keys = reinterpret_cast<int32_t *>(base + (size_t)8 * cap);
    w.pos = w.keys + h;
    w.list = w.pos + h;
    w.kidx = w.list + cap;
    w.cur = w.kidx + cap;
    return w;
}

__device__ __forceinline__ uint32_t sym_hash(int32_t j, int h) {
    return ((uint32_t)j * 2654435761u) & (uint32_t)(h - 1);   // Knuth's multiplicative hash
}

// table slot of an inserted key (linear probing, at most h probes)
__device__ __forceinline__ int sym_find(const SymWs &w, int32_t j) {
    uint32_t s = sym_hash(j, w.h);
    for (int probe = 0; probe < w.h; ++probe) {
        const int32_t k = w.keys[s];
        if (k == j || k < 0) return k == j ? (int)s : -1;
        s = (s + 1) & (uint32_t)(w.h - 1);
    }
    return -1;
}

// candidate index of an inserted key (-1 if absent, which the callers skip)
__device__ __forceinline__ int sym_slot(const SymWs &w, int32_t j) {
    const int s = sym_find(w, j);
    return s < 0 ? -1 : w.pos[s];
}

// 1: inserted, 0: present already, -1: table full
__device__ __forceinline__ int sym_insert(const SymWs &w, int32_t j) {
    uint32_t s = sym_hash(j, w.h);
    for (int probe = 0; probe < w.h; ++probe) {
        const int32_t prev = atomicCAS(&w.keys[s], -1, j);
        if (prev == -1) return 1;
        if (prev == j) return 0;
        s = (s + 1) & (uint32_t)(w.h - 1);
    }
    return -1;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// inclusive prefix sum over the lanes
__device__ __forceinline__ int64_t warp_scan64(int64_t v, int lane) {
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

// One block row of the symbolic stage on one warp; false when the row has
// more candidates than the workspace holds (nothing written then).
template <int PASS>
__device__ bool sym_row(const SymArgs &g, int64_t i, const SymWs &w, int lane) {
    const unsigned FULL = 0xffffffffu;
    const unsigned below = (1u << lane) - 1u;
    const int64_t a0 = g.a_rowptr[i], a1 = g.a_rowptr[i + 1];
    for (int s = lane; s < w.h; s += 32) w.keys[s] = -1;
    __syncwarp();

    // candidates: every j reached by a product A_ik B_kj
    int n = 0;
    for (int64_t a = a0; a < a1; ++a) {
        const int32_t k = g.a_col[a];
        const int64_t b0 = g.b_rowptr[k], b1 = g.b_rowptr[k + 1];
        for (int64_t bb = b0; bb < b1; bb += 32) {
            const int64_t b = bb + lane;
            const int r = b < b1 ? sym_insert(w, g.b_col[b]) : 0;
            n += __popc(__ballot_sync(FULL, r == 1));
            if (__any_sync(FULL, r < 0) || n > w.cap) return false;
        }
    }
    __syncwarp();

    // the candidates in increasing j (bitonic sort over the next power of two)
    int base = 0;
    for (int s0 = 0; s0 < w.h; s0 += 32) {
        const int32_t key = w.keys[s0 + lane];
        const unsigned m = __ballot_sync(FULL, key >= 0);
        if (key >= 0) w.list[base + __popc(m & below)] = key;
        base += __popc(m);
    }
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int t = n + lane; t < n2; t += 32) w.list[t] = INT_MAX;
    __syncwarp();
    for (int kk = 2; kk <= n2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = lane; t < n2; t += 32) {
                const int l = t ^ jj;
                if (l > t) {
                    const int32_t x = w.list[t], y = w.list[l];
                    if ((x > y) == ((t & kk) == 0)) {
                        w.list[t] = y;
                        w.list[l] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (int p = lane; p < n; p += 32) {
        const int sl = sym_find(w, w.list[p]);
        if (sl >= 0) w.pos[sl] = p;
        w.bound[p] = 0.0;
    }
    __syncwarp();

    // Eq. 3 bounds, summed over k in increasing plan order (a fixed order: the
    // kept set does not depend on the schedule)
    for (int64_t a = a0; a < a1; ++a) {
        const int32_t k = g.a_col[a];
        const double na = g.a_norm[a];
        for (int64_t b = g.b_rowptr[k] + lane; b < g.b_rowptr[k + 1]; b += 32) {
            const int p = sym_slot(w, g.b_col[b]);
            if (p >= 0) w.bound[p] += na * g.b_norm[b];
        }
        __syncwarp();
    }

    // kept candidates (bound >= eps) numbered in increasing j; their values
    const int bi = g.a_rowsize[i];
    int nk = 0;
    int64_t nval = 0;
    for (int p0 = 0; p0 < n; p0 += 32) {
        const int p = p0 + lane;
        const bool keep = p < n && w.bound[p] >= g.eps;
        const unsigned m = __ballot_sync(FULL, keep);
        if (p < n) {
            w.kidx[p] = keep ? nk + __popc(m & below) : -1;
            w.cur[p] = 0;
        }
        if (keep) nval += (int64_t)bi * g.b_colsize[w.list[p]];
        nk += __popc(m);
    }
    nval = warp_sum64(nval);
    __syncwarp();

    // products of every kept candidate
    int64_t nprod = 0;
    for (int64_t a = a0; a < a1; ++a) {
        const int32_t k = g.a_col[a];
        for (int64_t b = g.b_rowptr[k] + lane; b < g.b_rowptr[k + 1]; b += 32) {
            const int p = sym_slot(w, g.b_col[b]);
            if (p >= 0 && w.kidx[p] >= 0) {
                w.cur[p] += 1;
                nprod += 1;
            }
        }
        __syncwarp();
    }
    nprod = warp_sum64(nprod);
    if (PASS == 1) {
        if (lane == 0) {
            g.cnt_out[i] = nk;
            g.cnt_prod[i] = nprod;
            g.cnt_val[i] = nval;
        }
        return true;
    }

    // pass 2: the kept blocks, their value offsets and product ranges
    const int64_t obase = g.off_out[i], pbase = g.off_prod[i], vbase = g.off_val[i];
    int64_t run_p = 0, run_v = 0;
    for (int p0 = 0; p0 < n; p0 += 32) {
        const int p = p0 + lane;
        const bool keep = p < n && w.kidx[p] >= 0;
        const int bj = keep ? g.b_colsize[w.list[p]] : 0;
        const int64_t c = keep ? w.cur[p] : 0, v = keep ? (int64_t)bi * bj : 0;
        const int64_t ic = warp_scan64(c, lane), iv = warp_scan64(v, lane);
        if (keep) {
            const int64_t o = obase + w.kidx[p];
            g.out_col[o] = w.list[p];
            g.out_bi[o] = bi;
            g.out_bj[o] = bj;
            g.out_uoff[o] = vbase + run_v + iv - v;
            g.out_pbeg[o] = pbase + run_p + ic - c;
            w.cur[p] = (int32_t)(run_p + ic - c);   // the block's cursor in the row's product range
        }
        run_p += __shfl_sync(FULL, ic, 31);
        run_v += __shfl_sync(FULL, iv, 31);
    }
    __syncwarp();

    // product lists: inner sizes b_k in increasing order, k in plan order within a size
    int s_prev = 0;
    for (;;) {
        int s_min = INT_MAX;
        for (int64_t a = a0 + lane; a < a1; a += 32) {
            const int sz = g.a_w[a];
            if (sz > s_prev && sz < s_min) s_min = sz;
        }
        for (int m = 16; m > 0; m >>= 1) s_min = min(s_min, __shfl_xor_sync(FULL, s_min, m));
        if (s_min == INT_MAX) break;
        for (int64_t a = a0; a < a1; ++a) {
            if (g.a_w[a] != s_min) continue;
            const int32_t k = g.a_col[a];
            for (int64_t b = g.b_rowptr[k] + lane; b < g.b_rowptr[k + 1]; b += 32) {
                const int p = sym_slot(w, g.b_col[b]);
                if (p >= 0 && w.kidx[p] >= 0) {
                    const int64_t u = pbase + w.cur[p];
                    w.cur[p] += 1;
                    g.pa[u] = g.a_pbase[a];
                    g.kpa[u] = g.a_kp[a];
                    g.pb[u] = g.b_pbase[b];
                    g.kpb[u] = g.b_kp[b];
                    g.bk[u] = s_min;
                }
            }
            __syncwarp();
        }
        s_prev = s_min;
    }
    return true;
}

template <int PASS>
__global__ void __launch_bounds__(128) spgemm_symbolic_kernel(SymArgs g, int warps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t t = (int64_t)blockIdx.x * warps + warp; t < g.n_rows; t += (int64_t)gridDim.x * warps) {
        const int64_t i = g.rows ? g.rows[t] : t;
        if (PASS == 2 && !g.global_ws && g.overflow[i]) continue;   // served by the global-workspace pass
        const SymWs w = g.global_ws ? sym_ws(g.ws + g.ws_off[t], g.ws_h[t], g.ws_cap[t])
                                    : sym_ws(smem_raw + (size_t)warp * sym_ws_bytes(kSymHash, kSymCap), kSymHash,
                                             kSymCap);
        const bool ok = sym_row<PASS>(g, i, w, lane);
        if (PASS == 1 && lane == 0) {
            g.overflow[i] = ok ? 0 : 1;
            if (!ok) g.cnt_out[i] = g.cnt_prod[i] = g.cnt_val[i] = 0;
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_spgemm_symbolic(int pass, const SymArgs &g, cudaStream_t s) {
    if (g.n_rows == 0) return cudaSuccess;
    const int warps = 4;
    const size_t smem = g.global_ws ? 0 : (size_t)warps * sym_ws_bytes(kSymHash, kSymCap);
    const int64_t need = (g.n_rows + warps - 1) / warps;
    const int grid = (int)(need < 8192 ? need : 8192);
    const void *k = pass == 1 ? (const void *)spgemm_symbolic_kernel<1> : (const void *)spgemm_symbolic_kernel<2>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (pass == 1) spgemm_symbolic_kernel<1><<<grid, warps * 32, smem, s>>>(g, warps);
    else spgemm_symbolic_kernel<2><<<grid, warps * 32, smem, s>>>(g, warps);
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
