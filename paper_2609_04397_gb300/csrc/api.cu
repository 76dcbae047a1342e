// C ABI of the library: validation, the planner (shape-class registry,
// shape-grouped value pages, work items), and dispatch of the product kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/vbcsr.h"
#include "internal.cuh"

using namespace vbcsr;

// ---------------------------------------------------------------------------
// status handling

static thread_local std::string g_detail;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_detail = buf;
    return code;
}

static int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(VBCSR_ERR_NO_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(VBCSR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                        \
    do {                                            \
        cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

extern "C" const char *vbcsr_error_string(int status) {
    switch (status) {
        case VBCSR_OK: return "ok";
        case VBCSR_ERR_INVALID_ARG: return "invalid argument";
        case VBCSR_ERR_PATTERN: return "invalid block pattern";
        case VBCSR_ERR_CUDA: return "CUDA error";
        case VBCSR_ERR_NO_MEMORY: return "out of memory";
        case VBCSR_ERR_UNSUPPORTED: return "unsupported request";
        case VBCSR_ERR_DEVICE_CHECK: return "device self-check failed";
        case VBCSR_ERR_ALIAS: return "output aliases an input";
        default: return "unknown status";
    }
}

extern "C" const char *vbcsr_last_error_detail(void) { return g_detail.c_str(); }

// ---------------------------------------------------------------------------
// handle

namespace {

struct Bucket {
    int B;
    int64_t begin, count;   // range in the items array
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct vbcsr_matrix {
    int device = 0;
    int dtype = VBCSR_F64;
    size_t esize = 8;
    int64_t n_brows = 0, n_bcols = 0, n_rows = 0, n_cols = 0, nblk = 0, nnz = 0, panel_elems = 0;
    int32_t n_structs = 1;
    int backend = VBCSR_BACKEND_VBCSR;
    int csr_lanes[2] = {2, 8};      // lanes per row of the scalar kernel: FP64 / FP32-pipe kinds
    int kc_b[kMaxB + 1] = {0};      // column tile per row count (0: from k)
    int warps_b[kMaxB + 1] = {0};   // warps per CTA per row count (0: 4)
    int schedule = VBCSR_SCHED_PERSISTENT;   // or one launch per row count (VBCSR_SCHED_BUCKETED)
    int persist_warps = 0;          // warps per CTA of the persistent launch (0: 4)
    int debug_checks = 0;

    // host copies
    std::vector<int32_t> row_b, col_b;
    std::vector<int64_t> row_off, col_off;
    std::vector<int64_t> uoff;                 // packed-order offset of user block u (nblk + 1)
    std::vector<int32_t> cls_bi, cls_bj;       // shape-class registry
    std::vector<int64_t> cls_count;

    std::vector<Bucket> fwd_buckets, adj_buckets;
    // host copies of the plan, for the symbolic stage of the block product
    std::vector<int64_t> h_rowptr;     // plan blocks of every block row
    std::vector<int32_t> h_pcol;       // block column of every plan block
    std::vector<int32_t> h_ucol;       // block column of every block in the caller's order
    std::vector<int64_t> h_pbase;      // panel element of its (0, 0) entry
    std::vector<int32_t> h_kp;         // panel stride of its row

    // device
    std::vector<DevBuf> bufs;
    void *panel = nullptr;        // values in panels (dtype)
    float *panel32 = nullptr;     // FP32 copy for the mixed modes (FP64 operators), lazily built
    bool panel32_valid = false;
    float *xconv = nullptr;       // FP32 copy of the current X for the mixed modes (grown on demand)
    size_t xconv_elems = 0;
    float2 *paneldf = nullptr;    // (hi, lo) FP32 pairs of the values for the double-FP32 mode
    bool paneldf_valid = false;
    float2 *xdf = nullptr;        // (hi, lo) pairs of the current X for the double-FP32 mode
    size_t xdf_elems = 0;
    uint32_t *panelbf = nullptr;  // values split into packed bf16 (hi, lo) words for the BF16X2 mode
    bool panelbf_valid = false;
    uint32_t *xbf = nullptr;      // the current X split the same way
    size_t xbf_elems = 0;
    uint16_t *panelbp = nullptr;  // the BF16X2 pieces of the values as two bf16 planes (hi, then lo)
    bool panelbp_valid = false;
    uint16_t *xbp = nullptr;      // the current X as two bf16 planes [rows, pipe_ldp(k)] (hi, then lo)
    size_t xbp_elems = 0;
    WorkItem *fwd_items = nullptr, *adj_items = nullptr;   // bucketed by row count
    WorkItem *fwd_lpt = nullptr, *adj_lpt = nullptr;       // all items, descending cost
    int64_t n_fwd_items = 0, n_adj_items = 0;
    long long *queue = nullptr;                            // work counter of the persistent launch
    int32_t *fl_xrow = nullptr, *fl_pcol = nullptr, *fl_w = nullptr, *fl_kp = nullptr, *fl_bi = nullptr;
    int64_t *fl_uoff = nullptr, *fl_pbase = nullptr;
    int64_t *tl_pbase = nullptr;
    int32_t *tl_kp = nullptr, *tl_bi = nullptr, *tl_xrow = nullptr, *tl_vcol = nullptr;
    int64_t *prow_ptr = nullptr, *d_row_off = nullptr;
    int32_t *d_row_b = nullptr;
    double *partials = nullptr;
    double *item_partials = nullptr;   // one dot share per work item (persistent launches)
    double *dot_scratch = nullptr;     // first-stage sums of long fixed-order reductions
    int *err = nullptr;
    int64_t device_bytes = 0;

    // reciprocal-space sampling (handles made by vbcsr_create_kspace)
    bool kspace = false;
    int64_t ks_edges = 0;
    int64_t *ks_ptr = nullptr;       // edges of every union block (nblk + 1), edges sorted by block
    double *ks_shift = nullptr;      // s_e = R [+ tau_j - tau_i] of every sorted edge (3 doubles)
    int64_t *ks_voff = nullptr;      // offset of every sorted edge's real block in ks_vals
    double *ks_vals = nullptr;       // the image blocks, row-major
    int64_t *ks_uoff = nullptr;      // packed offset of every union block
    int32_t *ks_ubn = nullptr;       // entries of every union block
    double2 *ks_phase = nullptr;     // phase of every sorted edge at the current k
    double2 *ks_stage = nullptr;     // packed complex values at the current k

    ~vbcsr_matrix() {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != device) cudaSetDevice(device);
        for (auto &b : bufs)
            if (b.p) cudaFree(b.p);
        if (cur != device) cudaSetDevice(cur);
    }

    template <typename T>
    cudaError_t alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) return e;
        bufs.push_back({q, count * sizeof(T)});
        device_bytes += (int64_t)(count * sizeof(T));
        *p = static_cast<T *>(q);
        return cudaSuccess;
    }
};

template <typename T>
static cudaError_t upload(vbcsr_matrix *A, T **dst, const std::vector<T> &src, cudaStream_t s) {
    cudaError_t e = A->alloc(dst, src.size());
    if (e != cudaSuccess) return e;
    if (src.empty()) return cudaSuccess;
    e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);   // host vectors are freed by the caller afterwards
}

// ---------------------------------------------------------------------------
// validation and planning

static const int32_t kMaxBlockSize = 4096;

static int validate_pattern(int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize,
                            const int32_t *col_bsize, const int64_t *block_row_ptr,
                            const int32_t *block_col_idx) {
    if (n_brows < 0 || n_bcols < 0) return fail(VBCSR_ERR_INVALID_ARG, "negative block count");
    if (n_brows > 0 && !row_bsize) return fail(VBCSR_ERR_INVALID_ARG, "row_bsize is NULL");
    if (n_bcols > 0 && !col_bsize) return fail(VBCSR_ERR_INVALID_ARG, "col_bsize is NULL");
    if (!block_row_ptr) return fail(VBCSR_ERR_INVALID_ARG, "block_row_ptr is NULL");
    int64_t rows = 0, cols = 0;
    for (int64_t i = 0; i < n_brows; ++i) {
        if (row_bsize[i] < 1 || row_bsize[i] > kMaxBlockSize)
            return fail(VBCSR_ERR_PATTERN, "row_bsize[%lld] = %d outside [1, %d]", (long long)i, row_bsize[i],
                        kMaxBlockSize);
        rows += row_bsize[i];
    }
    for (int64_t j = 0; j < n_bcols; ++j) {
        if (col_bsize[j] < 1 || col_bsize[j] > kMaxBlockSize)
            return fail(VBCSR_ERR_PATTERN, "col_bsize[%lld] = %d outside [1, %d]", (long long)j, col_bsize[j],
                        kMaxBlockSize);
        cols += col_bsize[j];
    }
    if (rows >= (1LL << 31) || cols >= (1LL << 31))
        return fail(VBCSR_ERR_PATTERN, "scalar size %lld x %lld reaches 2^31", (long long)rows, (long long)cols);
    if (block_row_ptr[0] != 0) return fail(VBCSR_ERR_PATTERN, "block_row_ptr[0] = %lld, expected 0",
                                           (long long)block_row_ptr[0]);
    for (int64_t i = 0; i < n_brows; ++i)
        if (block_row_ptr[i + 1] < block_row_ptr[i])
            return fail(VBCSR_ERR_PATTERN, "block_row_ptr decreases at row %lld", (long long)i);
    const int64_t nblk = block_row_ptr[n_brows];
    if (nblk > 0 && !block_col_idx) return fail(VBCSR_ERR_INVALID_ARG, "block_col_idx is NULL");
    if (nblk >= (1LL << 31)) return fail(VBCSR_ERR_PATTERN, "%lld blocks reach 2^31", (long long)nblk);
    std::vector<int32_t> tmp;
    for (int64_t i = 0; i < n_brows; ++i) {
        bool increasing = true;   // strictly increasing columns: in range and free of duplicates
        for (int64_t u = block_row_ptr[i]; u < block_row_ptr[i + 1]; ++u) {
            const int32_t c = block_col_idx[u];
            if (c < 0 || c >= n_bcols)
                return fail(VBCSR_ERR_PATTERN, "column %d of block row %lld outside [0, %lld)", c, (long long)i,
                            (long long)n_bcols);
            if (u > block_row_ptr[i] && c <= block_col_idx[u - 1]) increasing = false;
        }
        if (increasing) continue;
        tmp.assign(block_col_idx + block_row_ptr[i], block_col_idx + block_row_ptr[i + 1]);
        std::sort(tmp.begin(), tmp.end());
        for (size_t e = 1; e < tmp.size(); ++e)
            if (tmp[e] == tmp[e - 1])
                return fail(VBCSR_ERR_PATTERN, "duplicate block (%lld, %d)", (long long)i, tmp[e]);
    }
    return VBCSR_OK;
}

static int ceil_to(int64_t v, int m) { return (int)((v + m - 1) / m * m); }

// f(begin, end) over [0, n) split into contiguous ranges on up to 16 host
// threads (one thread below `grain` items per thread); f must only write what
// its own range owns
template <typename F>
static void host_parallel(int64_t n, int64_t grain, F f) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int64_t nt = std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 16, n / grain}));
    if (nt == 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> pool;
    for (int64_t t = 1; t < nt; ++t) pool.emplace_back([&, t]() { f(n * t / nt, n * (t + 1) / nt); });
    f((int64_t)0, n / nt);
    for (auto &th : pool) th.join();
}

// Longest-processing-time order for the persistent launch: the costliest
// items (rows x virtual columns) first, so that the queue ends with small ones.
// Descending-cost order of the persistent launches. Costs are compared in
// classes about 19 % wide (a quarter of a binary order of magnitude), and
// items of one class keep page order: the expensive items still come first,
// so the last items the warps take are the cheap ones, while warps that take
// consecutive items work on neighbouring block rows, whose X rows they share
// through the caches (exact-cost order interleaves the block rows of every
// structure of a batched operator).
static int cost_class(const WorkItem &w) {
    const double c = (double)w.B * (double)(w.K + 8);
    return (int)std::floor(4.0 * std::log2(c));
}

static void sort_by_cost(std::vector<WorkItem> &items) {
    std::stable_sort(items.begin(), items.end(),
                     [](const WorkItem &x, const WorkItem &y) { return cost_class(x) > cost_class(y); });
}

static int build(vbcsr_matrix *A, int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize,
                 const int32_t *col_bsize, const int64_t *block_row_ptr, const int32_t *block_col_idx,
                 const void *values, int values_on_device, cudaStream_t s) {
    A->n_brows = n_brows;
    A->n_bcols = n_bcols;
    A->row_b.assign(row_bsize, row_bsize + n_brows);
    A->col_b.assign(col_bsize, col_bsize + n_bcols);
    A->row_off.assign(n_brows + 1, 0);
    A->col_off.assign(n_bcols + 1, 0);
    for (int64_t i = 0; i < n_brows; ++i) A->row_off[i + 1] = A->row_off[i] + row_bsize[i];
    for (int64_t j = 0; j < n_bcols; ++j) A->col_off[j + 1] = A->col_off[j] + col_bsize[j];
    A->n_rows = A->row_off[n_brows];
    A->n_cols = A->col_off[n_bcols];
    const int64_t nblk = block_row_ptr[n_brows];
    A->nblk = nblk;

    // packed-order offsets
    A->uoff.assign(nblk + 1, 0);
    for (int64_t i = 0; i < n_brows; ++i)
        for (int64_t u = block_row_ptr[i]; u < block_row_ptr[i + 1]; ++u)
            A->uoff[u + 1] = A->uoff[u] + (int64_t)row_bsize[i] * col_bsize[block_col_idx[u]];
    A->nnz = A->uoff[nblk];

    // backend (Sec. II.B): scalar, uniform-block or variable-block
    {
        bool scalar = true, uniform = n_brows > 0 || n_bcols > 0;
        const int32_t b0 = n_brows > 0 ? row_bsize[0] : (n_bcols > 0 ? col_bsize[0] : 1);
        for (int64_t i = 0; i < n_brows; ++i) {
            scalar &= row_bsize[i] == 1;
            uniform &= row_bsize[i] == b0;
        }
        for (int64_t j = 0; j < n_bcols; ++j) {
            scalar &= col_bsize[j] == 1;
            uniform &= col_bsize[j] == b0;
        }
        A->backend = scalar ? VBCSR_BACKEND_CSR : (uniform ? VBCSR_BACKEND_BSR : VBCSR_BACKEND_VBCSR);
        if (scalar) {
            // FP64 operations are charged per warp instruction on GB300's narrow FP64
            // pipe, so an FP64 (or double-FP32) row gets few lanes (every instruction
            // carries ~32 useful lanes, the finishing butterfly is short); FP32 rows
            // get a few more. Measured on a 43.6M-entry scalar graph (26.5 entries per
            // row): 4 lanes per FP32 row ran FP32 / BF16X2 products 2.3x / 1.7x
            // faster (k = 1 / 16) than 16 lanes
            const double avg = n_brows > 0 ? (double)nblk / (double)n_brows : 0.0;
            A->csr_lanes[0] = avg <= 64 ? 2 : (avg <= 256 ? 4 : 8);
            A->csr_lanes[1] = avg <= 32 ? 4 : (avg <= 128 ? 8 : (avg <= 512 ? 16 : 32));
        }
    }

    // shape-class registry (Sec. III.B): every distinct (b_i, b_j), in increasing
    // (b_i, b_j) order. Block sizes are at most kMaxBlockSize, so the counts go
    // to a dense table over the distinct row and column sizes (one pass over the
    // blocks); an ordered map serves the rare pattern with very many sizes.
    {
        std::vector<int32_t> ridx(kMaxBlockSize + 1, -1), cidx(kMaxBlockSize + 1, -1);
        std::vector<int32_t> rs, cs;
        for (int64_t i = 0; i < n_brows; ++i)
            if (ridx[row_bsize[i]] < 0) { ridx[row_bsize[i]] = 0; rs.push_back(row_bsize[i]); }
        for (int64_t j = 0; j < n_bcols; ++j)
            if (cidx[col_bsize[j]] < 0) { cidx[col_bsize[j]] = 0; cs.push_back(col_bsize[j]); }
        std::sort(rs.begin(), rs.end());
        std::sort(cs.begin(), cs.end());
        for (size_t t = 0; t < rs.size(); ++t) ridx[rs[t]] = (int32_t)t;
        for (size_t t = 0; t < cs.size(); ++t) cidx[cs[t]] = (int32_t)t;
        if (rs.size() * cs.size() <= ((size_t)1 << 20)) {
            std::vector<int64_t> cnt(rs.size() * cs.size(), 0);
            for (int64_t i = 0; i < n_brows; ++i) {
                int64_t *row = cnt.data() + (size_t)ridx[row_bsize[i]] * cs.size();
                for (int64_t u = block_row_ptr[i]; u < block_row_ptr[i + 1]; ++u)
                    row[cidx[col_bsize[block_col_idx[u]]]] += 1;
            }
            for (size_t r = 0; r < rs.size(); ++r)
                for (size_t c = 0; c < cs.size(); ++c)
                    if (cnt[r * cs.size() + c]) {
                        A->cls_bi.push_back(rs[r]);
                        A->cls_bj.push_back(cs[c]);
                        A->cls_count.push_back(cnt[r * cs.size() + c]);
                    }
        } else {
            std::map<std::pair<int32_t, int32_t>, int64_t> reg;
            for (int64_t i = 0; i < n_brows; ++i)
                for (int64_t u = block_row_ptr[i]; u < block_row_ptr[i + 1]; ++u)
                    reg[{row_bsize[i], col_bsize[block_col_idx[u]]}] += 1;
            for (auto &kv : reg) {
                A->cls_bi.push_back(kv.first.first);
                A->cls_bj.push_back(kv.first.second);
                A->cls_count.push_back(kv.second);
            }
        }
    }

    // plan order: blocks of every row sorted by column (rows given sorted keep
    // their order without a sort)
    std::vector<int32_t> perm(nblk);   // plan block -> user block
    for (int64_t i = 0; i < n_brows; ++i) {
        const int64_t b0 = block_row_ptr[i], b1 = block_row_ptr[i + 1];
        bool sorted = true;
        for (int64_t u = b0; u < b1; ++u) {
            perm[u] = (int32_t)u;
            if (u > b0 && block_col_idx[u] < block_col_idx[u - 1]) sorted = false;
        }
        if (!sorted)
            std::sort(perm.begin() + b0, perm.begin() + b1,
                      [&](int32_t x, int32_t y) { return block_col_idx[x] < block_col_idx[y]; });
    }

    // panel widths; pages ordered by row height
    // (scalar rows are short - ~27 entries in an atom-like graph - so padding them to
    // 8 would add ~20 % to their values; 4 keeps every row start 16-byte aligned, all
    // that the FP32 vector loads and the bulk copies need)
    std::vector<int64_t> K(n_brows, 0), Kp(n_brows, 0), poff(n_brows, 0);
    const int pad = A->backend == VBCSR_BACKEND_CSR ? kPadKScalar : kPadK;
    for (int64_t i = 0; i < n_brows; ++i) {
        int64_t w = 0;
        for (int64_t u = block_row_ptr[i]; u < block_row_ptr[i + 1]; ++u) w += col_bsize[block_col_idx[u]];
        if (w >= (1LL << 31) - kPadK) return fail(VBCSR_ERR_PATTERN, "block row %lld too wide", (long long)i);
        K[i] = w;
        Kp[i] = ceil_to(w, pad);
    }
    std::vector<int64_t> page_order(n_brows);
    for (int64_t i = 0; i < n_brows; ++i) page_order[i] = i;
    std::stable_sort(page_order.begin(), page_order.end(),
                     [&](int64_t x, int64_t y) { return row_bsize[x] < row_bsize[y]; });
    int64_t pos = 0;
    for (int64_t i : page_order) {
        poff[i] = pos;
        pos += (int64_t)row_bsize[i] * Kp[i];
    }
    A->panel_elems = pos;

    // plan block list
    std::vector<int32_t> fl_xrow(nblk), fl_pcol(nblk), fl_w(nblk), fl_kp(nblk), fl_bi(nblk);
    std::vector<int64_t> fl_uoff(nblk), fl_pbase(nblk), prow_ptr(block_row_ptr, block_row_ptr + n_brows + 1);
    host_parallel(n_brows, 4096, [&](int64_t i0, int64_t i1) {   // block rows own their list ranges
        for (int64_t i = i0; i < i1; ++i) {
            int64_t pc = 0;
            for (int64_t l = block_row_ptr[i]; l < block_row_ptr[i + 1]; ++l) {
                const int32_t u = perm[l];
                const int32_t j = block_col_idx[u];
                fl_xrow[l] = (int32_t)A->col_off[j];
                fl_pcol[l] = (int32_t)pc;
                fl_w[l] = col_bsize[j];
                fl_kp[l] = (int32_t)Kp[i];
                fl_bi[l] = row_bsize[i];
                fl_uoff[l] = A->uoff[u];
                fl_pbase[l] = poff[i] + pc;
                pc += col_bsize[j];
            }
        }
    });

    // forward work items, bucketed by row count
    {
        std::vector<std::vector<WorkItem>> bk(kMaxB + 1);
        for (int64_t i : page_order) {
            // a row taller than kMaxB is cut into ceil(b / kMaxB) near-equal chunks
            const int32_t nch = (row_bsize[i] + kMaxB - 1) / kMaxB;
            for (int32_t c = 0, r0 = 0; c < nch; ++c) {
                WorkItem w;
                w.B = row_bsize[i] / nch + (c < row_bsize[i] % nch ? 1 : 0);
                w.vbase = poff[i] + (int64_t)r0 * Kp[i];
                w.yrow = A->row_off[i] + r0;
                w.lbegin = block_row_ptr[i];
                w.nlist = (int32_t)(block_row_ptr[i + 1] - block_row_ptr[i]);
                w.K = (int32_t)K[i];
                w.Kp = (int32_t)Kp[i];
                bk[w.B].push_back(w);
                r0 += w.B;
            }
        }
        std::vector<WorkItem> items;
        for (int b = 1; b <= kMaxB; ++b) {
            if (bk[b].empty()) continue;
            A->fwd_buckets.push_back({b, (int64_t)items.size(), (int64_t)bk[b].size()});
            items.insert(items.end(), bk[b].begin(), bk[b].end());
        }
        CUDA_TRY(upload(A, &A->fwd_items, items, s), "upload forward items");
        A->n_fwd_items = (int64_t)items.size();
        sort_by_cost(items);
        CUDA_TRY(upload(A, &A->fwd_lpt, items, s), "upload forward items");
    }

    // transposed list and adjoint work items
    {
        std::vector<int64_t> tptr(n_bcols + 1, 0);
        for (int64_t l = 0; l < nblk; ++l) tptr[block_col_idx[perm[l]] + 1] += 1;
        for (int64_t j = 0; j < n_bcols; ++j) tptr[j + 1] += tptr[j];
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        std::vector<int64_t> tl_pbase(nblk);
        std::vector<int32_t> tl_kp(nblk), tl_bi(nblk), tl_xrow(nblk), tl_vcol(nblk);
        // rows increasing inside each column: every thread walks all blocks in row
        // order and places those of its own range of columns
        host_parallel(n_bcols, 4096, [&](int64_t j0, int64_t j1) {
            for (int64_t i = 0; i < n_brows; ++i) {
                for (int64_t l = block_row_ptr[i]; l < block_row_ptr[i + 1]; ++l) {
                    const int32_t j = block_col_idx[perm[l]];
                    if (j < j0 || j >= j1) continue;
                    const int64_t e = fill[j]++;
                    tl_pbase[e] = fl_pbase[l];
                    tl_kp[e] = (int32_t)Kp[i];
                    tl_bi[e] = row_bsize[i];
                    tl_xrow[e] = (int32_t)A->row_off[i];
                }
            }
        });
        std::vector<int64_t> Kt(n_bcols, 0);
        for (int64_t j = 0; j < n_bcols; ++j) {
            int64_t v = 0;
            for (int64_t e = tptr[j]; e < tptr[j + 1]; ++e) {
                tl_vcol[e] = (int32_t)v;
                v += tl_bi[e];
            }
            if (v >= (1LL << 31)) return fail(VBCSR_ERR_PATTERN, "block column %lld too tall", (long long)j);
            Kt[j] = v;
        }
        std::vector<int64_t> col_order(n_bcols);
        for (int64_t j = 0; j < n_bcols; ++j) col_order[j] = j;
        std::stable_sort(col_order.begin(), col_order.end(),
                         [&](int64_t x, int64_t y) { return col_bsize[x] < col_bsize[y]; });
        std::vector<std::vector<WorkItem>> bk(kMaxB + 1);
        for (int64_t j : col_order) {
            const int32_t nch = (col_bsize[j] + kMaxB - 1) / kMaxB;
            for (int32_t c = 0, q0 = 0; c < nch; ++c) {
                WorkItem w;
                w.B = col_bsize[j] / nch + (c < col_bsize[j] % nch ? 1 : 0);
                w.vbase = 0;
                w.yrow = A->col_off[j] + q0;
                w.lbegin = tptr[j];
                w.nlist = (int32_t)(tptr[j + 1] - tptr[j]);
                w.K = (int32_t)Kt[j];
                w.Kp = q0;
                bk[w.B].push_back(w);
                q0 += w.B;
            }
        }
        std::vector<WorkItem> items;
        for (int b = 1; b <= kMaxB; ++b) {
            if (bk[b].empty()) continue;
            A->adj_buckets.push_back({b, (int64_t)items.size(), (int64_t)bk[b].size()});
            items.insert(items.end(), bk[b].begin(), bk[b].end());
        }
        CUDA_TRY(upload(A, &A->adj_items, items, s), "upload adjoint items");
        A->n_adj_items = (int64_t)items.size();
        sort_by_cost(items);
        CUDA_TRY(upload(A, &A->adj_lpt, items, s), "upload adjoint items");
        CUDA_TRY(upload(A, &A->tl_pbase, tl_pbase, s), "upload");
        CUDA_TRY(upload(A, &A->tl_kp, tl_kp, s), "upload");
        CUDA_TRY(upload(A, &A->tl_bi, tl_bi, s), "upload");
        CUDA_TRY(upload(A, &A->tl_xrow, tl_xrow, s), "upload");
        CUDA_TRY(upload(A, &A->tl_vcol, tl_vcol, s), "upload");
    }
    CUDA_TRY(A->alloc(&A->item_partials, (size_t)std::max(A->n_fwd_items, A->n_adj_items)),
             "alloc per-item dot shares");

    A->h_rowptr = prow_ptr;
    A->h_ucol.assign(block_col_idx, block_col_idx + nblk);
    A->h_pcol.resize(nblk);
    for (int64_t l = 0; l < nblk; ++l) A->h_pcol[l] = block_col_idx[perm[l]];
    A->h_pbase = fl_pbase;
    A->h_kp = fl_kp;
    CUDA_TRY(upload(A, &A->fl_xrow, fl_xrow, s), "upload");
    CUDA_TRY(upload(A, &A->fl_pcol, fl_pcol, s), "upload");
    CUDA_TRY(upload(A, &A->fl_w, fl_w, s), "upload");
    CUDA_TRY(upload(A, &A->fl_kp, fl_kp, s), "upload");
    CUDA_TRY(upload(A, &A->fl_bi, fl_bi, s), "upload");
    CUDA_TRY(upload(A, &A->fl_uoff, fl_uoff, s), "upload");
    CUDA_TRY(upload(A, &A->fl_pbase, fl_pbase, s), "upload");
    CUDA_TRY(upload(A, &A->prow_ptr, prow_ptr, s), "upload");
    CUDA_TRY(upload(A, &A->d_row_off, A->row_off, s), "upload");
    CUDA_TRY(upload(A, &A->d_row_b, A->row_b, s), "upload");
    CUDA_TRY(A->alloc(&A->partials, kPartialsCap), "alloc partials");
    CUDA_TRY(A->alloc(&A->dot_scratch, (size_t)kDotScratch), "alloc partials");
    CUDA_TRY(A->alloc(&A->err, 1), "alloc error word");
    CUDA_TRY(A->alloc(&A->queue, 1), "alloc work counter");
    CUDA_TRY(cudaMemsetAsync(A->err, 0, sizeof(int), s), "memset");

    // value pages
    unsigned char *panel = nullptr;
    // two elements of slack after the pages: the adjoint reads 8-byte values in aligned pairs
    CUDA_TRY(A->alloc(&panel, (size_t)(A->panel_elems + 2) * A->esize), "alloc value pages");
    A->panel = panel;
    CUDA_TRY(cudaMemsetAsync(A->panel, 0, (size_t)(A->panel_elems + 2) * A->esize, s), "memset");
    if (A->nnz > 0 && values) {
        const void *src = values;
        void *staged = nullptr;
        if (!values_on_device) {
            CUDA_TRY(cudaMalloc(&staged, (size_t)A->nnz * A->esize), "alloc staging");
            cudaError_t e = cudaMemcpyAsync(staged, values, (size_t)A->nnz * A->esize, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) { cudaFree(staged); return cuda_fail(e, "copy values"); }
            src = staged;
        }
        cudaError_t e = launch_permute_values((int)A->esize, true, nblk, A->fl_uoff, A->fl_pbase,
                                              A->fl_kp, A->fl_bi, A->fl_w, src, A->panel, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (staged) cudaFree(staged);
        if (e != cudaSuccess) return cuda_fail(e, "scatter values");
        if (e2 != cudaSuccess) return cuda_fail(e2, "scatter values");
    }
    CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
    return VBCSR_OK;
}

// zero_values: values may be NULL and the pages start at zero (k-space handles)
static int create_common(vbcsr_t **out, int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize,
                         const int32_t *col_bsize, const int64_t *block_row_ptr, const int32_t *block_col_idx,
                         const void *values, int dtype, int values_on_device, void *stream, int32_t n_structs,
                         bool zero_values = false) {
    if (!out) return fail(VBCSR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dtype != VBCSR_F64 && dtype != VBCSR_F32 && dtype != VBCSR_C128)
        return fail(VBCSR_ERR_INVALID_ARG, "dtype %d", dtype);
    if (values_on_device != 0 && values_on_device != 1)
        return fail(VBCSR_ERR_INVALID_ARG, "values_on_device must be 0 or 1");
    int rc = validate_pattern(n_brows, n_bcols, row_bsize, col_bsize, block_row_ptr, block_col_idx);
    if (rc) return rc;
    if (!values && block_row_ptr[n_brows] > 0 && !zero_values) return fail(VBCSR_ERR_INVALID_ARG, "values is NULL");
    vbcsr_matrix *A = new (std::nothrow) vbcsr_matrix();
    if (!A) return fail(VBCSR_ERR_NO_MEMORY, "host allocation");
    cudaError_t e = cudaGetDevice(&A->device);
    if (e != cudaSuccess) { delete A; return cuda_fail(e, "cudaGetDevice"); }
    A->dtype = dtype;
    A->esize = dtype == VBCSR_C128 ? 16 : (dtype == VBCSR_F64 ? 8 : 4);
    A->n_structs = n_structs;
    const char *dbg = getenv("VBCSR_DEBUG_CHECKS");
    A->debug_checks = (dbg && dbg[0] && dbg[0] != '0') ? 1 : 0;
    try {
        rc = build(A, n_brows, n_bcols, row_bsize, col_bsize, block_row_ptr, block_col_idx, values,
                   values_on_device, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        rc = fail(VBCSR_ERR_NO_MEMORY, "host allocation in planner");
    }
    if (rc) { delete A; return rc; }
    *out = A;
    return VBCSR_OK;
}

extern "C" int vbcsr_create(vbcsr_t **out, int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize,
                            const int32_t *col_bsize, const int64_t *block_row_ptr, const int32_t *block_col_idx,
                            const void *values, int dtype, int values_on_device, void *stream) {
    return create_common(out, n_brows, n_bcols, row_bsize, col_bsize, block_row_ptr, block_col_idx, values, dtype,
                         values_on_device, stream, 1);
}

extern "C" int vbcsr_create_batched(vbcsr_t **out, int64_t n_structs, const int64_t *sbo, const int64_t *sco,
                                    const int32_t *row_bsize, const int32_t *col_bsize,
                                    const int64_t *block_row_ptr, const int32_t *block_col_idx,
                                    const void *values, int dtype, int values_on_device, void *stream) {
    if (!out) return fail(VBCSR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_structs < 1 || n_structs >= (1LL << 31)) return fail(VBCSR_ERR_INVALID_ARG, "n_structs %lld", (long long)n_structs);
    if (!sbo || !sco || !block_row_ptr) return fail(VBCSR_ERR_INVALID_ARG, "offset array is NULL");
    if (sbo[0] != 0 || sco[0] != 0) return fail(VBCSR_ERR_PATTERN, "structure offsets must start at 0");
    for (int64_t s = 0; s < n_structs; ++s)
        if (sbo[s + 1] < sbo[s] || sco[s + 1] < sco[s])
            return fail(VBCSR_ERR_PATTERN, "structure offsets decrease at %lld", (long long)s);
    const int64_t n_brows = sbo[n_structs], n_bcols = sco[n_structs];
    if (n_brows < 0 || n_bcols < 0) return fail(VBCSR_ERR_INVALID_ARG, "negative size");
    if (block_row_ptr[0] != 0) return fail(VBCSR_ERR_PATTERN, "block_row_ptr[0] must be 0");
    for (int64_t i = 0; i < n_brows; ++i)
        if (block_row_ptr[i + 1] < block_row_ptr[i]) return fail(VBCSR_ERR_PATTERN, "block_row_ptr decreases");
    const int64_t nblk = block_row_ptr[n_brows];
    if (nblk > 0 && !block_col_idx) return fail(VBCSR_ERR_INVALID_ARG, "block_col_idx is NULL");
    std::vector<int32_t> gcol;
    try {
        gcol.resize(nblk);
    } catch (const std::bad_alloc &) {
        return fail(VBCSR_ERR_NO_MEMORY, "host allocation");
    }
    for (int64_t s = 0; s < n_structs; ++s) {
        const int64_t ncol_s = sco[s + 1] - sco[s];
        for (int64_t i = sbo[s]; i < sbo[s + 1]; ++i)
            for (int64_t u = block_row_ptr[i]; u < block_row_ptr[i + 1]; ++u) {
                const int32_t c = block_col_idx[u];
                if (c < 0 || c >= ncol_s)
                    return fail(VBCSR_ERR_PATTERN, "local column %d of block row %lld outside structure %lld", c,
                                (long long)i, (long long)s);
                gcol[u] = (int32_t)(c + sco[s]);
            }
    }
    return create_common(out, n_brows, n_bcols, row_bsize, col_bsize, block_row_ptr, gcol.data(), values, dtype,
                         values_on_device, stream, (int32_t)n_structs);
}

// ---------------------------------------------------------------------------
// reciprocal-space sampling of a periodic operator (Eq. 4)

extern "C" int vbcsr_create_kspace(vbcsr_t **out, int64_t n_atoms, const int32_t *bsize, int64_t n_edges,
                                   const int32_t *edge_i, const int32_t *edge_j, const int32_t *edge_R,
                                   const double *edge_values, const double *tau, void *stream) {
    if (!out) return fail(VBCSR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_atoms < 0 || n_edges < 0) return fail(VBCSR_ERR_INVALID_ARG, "negative size");
    if (n_atoms > 0 && !bsize) return fail(VBCSR_ERR_INVALID_ARG, "bsize is NULL");
    if (n_edges > 0 && (!edge_i || !edge_j || !edge_R || !edge_values))
        return fail(VBCSR_ERR_INVALID_ARG, "edge array is NULL");
    if (n_atoms >= (1LL << 31) || n_edges >= (1LL << 31)) return fail(VBCSR_ERR_INVALID_ARG, "size reaches 2^31");
    for (int64_t a = 0; a < n_atoms; ++a)
        if (bsize[a] < 1 || bsize[a] > kMaxBlockSize)
            return fail(VBCSR_ERR_PATTERN, "bsize[%lld] = %d outside [1, %d]", (long long)a, bsize[a], kMaxBlockSize);
    cudaStream_t s = (cudaStream_t)stream;
    try {
        // edges sorted by (i, j), stable: the union pattern and each union block's edges
        std::vector<int64_t> order(n_edges), evoff(n_edges + 1, 0);
        for (int64_t e = 0; e < n_edges; ++e) {
            if (edge_i[e] < 0 || edge_i[e] >= n_atoms || edge_j[e] < 0 || edge_j[e] >= n_atoms)
                return fail(VBCSR_ERR_PATTERN, "edge %lld joins atoms outside [0, %lld)", (long long)e,
                            (long long)n_atoms);
            order[e] = e;
            evoff[e + 1] = evoff[e] + (int64_t)bsize[edge_i[e]] * bsize[edge_j[e]];
        }
        std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
            return edge_i[x] != edge_i[y] ? edge_i[x] < edge_i[y] : edge_j[x] < edge_j[y];
        });
        std::vector<int64_t> rowptr(n_atoms + 1, 0), ks_ptr(1, 0), ks_voff(n_edges);
        std::vector<int32_t> cols, ubn;
        std::vector<double> shift(3 * (size_t)n_edges);
        for (int64_t t = 0; t < n_edges; ++t) {
            const int64_t e = order[t];
            const int32_t i = edge_i[e], j = edge_j[e];
            const bool fresh = t == 0 || edge_i[order[t - 1]] != i || edge_j[order[t - 1]] != j;
            if (fresh) {
                cols.push_back(j);
                ubn.push_back(bsize[i] * bsize[j]);
                rowptr[i + 1] += 1;
                if (t > 0) ks_ptr.push_back(t);
            }
            ks_voff[t] = evoff[e];
            for (int d = 0; d < 3; ++d)
                shift[3 * t + d] = (double)edge_R[3 * e + d] + (tau ? tau[3 * (int64_t)j + d] - tau[3 * (int64_t)i + d] : 0.0);
        }
        if (n_edges > 0) ks_ptr.push_back(n_edges);
        for (int64_t a = 0; a < n_atoms; ++a) rowptr[a + 1] += rowptr[a];
        const int64_t nblk = (int64_t)cols.size();
        int rc = create_common(out, n_atoms, n_atoms, bsize, bsize, rowptr.data(), cols.data(), nullptr, VBCSR_C128,
                               0, stream, 1, true);
        if (rc) return rc;
        vbcsr_matrix *A = *out;
        auto bail = [&](int code) {
            delete A;
            *out = nullptr;
            return code;
        };
        A->kspace = true;
        A->ks_edges = n_edges;
        std::vector<int64_t> uo(A->uoff.begin(), A->uoff.begin() + nblk);
        std::vector<double> vals(edge_values, edge_values + evoff[n_edges]);
        cudaError_t e = upload(A, &A->ks_ptr, ks_ptr, s);
        if (e == cudaSuccess) e = upload(A, &A->ks_shift, shift, s);
        if (e == cudaSuccess) e = upload(A, &A->ks_voff, ks_voff, s);
        if (e == cudaSuccess) e = upload(A, &A->ks_vals, vals, s);
        if (e == cudaSuccess) e = upload(A, &A->ks_uoff, uo, s);
        if (e == cudaSuccess) e = upload(A, &A->ks_ubn, ubn, s);
        if (e == cudaSuccess) e = A->alloc(&A->ks_phase, (size_t)n_edges);
        if (e == cudaSuccess) e = A->alloc(&A->ks_stage, (size_t)A->nnz);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "upload the lattice images"));
    } catch (const std::bad_alloc &) {
        if (*out) {
            delete *out;
            *out = nullptr;
        }
        return fail(VBCSR_ERR_NO_MEMORY, "host allocation");
    }
    return VBCSR_OK;
}

extern "C" int vbcsr_set_kpoint(vbcsr_t *A, const double *kfrac, void *stream) {
    if (!A || !kfrac) return fail(VBCSR_ERR_INVALID_ARG, "NULL argument");
    if (!A->kspace) return fail(VBCSR_ERR_INVALID_ARG, "not a handle made by vbcsr_create_kspace");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(launch_ksample(A->nblk, A->ks_edges, A->ks_ptr, A->ks_shift, A->ks_voff, A->ks_vals, A->ks_uoff,
                            A->ks_ubn, kfrac, A->ks_phase, A->ks_stage, s),
             "k-space sampling");
    CUDA_TRY(launch_permute_values((int)A->esize, true, A->nblk, A->fl_uoff, A->fl_pbase, A->fl_kp, A->fl_bi,
                                   A->fl_w, A->ks_stage, A->panel, s),
             "scatter values");
    return VBCSR_OK;
}

extern "C" int vbcsr_destroy(vbcsr_t *A) {
    delete A;
    return VBCSR_OK;
}

// ---------------------------------------------------------------------------
// values

static int refresh_panelbf(vbcsr_t *A, cudaStream_t s) {
    if (A->dtype != VBCSR_F64) return VBCSR_OK;
    if (!A->panelbf) CUDA_TRY(A->alloc(&A->panelbf, (size_t)A->panel_elems), "alloc split value copy");
    CUDA_TRY(launch_split_bf16((const double *)A->panel, A->panelbf, A->panel_elems, s), "split values");
    A->panelbf_valid = true;
    return VBCSR_OK;
}

static int refresh_panelbp(vbcsr_t *A, cudaStream_t s) {
    if (A->dtype != VBCSR_F64) return VBCSR_OK;
    if (!A->panelbp) CUDA_TRY(A->alloc(&A->panelbp, 2 * (size_t)A->panel_elems), "alloc bf16 value planes");
    CUDA_TRY(launch_split_bf16_planes((const double *)A->panel, A->panelbp, A->panelbp + A->panel_elems,
                                      A->panel_elems, s),
             "split values");
    A->panelbp_valid = true;
    return VBCSR_OK;
}

static int refresh_panel32(vbcsr_t *A, cudaStream_t s) {
    if (A->dtype != VBCSR_F64) return VBCSR_OK;
    if (!A->panel32) CUDA_TRY(A->alloc(&A->panel32, (size_t)A->panel_elems), "alloc FP32 value copy");
    CUDA_TRY(launch_convert_f64_to_f32((const double *)A->panel, A->panel32, A->panel_elems, s), "convert");
    A->panel32_valid = true;
    return VBCSR_OK;
}

static int refresh_paneldf(vbcsr_t *A, cudaStream_t s) {
    if (!A->paneldf) CUDA_TRY(A->alloc(&A->paneldf, (size_t)A->panel_elems + 2), "alloc double-FP32 value copy");
    CUDA_TRY(launch_split_df(A->panel_elems, 1, (const double *)A->panel, 1, A->paneldf, s), "split values");
    A->paneldf_valid = true;
    return VBCSR_OK;
}

// Grow a handle-owned scratch buffer to at least `need` elements.
template <typename T>
static int grow(vbcsr_t *A, T **buf, size_t *have, size_t need, cudaStream_t s, const char *what) {
    if (need <= *have) return VBCSR_OK;
    if (*buf) {
        CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        for (auto &b : A->bufs)
            if (b.p == (void *)*buf) {
                cudaFree(b.p);
                A->device_bytes -= (int64_t)b.bytes;
                b.p = nullptr;
            }
        *buf = nullptr;
        *have = 0;
    }
    CUDA_TRY(A->alloc(buf, need), what);
    *have = need;
    return VBCSR_OK;
}

extern "C" int vbcsr_set_values(vbcsr_t *A, const void *values, int on_device, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (on_device != 0 && on_device != 1) return fail(VBCSR_ERR_INVALID_ARG, "on_device must be 0 or 1");
    if (A->nnz == 0) return VBCSR_OK;
    if (!values) return fail(VBCSR_ERR_INVALID_ARG, "values is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const void *src = values;
    void *staged = nullptr;
    if (!on_device) {
        CUDA_TRY(cudaMalloc(&staged, (size_t)A->nnz * A->esize), "alloc staging");
        cudaError_t e = cudaMemcpyAsync(staged, values, (size_t)A->nnz * A->esize, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { cudaFree(staged); return cuda_fail(e, "copy values"); }
        src = staged;
    }
    cudaError_t e = launch_permute_values((int)A->esize, true, A->nblk, A->fl_uoff, A->fl_pbase, A->fl_kp,
                                          A->fl_bi, A->fl_w, src, A->panel, s);
    if (staged) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(staged);
        if (e2 != cudaSuccess) return cuda_fail(e2, "set_values");
    }
    if (e != cudaSuccess) return cuda_fail(e, "set_values");
    if (A->panel32) {
        int rc = refresh_panel32(A, s);
        if (rc) return rc;
    }
    if (A->panelbf) {
        int rc = refresh_panelbf(A, s);
        if (rc) return rc;
    }
    if (A->panelbp) {
        int rc = refresh_panelbp(A, s);
        if (rc) return rc;
    }
    if (A->paneldf) return refresh_paneldf(A, s);
    return VBCSR_OK;
}

extern "C" int vbcsr_get_values(const vbcsr_t *Ac, void *values, int on_device, void *stream) {
    vbcsr_t *A = const_cast<vbcsr_t *>(Ac);
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (on_device != 0 && on_device != 1) return fail(VBCSR_ERR_INVALID_ARG, "on_device must be 0 or 1");
    if (A->nnz == 0) return VBCSR_OK;
    if (!values) return fail(VBCSR_ERR_INVALID_ARG, "values is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    void *dst = values;
    void *staged = nullptr;
    if (!on_device) {
        CUDA_TRY(cudaMalloc(&staged, (size_t)A->nnz * A->esize), "alloc staging");
        dst = staged;
    }
    cudaError_t e = launch_permute_values((int)A->esize, false, A->nblk, A->fl_uoff, A->fl_pbase,
                                          A->fl_kp, A->fl_bi, A->fl_w, dst, A->panel, s);
    if (staged) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(values, staged, (size_t)A->nnz * A->esize, cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(staged);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return cuda_fail(e, "get_values");
    return VBCSR_OK;
}

// ---------------------------------------------------------------------------
// products

namespace vbcsr {
const void *fma_f64_kernel(bool trans, bool persistent, int B);
const void *fma_f32_kernel(bool trans, bool persistent, int B, bool ring);
const void *fma_f32_on_f64_kernel(bool trans, bool persistent, int B, bool ring);
const void *fma_df_kernel(bool trans, bool persistent, int B, bool narrow, bool ring);
const void *mma_kernel_ptr(int mode, bool xdouble, bool trans, bool staged, int64_t k);
}  // namespace vbcsr

// True when the [rows, k] windows of two row-major panels share an element.
// Disjoint column slices of one wider panel (equal leading dimensions) do not.
static bool overlap(const void *a, int64_t rows_a, int64_t lda, const void *b, int64_t rows_b, int64_t ldb,
                    int64_t k, size_t es) {
    if (rows_a == 0 || rows_b == 0) return false;
    const char *a0 = (const char *)a, *a1 = a0 + ((rows_a - 1) * lda + k) * (int64_t)es;
    const char *b0 = (const char *)b, *b1 = b0 + ((rows_b - 1) * ldb + k) * (int64_t)es;
    if (!(a0 < b1 && b0 < a1)) return false;
    if (lda == ldb && lda > 1) {
        const int64_t bytes = (int64_t)(b0 - a0);
        if (bytes % (int64_t)es == 0) {
            const int64_t d = bytes / (int64_t)es;
            const int64_t r = ((d % lda) + lda) % lda;
            if (r >= k && r <= lda - k) return false;
        }
    }
    return true;
}

static int auto_kc(int64_t k) {
    int kc = 1;
    while (kc < k && kc < 32) kc <<= 1;
    return kc;
}

static int cached_cap(const void *kernel, int warps, size_t smem) {
    static std::map<std::pair<const void *, int>, int> cache;
    auto key = std::make_pair(kernel, warps);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int c = max_resident_ctas(kernel, warps * 32, smem);
    if (c > 0) cache[key] = c;
    return c;
}

// Form of X that a product's kernel reads.
// kXF32P: FP32 with rows pipe_ldp(k) elements apart (the pipelined TF32 kernels), kept in
// the buffer of the bf16 planes (the same bytes: 2 x 2 B or 4 B per element)
enum { kXAsGiven = 0, kXF32 = 1, kXSplit = 2, kXPairs = 3, kXPlanes = 4, kXF32P = 5 };

// Which kernel family serves a product, and which mixed-precision copies of
// the values and of X it reads (built on first use by run_product).
struct ModePlan {
    int mode;                 // effective precision code
    bool f64, cplx;
    bool fma;                 // CUDA-core kernels in the operator's or the FP32 / double-FP32 arithmetic
    bool csr_kernel;          // the scalar kernel of a CSR-backend operator
    bool split;               // a tensor-core mode on the CUDA cores (thin products, scalar operators)
    bool presplit;            // BF16X2 on operands split once into packed bf16 (hi, lo) words
    bool pipe;                // BF16X2 on the tensor cores, operands as bf16 planes through shared memory
    bool pipe_tf;             // TF32 / TF32X3 on the tensor cores, FP32 operands through shared memory
    bool need_panel32, need_panelbf, need_paneldf, need_panelbp;
    int xkind;                // kXAsGiven, kXF32, kXSplit, kXPairs, kXPlanes or kXF32P
};

static ModePlan plan_mode(const vbcsr_t *A, bool trans, int64_t k, int precision) {
    ModePlan p;
    p.f64 = A->dtype == VBCSR_F64;
    p.cplx = A->dtype == VBCSR_C128;
    p.mode = precision;
    if (!p.f64 && p.mode == VBCSR_PREC_F32) p.mode = VBCSR_PREC_NATIVE;
    p.fma = (p.mode == VBCSR_PREC_NATIVE || p.mode == VBCSR_PREC_F32 || p.mode == VBCSR_PREC_DF32);
    // a tensor-core mode on a product too thin for an MMA tile (few columns, or the
    // single-row items of a scalar operator) runs its piece products on the CUDA cores
    p.csr_kernel = A->backend == VBCSR_BACKEND_CSR && !trans && !p.cplx && !(A->schedule & VBCSR_SCHED_NO_CSR);
    p.split = !p.fma && p.f64 && !trans && (k <= kSplitFmaMaxK || p.csr_kernel);
    // the BF16X2 forward kernels of an FP64 operator (the plain tensor-core kernel
    // and the CUDA-core form of thin products; the staged kernel splits itself, the
    // scalar kernel reads FP32) read values and X split once into packed bf16
    // (hi, lo) words
    // the forward tensor-core product of the BF16X2 mode runs the pipelined kernel on
    // bf16 planes, except on scalar operators (their panel rows are 16-byte, not
    // 8-element, aligned) and with the staged variant selected
    p.pipe = p.f64 && p.mode == VBCSR_PREC_BF16X2 && !trans && !p.split && !p.csr_kernel &&
             !(A->schedule & VBCSR_SCHED_MMA_STAGED) && A->backend != VBCSR_BACKEND_CSR;
    // the TF32 modes likewise run the pipelined kernel on the FP32 copy of the values, up
    // to 16 columns (at 17-32 its 32-column tiles hold 4 CTAs per SM and the register-load
    // kernel is 3 % faster: 0.58 against 0.60 ms at k = 32 on the 50k-atom operator)
    p.pipe_tf = p.f64 && (p.mode == VBCSR_PREC_TF32 || p.mode == VBCSR_PREC_TF32X3) && !trans && !p.split &&
                k <= 16 && !p.csr_kernel && !(A->schedule & VBCSR_SCHED_MMA_STAGED) &&
                A->backend != VBCSR_BACKEND_CSR;
    p.presplit = p.f64 && p.mode == VBCSR_PREC_BF16X2 && !trans && !p.csr_kernel && !p.pipe &&
                 (p.split || !(A->schedule & VBCSR_SCHED_MMA_STAGED));
    p.need_panel32 =
        p.f64 && p.mode != VBCSR_PREC_NATIVE && p.mode != VBCSR_PREC_DF32 && !p.presplit && !p.pipe;
    p.need_panelbf = p.presplit;
    p.need_panelbp = p.pipe;
    p.need_paneldf = p.mode == VBCSR_PREC_DF32;
    p.xkind = !p.f64 || p.mode == VBCSR_PREC_NATIVE ? kXAsGiven
            : p.mode == VBCSR_PREC_DF32             ? kXPairs
            : p.pipe                                ? kXPlanes
            : p.pipe_tf                             ? kXF32P
            : p.presplit                            ? kXSplit
                                                    : kXF32;
    return p;
}

// True when every mixed-precision copy that a product of `xrows` x k needs is
// already built and large enough, so that run_product allocates nothing.
static bool mode_buffers_ready(const vbcsr_t *A, const ModePlan &p, int64_t xrows, int64_t k) {
    if (p.need_panel32 && !A->panel32_valid) return false;
    if (p.need_panelbf && !A->panelbf_valid) return false;
    if (p.need_paneldf && !A->paneldf_valid) return false;
    if (p.need_panelbp && !A->panelbp_valid) return false;
    const size_t need = (size_t)xrows * (size_t)k;
    switch (p.xkind) {
        case kXF32: return A->xconv_elems >= need;
        case kXSplit: return A->xbf_elems >= need;
        case kXPairs: return A->xdf_elems >= need;
        case kXPlanes:
        case kXF32P: return A->xbp_elems >= 2 * (size_t)xrows * (size_t)pipe_ldp(k);
        default: return true;
    }
}

// Chebyshev steps on the plain tensor-core forward kernel exchange X in
// the kernel's own form: a step reads t_n already converted (x_in, [rows, k],
// leading dimension k) and its epilogue writes t_{n+1} converted as well
// (x_out), so no separate conversion pass runs between steps.
struct FusedX {
    const void *x_in;   // X in the form the kernel reads, or NULL: convert X here
    void *x_out;        // where the epilogue writes the output in that form, or NULL
};

// True when a forward product of this plan runs the plain tensor-core kernel
// on a converted X (FP32, or packed bf16 pieces), i.e. when FusedX applies.
static bool fused_x_applies(const vbcsr_t *A, const ModePlan &p) {
    return !p.fma && !p.split && !p.cplx &&
           (p.xkind == kXF32 || p.xkind == kXSplit || p.xkind == kXPlanes || p.xkind == kXF32P) &&
           !(A->schedule & VBCSR_SCHED_MMA_STAGED);
}

// dot_scale multiplies the fused dot product before it is stored (1 for the
// public epilogue, 1 / (N k) for the Chebyshev moments).
static int run_product(vbcsr_t *A, bool trans, int64_t k, double alpha, const void *X, int64_t ldx, double beta,
                       void *Y, int64_t ldy, const vbcsr_epilogue_t *epi, int precision, cudaStream_t s,
                       double dot_scale = 1.0, const FusedX *fx = nullptr) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (k < 0) return fail(VBCSR_ERR_INVALID_ARG, "k = %lld", (long long)k);
    if (precision < VBCSR_PREC_NATIVE || precision > VBCSR_PREC_DF32)
        return fail(VBCSR_ERR_INVALID_ARG, "precision %d", precision);
    if (precision == VBCSR_PREC_DF32 && A->dtype != VBCSR_F64)
        return fail(VBCSR_ERR_UNSUPPORTED, "the double-FP32 mode needs an FP64 operator");
    const bool cplx = A->dtype == VBCSR_C128;
    if (cplx && precision != VBCSR_PREC_NATIVE)
        return fail(VBCSR_ERR_UNSUPPORTED, "complex operators run in NATIVE precision only");
    const int64_t xrows = trans ? A->n_rows : A->n_cols;
    const int64_t yrows = trans ? A->n_cols : A->n_rows;
    const bool want_dot = epi && epi->dot_out;
    if (k == 0 || yrows == 0) {
        if (want_dot) CUDA_TRY(cudaMemsetAsync(epi->dot_out, 0, sizeof(double), s), "memset dot");
        return VBCSR_OK;
    }
    if (ldx < k || ldy < k) return fail(VBCSR_ERR_INVALID_ARG, "leading dimension below k");
    if (!Y) return fail(VBCSR_ERR_INVALID_ARG, "Y is NULL");
    if (alpha != 0.0 && xrows > 0 && !X) return fail(VBCSR_ERR_INVALID_ARG, "X is NULL");
    if (alpha != 0.0 && X && overlap(X, xrows, ldx, Y, yrows, ldy, k, A->esize))
        return fail(VBCSR_ERR_ALIAS, "Y overlaps X");
    const double gamma = epi ? epi->gamma : 0.0;
    if (gamma != 0.0 && (!epi->Z || epi->ldz < k)) return fail(VBCSR_ERR_INVALID_ARG, "epilogue Z / ldz");
    if (want_dot && (!epi->R || epi->ldr < k)) return fail(VBCSR_ERR_INVALID_ARG, "epilogue R / ldr");

    const ModePlan mp = plan_mode(A, trans, k, precision);
    const bool f64 = mp.f64;
    const int mode = mp.mode;
    const bool fma = mp.fma, csr_kernel = mp.csr_kernel, split = mp.split, presplit = mp.presplit;
    const int mma_mode = presplit ? kBF16X2Presplit : mode;
    if (mp.need_panel32 && !A->panel32_valid) {
        int rc = refresh_panel32(A, s);
        if (rc) return rc;
    }
    if (mp.need_panelbf && !A->panelbf_valid) {
        int rc = refresh_panelbf(A, s);
        if (rc) return rc;
    }
    if (mp.need_paneldf && !A->paneldf_valid) {
        int rc = refresh_paneldf(A, s);
        if (rc) return rc;
    }
    if (mp.need_panelbp && !A->panelbp_valid) {
        int rc = refresh_panelbp(A, s);
        if (rc) return rc;
    }
    const bool piped = mp.pipe || mp.pipe_tf;
    const int64_t ldp = piped ? pipe_ldp(k) : 0;   // X row stride of the pipelined kernels

    // The mixed modes read X as FP32 (the double-FP32 mode as hi/lo pairs):
    // convert an FP64 X once here rather than at every gather inside the
    // kernel (each X row is gathered by ~30 work items).
    const bool fused = fx && !trans && fused_x_applies(A, mp);
    if (fused && fx->x_in && alpha != 0.0 && xrows > 0) {
        X = fx->x_in;
        ldx = piped ? ldp : k;
    } else if (mp.xkind != kXAsGiven && alpha != 0.0 && xrows > 0) {
        const size_t need = (size_t)xrows * (size_t)k;
        if (mp.xkind == kXPlanes) {
            int rc = grow(A, &A->xbp, &A->xbp_elems, 2 * (size_t)xrows * (size_t)ldp, s, "alloc bf16 planes of X");
            if (rc) return rc;
            CUDA_TRY(launch_split_bf16_planes_panel(xrows, k, (const double *)X, ldx, A->xbp,
                                                    A->xbp + (size_t)xrows * ldp, ldp, s),
                     "split X");
            X = A->xbp;
            ldx = ldp;
        } else if (mp.xkind == kXF32P) {
            int rc = grow(A, &A->xbp, &A->xbp_elems, 2 * (size_t)xrows * (size_t)ldp, s, "alloc FP32 rows of X");
            if (rc) return rc;
            CUDA_TRY(launch_convert_panel_f64_to_f32(xrows, k, (const double *)X, ldx, (float *)A->xbp, ldp, s),
                     "convert X");
            X = A->xbp;
            ldx = ldp;
        } else if (mp.xkind == kXPairs) {
            int rc = grow(A, &A->xdf, &A->xdf_elems, need, s, "alloc double-FP32 copy of X");
            if (rc) return rc;
            CUDA_TRY(launch_split_df(xrows, k, (const double *)X, ldx, A->xdf, s), "split X");
            X = A->xdf;
        } else if (mp.xkind == kXSplit) {
            int rc = grow(A, &A->xbf, &A->xbf_elems, need, s, "alloc split copy of X");
            if (rc) return rc;
            CUDA_TRY(launch_split_bf16_panel(xrows, k, (const double *)X, ldx, A->xbf, s), "split X");
            X = A->xbf;
        } else {
            int rc = grow(A, &A->xconv, &A->xconv_elems, need, s, "alloc FP32 copy of X");
            if (rc) return rc;
            CUDA_TRY(launch_convert_panel_f64_to_f32(xrows, k, (const double *)X, ldx, A->xconv, k, s), "convert X");
            X = A->xconv;
        }
        if (!piped) ldx = k;
    }

    // FP32 values (an FP32 operator, or the F32 mode of an FP64 one) at k >= 8 under the
    // persistent schedule run the pipelined CUDA-core kernel when X rows are 16-byte aligned
    const bool fpipe = fma && !trans && !cplx && !csr_kernel && A->backend != VBCSR_BACKEND_CSR &&
                       (mode == VBCSR_PREC_F32 || (!f64 && mode == VBCSR_PREC_NATIVE)) && k >= 8 &&
                       (A->schedule & VBCSR_SCHED_PERSISTENT) && !(A->schedule & VBCSR_SCHED_NO_FPIPE) &&
                       ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    ProdArgs a;
    memset(&a, 0, sizeof(a));
    a.values = mode == VBCSR_PREC_DF32 ? (const void *)A->paneldf
             : mp.pipe ? (const void *)A->panelbp
             : presplit ? (const void *)A->panelbf
             : (f64 && mode != VBCSR_PREC_NATIVE) ? (const void *)A->panel32 : A->panel;
    a.fl = {A->fl_xrow, A->fl_pcol, A->fl_w};
    a.tl = {A->tl_pbase, A->tl_kp, A->tl_bi, A->tl_xrow, A->tl_vcol};
    a.k = k;
    a.alpha = alpha;
    a.beta = beta;
    a.gamma = gamma;
    a.alpha32 = (float)alpha;
    a.beta32 = (float)beta;
    a.gamma32 = (float)gamma;
    a.beta_nz = beta != 0.0;
    a.gamma_nz = gamma != 0.0;
    a.X = X;
    a.ldx = ldx;
    a.Y = Y;
    a.ldy = ldy;
    a.Z = gamma != 0.0 ? epi->Z : nullptr;
    a.ldz = gamma != 0.0 ? epi->ldz : 0;
    a.R = want_dot ? epi->R : nullptr;
    a.ldr = want_dot ? epi->ldr : 0;
    a.x_rows = xrows;
    a.err = A->err;
    a.debug_checks = A->debug_checks;
    a.xs_out = fused && fx->x_out ? fx->x_out : nullptr;
    if (mp.pipe) {
        a.v_plane = A->panel_elems;
        a.x_plane = xrows * ldp;
        a.xs_plane = yrows * ldp;
    }
    const int kc_auto = auto_kc(k);
    // FP32 values and double-FP32 pairs in the CUDA-core forward kernels with
    // column tiles of 8 or more go through the shared-memory ring unless the
    // schedule opts out. Measured on the 50k-atom operator: FP32 10 / 20 / 18 %
    // and double-FP32 8 / 8 / 5 % faster at k = 8 / 16 / 32 (FP32 1.5 % slower at
    // k = 4); double-FP32 in one persistent launch over many row counts (nine on
    // the variable-block domain) 6-18 % slower, so not there.
    const bool many_heights = A->fwd_buckets.size() > 2 && (A->schedule & VBCSR_SCHED_PERSISTENT);
    a.value_ring = fma && !trans && !cplx &&
                           (mode == VBCSR_PREC_F32 || (mode == VBCSR_PREC_DF32 && !many_heights) ||
                            (!f64 && mode == VBCSR_PREC_NATIVE)) &&
                           !(A->schedule & VBCSR_SCHED_NO_RING) && kc_auto >= 8
                       ? 1
                       : 0;
    auto kc_for = [&](int B) { return A->kc_b[B] ? std::min(A->kc_b[B], kc_auto) : kc_auto; };

    // the double-FP32 persistent forward kernel in its narrow form when the
    // operator has more than two row counts (the wide form's larger code then
    // runs slower, see process_item)
    const bool df_narrow = A->fwd_buckets.size() > 2;
    int64_t used = 0;
    bool per_item_dot = false;   // the persistent CUDA-core launch writes one dot share per item
    // one launch of `kern` over items[0..n) with `warps` warps per CTA
    auto launch = [&](int B, const WorkItem *items, int64_t n, int warps, const void *kern, size_t smem) -> int {
        a.items = items;
        a.n_items = n;
        a.warps = warps;
        cudaError_t pending = cudaGetLastError();
        if (pending != cudaSuccess) return cuda_fail(pending, "error pending before the product launch");
        const int cap = cached_cap(kern, warps, smem);
        if (cap < 0) return cuda_fail(cudaGetLastError(), "occupancy query of the product kernel");
        const int64_t need = (n + warps - 1) / warps;
        a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, cap));
        a.partials = nullptr;
        a.item_partials = nullptr;
        if (want_dot && per_item_dot) {
            a.item_partials = A->item_partials;
        } else if (want_dot) {
            if (used + a.grid > kPartialsCap) return fail(VBCSR_ERR_UNSUPPORTED, "too many CTAs for the dot");
            a.partials = A->partials + used;
            used += a.grid;
        }
        cudaError_t e;
        if (fpipe)
            e = launch_fma32_pipe(f64, a, s);
        else if (mode == VBCSR_PREC_NATIVE)
            e = cplx ? launch_fma_c128(B, trans, a, s)
                     : (f64 ? launch_fma_f64(B, trans, a, s) : launch_fma_f32(B, trans, a, s));
        else if (mode == VBCSR_PREC_F32)
            e = launch_fma_f32_on_f64(B, trans, a, s);
        else if (mode == VBCSR_PREC_DF32)
            e = launch_fma_df(B, trans, a, s, df_narrow);
        else if (split)
            e = launch_fma_split(mma_mode, a, s);
        else if (piped)
            e = launch_mma_pipe(mp.pipe ? kBF16X2 : mode, a, s);
        else
            e = launch_mma(mma_mode, f64, trans, a, s);
        if (e != cudaSuccess) return cuda_fail(e, "product launch");
        return VBCSR_OK;
    };
    auto fma_kern = [&](bool persistent, int B) {
        const bool ring = a.value_ring != 0;
        if (cplx) return fma_c128_kernel(trans, persistent, B);
        if (mode == VBCSR_PREC_DF32) return fma_df_kernel(trans, persistent, B, df_narrow, ring);
        return (mode == VBCSR_PREC_NATIVE)
                   ? (f64 ? fma_f64_kernel(trans, persistent, B) : fma_f32_kernel(trans, persistent, B, ring))
                   : fma_f32_on_f64_kernel(trans, persistent, B, ring);
    };
    const int64_t n_all = trans ? A->n_adj_items : A->n_fwd_items;
    int rc = VBCSR_OK;
    if (!fma && !split) {
        // tensor-core kernel: the row count is a runtime mask, one launch serves every item
        const bool staged = !trans && (A->schedule & VBCSR_SCHED_MMA_STAGED);
        a.mma_staged = staged ? 1 : 0;
        if (!staged) {
            // the plain kernel takes items in descending cost from the work counter
            a.queue = A->queue;
            per_item_dot = true;
            CUDA_TRY(cudaMemsetAsync(A->queue, 0, sizeof(long long), s), "reset work counter");
        }
        const int pmode = mp.pipe ? kBF16X2 : mode;
        const void *kern = piped ? mma_pipe_kernel_ptr(pmode, k) : mma_kernel_ptr(mma_mode, f64, trans, staged, k);
        if (!kern) return fail(VBCSR_ERR_UNSUPPORTED, "precision %d not available for this operation", precision);
        rc = launch(0, trans ? A->adj_lpt : A->fwd_lpt, n_all, 4, kern,
                    piped ? mma_pipe_smem_bytes(pmode, k, 4) : mma_smem_bytes(trans, staged, 4));
    } else if (csr_kernel) {
        // scalar operator: several rows per warp; items are the scalar rows in page order
        const int kind = split ? (mode == VBCSR_PREC_TF32 ? kCsrSplitTF32
                                  : mode == VBCSR_PREC_TF32X3 ? kCsrSplitTF32X3 : kCsrSplitBF16X2)
                       : mode == VBCSR_PREC_DF32 ? kCsrDF
                       : mode == VBCSR_PREC_F32 ? kCsrF32OnF64 : (f64 ? kCsrF64 : kCsrF32);
        const int L = A->csr_lanes[csr_lane_class(kind)];
        a.items = A->fwd_items;
        a.n_items = A->n_fwd_items;
        a.warps = 8;
        cudaError_t pending = cudaGetLastError();
        if (pending != cudaSuccess) return cuda_fail(pending, "error pending before the product launch");
        const int cap = cached_cap(csr_kernel_ptr(kind, L, k), a.warps, 0);
        if (cap < 0) return cuda_fail(cudaGetLastError(), "occupancy query of the scalar kernel");
        const int64_t need = (a.n_items + a.warps * (32 / L) - 1) / (a.warps * (32 / L));
        a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, cap));
        if (want_dot) {
            a.partials = A->partials;
            used = a.grid;
        }
        CUDA_TRY(launch_csr(kind, L, a, s), "scalar product launch");
    } else if (fpipe) {
        // FP32 values, k >= 8, persistent schedule: the pipelined CUDA-core kernel
        a.queue = A->queue;
        per_item_dot = true;
        CUDA_TRY(cudaMemsetAsync(A->queue, 0, sizeof(long long), s), "reset work counter");
        rc = launch(0, A->fwd_lpt, n_all, 4, fma32_pipe_kernel_ptr(k, f64), fma32_pipe_smem_bytes(k, 4));
    } else if (split || (A->schedule & VBCSR_SCHED_PERSISTENT)) {
        // persistent launch over every row count, items in descending cost from a work queue
        // (the only launch shape of the CUDA-core form of the tensor-core modes)
        a.kc_log2_by_b = 0;
        for (int B = 1; B <= kMaxB; ++B) {
            int l = 0;
            while ((1 << l) < kc_for(B)) ++l;
            a.kc_log2_by_b |= (uint64_t)l << (3 * B);
        }
        a.queue = A->queue;
        per_item_dot = true;
        CUDA_TRY(cudaMemsetAsync(A->queue, 0, sizeof(long long), s), "reset work counter");
        const int warps = A->persist_warps ? A->persist_warps : 4;
        rc = launch(0, trans ? A->adj_lpt : A->fwd_lpt, n_all, warps,
                    split ? fma_split_kernel(mma_mode) : fma_kern(true, 0),
                    fma_smem_bytes(trans, warps, a.value_ring != 0));
    } else {
        const std::vector<Bucket> &buckets = trans ? A->adj_buckets : A->fwd_buckets;
        const WorkItem *items = trans ? A->adj_items : A->fwd_items;
        for (const Bucket &b : buckets) {
            a.kc = kc_for(b.B);
            const int warps = A->warps_b[b.B] ? A->warps_b[b.B] : 4;
            rc = launch(b.B, items + b.begin, b.count, warps, fma_kern(false, b.B),
                        fma_smem_bytes(trans, warps, a.value_ring != 0));
            if (rc) return rc;
        }
    }
    if (rc) return rc;
    if (want_dot)
        CUDA_TRY(launch_finalize_dot(per_item_dot ? A->item_partials : A->partials, per_item_dot ? n_all : used,
                                     dot_scale, epi->dot_out, A->dot_scratch, s),
                 "dot finalize");
    return VBCSR_OK;
}

extern "C" int vbcsr_spmm(vbcsr_t *A, int64_t k, double alpha, const void *X, int64_t ldx, double beta, void *Y,
                          int64_t ldy, int precision, void *stream) {
    return run_product(A, false, k, alpha, X, ldx, beta, Y, ldy, nullptr, precision, (cudaStream_t)stream);
}

extern "C" int vbcsr_spmm_adjoint(vbcsr_t *A, int64_t k, double alpha, const void *X, int64_t ldx, double beta,
                                  void *Y, int64_t ldy, int precision, void *stream) {
    return run_product(A, true, k, alpha, X, ldx, beta, Y, ldy, nullptr, precision, (cudaStream_t)stream);
}

extern "C" int vbcsr_spmm_ex(vbcsr_t *A, int transpose, int64_t k, double alpha, const void *X, int64_t ldx,
                             double beta, void *Y, int64_t ldy, const vbcsr_epilogue_t *epi, int precision,
                             void *stream) {
    if (transpose != 0 && transpose != 1) return fail(VBCSR_ERR_INVALID_ARG, "transpose must be 0 or 1");
    return run_product(A, transpose == 1, k, alpha, X, ldx, beta, Y, ldy, epi, precision, (cudaStream_t)stream);
}

// the pattern fields of a pattern-sampled product over the handle's forward items
static SddmmArgs sddmm_args(vbcsr_t *A) {
    SddmmArgs a;
    memset(&a, 0, sizeof(a));
    a.items = A->fwd_lpt;
    a.n_items = A->n_fwd_items;
    a.queue = A->queue;
    a.fl_xrow = A->fl_xrow;
    a.fl_pcol = A->fl_pcol;
    a.fl_w = A->fl_w;
    a.fl_uoff = A->fl_uoff;
    a.fl_pbase = A->fl_pbase;
    return a;
}

extern "C" int vbcsr_sddmm(vbcsr_t *A, int64_t k, double alpha, const void *Aop, int64_t lda, const void *Bop,
                           int64_t ldb, double beta, void *D, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (k < 0) return fail(VBCSR_ERR_INVALID_ARG, "k = %lld", (long long)k);
    if (A->dtype == VBCSR_C128) return fail(VBCSR_ERR_UNSUPPORTED, "pattern-sampled product of a complex operator");
    if (A->nnz == 0) return VBCSR_OK;
    if (!D) return fail(VBCSR_ERR_INVALID_ARG, "D is NULL");
    if (k > 0 && alpha != 0.0) {
        if (!Aop || !Bop) return fail(VBCSR_ERR_INVALID_ARG, "operand is NULL");
        if (lda < k || ldb < k) return fail(VBCSR_ERR_INVALID_ARG, "leading dimension below k");
    }
    SddmmArgs a = sddmm_args(A);
    a.k = alpha != 0.0 ? k : 0;
    a.alpha = alpha;
    a.beta = beta;
    a.A = Aop;
    a.lda = lda;
    a.B = Bop;
    a.ldb = ldb;
    a.D = D;
    CUDA_TRY(launch_sddmm(A->dtype == VBCSR_F64, a, (cudaStream_t)stream), "sddmm launch");
    return VBCSR_OK;
}

// ---------------------------------------------------------------------------
// Chebyshev moments (kernel polynomial method, Sec. V)

// The two converted-X panels of a recurrence whose forward products run the
// plain tensor-core kernel: xs[0] is the handle's conversion buffer
// (where the first product converts R), xs[1] the panel after it; both NULL
// when the fused form does not apply (the products then convert X themselves).
static int cheb_fused_buffers(vbcsr_t *A, int64_t k, int precision, void *xs[2], cudaStream_t s) {
    xs[0] = xs[1] = nullptr;
    if (A->dtype != VBCSR_F64) return VBCSR_OK;
    const ModePlan mp = plan_mode(A, false, k, precision);
    if (!fused_x_applies(A, mp) || A->n_rows == 0) return VBCSR_OK;
    const size_t panel = (size_t)A->n_rows * (size_t)k;
    if (mp.xkind == kXPlanes || mp.xkind == kXF32P) {
        const size_t planes = 2 * (size_t)A->n_rows * (size_t)pipe_ldp(k);
        int rc = grow(A, &A->xbp, &A->xbp_elems, 2 * planes, s, "alloc bf16 planes of the Chebyshev vectors");
        if (rc) return rc;
        xs[0] = A->xbp;
        xs[1] = A->xbp + planes;
    } else if (mp.xkind == kXSplit) {
        int rc = grow(A, &A->xbf, &A->xbf_elems, 2 * panel, s, "alloc split copies of the Chebyshev vectors");
        if (rc) return rc;
        xs[0] = A->xbf;
        xs[1] = A->xbf + panel;
    } else {
        int rc = grow(A, &A->xconv, &A->xconv_elems, 2 * panel, s, "alloc FP32 copies of the Chebyshev vectors");
        if (rc) return rc;
        xs[0] = A->xconv;
        xs[1] = A->xconv + panel;
    }
    return VBCSR_OK;
}


extern "C" int vbcsr_chebyshev(vbcsr_t *A, int64_t k, const double *R, int64_t ldr, int64_t n_moments,
                               double *moments, double *work, double *ckpt, int64_t ckpt_every, int precision,
                               void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (A->dtype != VBCSR_F64 && A->dtype != VBCSR_C128)
        return fail(VBCSR_ERR_UNSUPPORTED, "the recurrence needs an FP64 or complex operator");
    if (A->n_rows != A->n_cols) return fail(VBCSR_ERR_INVALID_ARG, "operator is not square");
    if (k < 1 || n_moments < 1) return fail(VBCSR_ERR_INVALID_ARG, "k and n_moments must be >= 1");
    if (!R || !moments || !work || ldr < k) return fail(VBCSR_ERR_INVALID_ARG, "R / moments / work / ldr");
    if (ckpt && ckpt_every < 1) return fail(VBCSR_ERR_INVALID_ARG, "ckpt_every must be >= 1");
    if (precision < VBCSR_PREC_NATIVE || precision > VBCSR_PREC_DF32)
        return fail(VBCSR_ERR_INVALID_ARG, "precision %d", precision);
    cudaStream_t s = (cudaStream_t)stream;
    // complex panels are handled by the real copy and dot kernels as cw = 2 real
    // columns per complex one (the dot of interleaved pairs is Re sum(conj(R) t))
    const int64_t cw = A->dtype == VBCSR_C128 ? 2 : 1;
    const int64_t N = A->n_rows, panel = N * k * cw;
    const double scale = 1.0 / ((double)N * (double)k);
    double *buf[2] = {work, work + panel};
    void *xs[2] = {nullptr, nullptr};
    if (n_moments > 1) {
        int rc = cheb_fused_buffers(A, k, precision, xs, s);
        if (rc) return rc;
    }

    int64_t used = 0;
    CUDA_TRY(launch_dot_panels(true, N, k * cw, R, ldr * cw, R, ldr * cw, A->partials, kPartialsCap, &used, s),
             "dot");
    CUDA_TRY(launch_finalize_dot(A->partials, used, scale, moments, A->dot_scratch, s), "dot");
    if (n_moments == 1) return VBCSR_OK;

    vbcsr_epilogue_t epi;
    memset(&epi, 0, sizeof(epi));
    epi.R = R;
    epi.ldr = ldr;
    // t_1 = H~ R  -> buf[1];  t_0 (a copy of R) -> buf[0]
    epi.dot_out = moments + 1;
    // with the fused form, t_n is also kept converted in xs[n & 1]
    const FusedX fx0 = {nullptr, xs[1]};
    int rc = run_product(A, false, k, 1.0, R, ldr, 0.0, buf[1], k, &epi, precision, s, scale, xs[1] ? &fx0 : nullptr);
    if (rc) return rc;
    auto store_pair = [&](int64_t m, const double *tm, int64_t ldm, const double *tm1) -> int {
        if (!ckpt || m % ckpt_every) return VBCSR_OK;
        double *slot = ckpt + (m / ckpt_every) * 2 * panel;
        CUDA_TRY(launch_copy_panel(N, k * cw, tm, ldm * cw, slot, k * cw, s), "checkpoint");
        CUDA_TRY(launch_copy_panel(N, k * cw, tm1, k * cw, slot + panel, k * cw, s), "checkpoint");
        return VBCSR_OK;
    };
    if ((rc = store_pair(0, R, ldr, buf[1]))) return rc;
    if (n_moments == 2) return VBCSR_OK;
    CUDA_TRY(launch_copy_panel(N, k * cw, R, ldr * cw, buf[0], k * cw, s), "copy R");
    // t_{n+1} = 2 H~ t_n - t_{n-1}: t_n in buf[n & 1], t_{n-1} (overwritten by t_{n+1}) in buf[(n+1) & 1]
    for (int64_t n = 1; n + 1 < n_moments; ++n) {
        double *tn = buf[n & 1], *tprev = buf[(n + 1) & 1];
        epi.dot_out = moments + n + 1;
        const FusedX fx = {xs[n & 1], xs[(n + 1) & 1]};
        rc = run_product(A, false, k, 2.0, tn, k, -1.0, tprev, k, &epi, precision, s, scale, xs[0] ? &fx : nullptr);
        if (rc) return rc;
        if ((rc = store_pair(n, tn, k, tprev))) return rc;
    }
    return VBCSR_OK;
}

extern "C" int vbcsr_chebyshev_backward(vbcsr_t *A, int64_t k, const double *R, int64_t ldr, int64_t M,
                                        const double *grad_mu, const double *ckpt, int64_t E, double d_scale,
                                        double *dvalues, double *work, int precision, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (!(d_scale != 0.0) || d_scale != d_scale || d_scale - d_scale != 0.0)
        return fail(VBCSR_ERR_INVALID_ARG, "d_scale = %g", d_scale);
    if (A->dtype != VBCSR_F64) return fail(VBCSR_ERR_UNSUPPORTED, "the recurrence needs an FP64 operator");
    if (A->n_rows != A->n_cols) return fail(VBCSR_ERR_INVALID_ARG, "operator is not square");
    if (k < 1 || M < 1 || E < 1) return fail(VBCSR_ERR_INVALID_ARG, "k, n_moments and ckpt_every must be >= 1");
    if (!R || ldr < k || !grad_mu || !dvalues || !work || (M > 1 && !ckpt))
        return fail(VBCSR_ERR_INVALID_ARG, "NULL argument or ldr < k");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = A->n_rows, panel = N * k, wide = E * k;
    if (A->nnz) CUDA_TRY(cudaMemsetAsync(dvalues, 0, (size_t)A->nnz * sizeof(double), s), "memset");
    if (M < 2) return VBCSR_OK;
    std::vector<double> gm(M);
    CUDA_TRY(cudaMemcpyAsync(gm.data(), grad_mu, M * sizeof(double), cudaMemcpyDeviceToHost, s), "copy grad_mu");
    CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
    const double scale = 1.0 / ((double)N * (double)k);
    double *cur = work, *nxt = work + panel;          // lam_{n+1}, lam_{n+2}
    double *T = work + 2 * panel, *L = T + N * wide;  // [N, E k] segment panels
    // lam_{M-1} = g_{M-1};  lam_M = 0
    CUDA_TRY(launch_axpby(N, k, gm[M - 1] * scale, R, ldr, 0.0, cur, k, s), "axpby");
    CUDA_TRY(cudaMemsetAsync(nxt, 0, (size_t)panel * sizeof(double), s), "memset");
    const int64_t nseg = (M - 1 + E - 1) / E;
    bool first = true;
    int rc;
    vbcsr_epilogue_t epi;
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        const int64_t n_lo = sg * E, n_hi = std::min((sg + 1) * E - 1, M - 2);
        const int64_t cnt = n_hi - n_lo + 1;
        const double *pair = ckpt + sg * 2 * panel;
        // recompute t_{n_lo} .. t_{n_hi} into the column slots of T
        CUDA_TRY(launch_copy_panel(N, k, pair, k, T, wide, s), "restore checkpoint");
        if (cnt > 1) CUDA_TRY(launch_copy_panel(N, k, pair + panel, k, T + k, wide, s), "restore checkpoint");
        for (int64_t e = 1; e + 1 < cnt; ++e) {
            memset(&epi, 0, sizeof(epi));
            epi.gamma = -1.0;
            epi.Z = T + (e - 1) * k;
            epi.ldz = wide;
            rc = run_product(A, false, k, 2.0, T + e * k, wide, 0.0, T + (e + 1) * k, wide, &epi, precision, s);
            if (rc) return rc;
        }
        for (int64_t n = n_hi; n >= n_lo; --n) {
            const int64_t e = n - n_lo;
            CUDA_TRY(launch_axpby(N, k, n >= 1 ? 2.0 : 1.0, cur, k, 0.0, L + e * k, wide, s), "axpby");
            if (n >= 1) {
                memset(&epi, 0, sizeof(epi));
                epi.gamma = gm[n] * scale;
                epi.Z = R;
                epi.ldz = ldr;
                rc = run_product(A, true, k, 2.0, cur, k, -1.0, nxt, k, &epi, precision, s);
                if (rc) return rc;
                std::swap(cur, nxt);
            }
        }
        SddmmArgs a = sddmm_args(A);
        a.k = cnt * k;
        a.alpha = 1.0 / d_scale;
        a.beta = first ? 0.0 : 1.0;
        a.A = L;
        a.lda = wide;
        a.B = T;
        a.ldb = wide;
        a.D = dvalues;
        if (A->nnz) CUDA_TRY(launch_sddmm(true, a, s), "sddmm");
        first = false;
    }
    return VBCSR_OK;
}

extern "C" int vbcsr_kpm_moments(vbcsr_t *A, int64_t k, const double *R, int64_t ldr, int64_t M, double *moments,
                                 double *work, int precision, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (A->dtype != VBCSR_F64 && A->dtype != VBCSR_C128)
        return fail(VBCSR_ERR_UNSUPPORTED, "the recurrence needs an FP64 or complex operator");
    if (A->n_rows != A->n_cols) return fail(VBCSR_ERR_INVALID_ARG, "operator is not square");
    if (k < 1 || M < 1) return fail(VBCSR_ERR_INVALID_ARG, "k and n_moments must be >= 1");
    if (!R || !moments || !work || ldr < k) return fail(VBCSR_ERR_INVALID_ARG, "R / moments / work / ldr");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t cw = A->dtype == VBCSR_C128 ? 2 : 1;   // real columns per (complex) column
    const int64_t N = A->n_rows, panel = N * k * cw;
    const double scale = 1.0 / ((double)N * (double)k);
    double *buf[2] = {work, work + panel};
    int64_t used = 0;
    auto self_dot = [&](const double *t, int64_t ld, double *out) -> int {
        CUDA_TRY(launch_dot_panels(true, N, k * cw, t, ld * cw, t, ld * cw, A->partials, kPartialsCap, &used, s),
                 "dot");
        CUDA_TRY(launch_finalize_dot(A->partials, used, scale, out, A->dot_scratch, s), "dot");
        return VBCSR_OK;
    };
    if (precision < VBCSR_PREC_NATIVE || precision > VBCSR_PREC_DF32)
        return fail(VBCSR_ERR_INVALID_ARG, "precision %d", precision);
    void *xs[2] = {nullptr, nullptr};
    if (M > 3) {
        int rc = cheb_fused_buffers(A, k, precision, xs, s);
        if (rc) return rc;
    }
    int rc = self_dot(R, ldr, moments);                                     // mu_0
    if (rc || M == 1) return rc;
    vbcsr_epilogue_t epi;
    memset(&epi, 0, sizeof(epi));
    epi.R = R;
    epi.ldr = ldr;
    epi.dot_out = moments + 1;                                             // mu_1 = <t_1, t_0>
    const FusedX fx0 = {nullptr, xs[1]};
    if ((rc = run_product(A, false, k, 1.0, R, ldr, 0.0, buf[1], k, &epi, precision, s, scale,
                          xs[1] ? &fx0 : nullptr)))
        return rc;
    CUDA_TRY(launch_copy_panel(N, k * cw, R, ldr * cw, buf[0], k * cw, s), "copy R");
    // t_n in buf[n & 1]; raw dots <t_n, t_n> -> moments[2n], <t_{n+1}, t_n> -> moments[2n+1]
    for (int64_t n = 1;; ++n) {
        double *tn = buf[n & 1], *tprev = buf[(n + 1) & 1];
        if (2 * n < M && (rc = self_dot(tn, k, moments + 2 * n))) return rc;
        if (2 * n + 1 >= M) break;
        epi.R = tn;
        epi.ldr = k;
        epi.dot_out = moments + 2 * n + 1;
        const FusedX fx = {xs[n & 1], xs[(n + 1) & 1]};
        if ((rc = run_product(A, false, k, 2.0, tn, k, -1.0, tprev, k, &epi, precision, s, scale,
                              xs[0] ? &fx : nullptr)))
            return rc;
    }
    CUDA_TRY(launch_kpm_fixup(moments, M, s), "moment fix-up");
    return VBCSR_OK;
}

extern "C" int vbcsr_kpm_dos(const double *moments, int64_t n_moments, int kernel, const double *x, int64_t n_x,
                             double *dos, void *stream) {
    if (n_moments < 1 || n_x < 0) return fail(VBCSR_ERR_INVALID_ARG, "n_moments %lld, n_x %lld",
                                             (long long)n_moments, (long long)n_x);
    if (kernel != VBCSR_KPM_NO_KERNEL && kernel != VBCSR_KPM_JACKSON)
        return fail(VBCSR_ERR_INVALID_ARG, "kernel %d", kernel);
    if (!moments || (n_x > 0 && (!x || !dos))) return fail(VBCSR_ERR_INVALID_ARG, "NULL argument");
    CUDA_TRY(launch_kpm_dos(moments, n_moments, kernel == VBCSR_KPM_JACKSON, x, n_x, dos, (cudaStream_t)stream),
             "kpm dos");
    return VBCSR_OK;
}

extern "C" int vbcsr_kpm_gap(const double *energies, const double *dos, int64_t n, double reference,
                             double threshold, double *out, void *stream) {
    if (n < 1) return fail(VBCSR_ERR_INVALID_ARG, "n = %lld", (long long)n);
    if (!energies || !dos || !out) return fail(VBCSR_ERR_INVALID_ARG, "NULL argument");
    if (reference != reference || threshold != threshold)
        return fail(VBCSR_ERR_INVALID_ARG, "reference / threshold is NaN");
    CUDA_TRY(launch_kpm_gap(energies, dos, n, reference, threshold, out, (cudaStream_t)stream), "kpm gap");
    return VBCSR_OK;
}

extern "C" int vbcsr_gershgorin(vbcsr_t *A, double *bounds, void *stream) {
    if (!A || !bounds) return fail(VBCSR_ERR_INVALID_ARG, "NULL argument");
    if (A->dtype != VBCSR_F64 && A->dtype != VBCSR_C128)
        return fail(VBCSR_ERR_UNSUPPORTED, "Gershgorin bounds need an FP64 or complex operator");
    if (A->n_rows != A->n_cols) return fail(VBCSR_ERR_INVALID_ARG, "operator is not square");
    if (A->n_rows == 0) return fail(VBCSR_ERR_INVALID_ARG, "empty operator");
    CUDA_TRY(launch_gershgorin(A->dtype == VBCSR_C128, A->fwd_items, A->n_fwd_items, A->panel, A->fl_xrow, A->fl_pcol,
                               A->fl_w, A->partials, kPartialsCap, bounds, (cudaStream_t)stream),
             "gershgorin");
    return VBCSR_OK;
}

extern "C" int vbcsr_shift_scale(vbcsr_t *A, double c, double d, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (A->dtype != VBCSR_F64 && A->dtype != VBCSR_C128)
        return fail(VBCSR_ERR_UNSUPPORTED, "shift/scale needs an FP64 or complex operator");
    if (A->n_rows != A->n_cols) return fail(VBCSR_ERR_INVALID_ARG, "operator is not square");
    if (!(d != 0.0) || d != d || c != c) return fail(VBCSR_ERR_INVALID_ARG, "c = %g, d = %g", c, d);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(launch_shift_scale(A->dtype == VBCSR_C128, A->fwd_items, A->n_fwd_items, A->panel, A->fl_xrow,
                                A->fl_pcol, A->fl_w, c,
                                d, s),
             "shift_scale");
    if (A->panel32) {
        int rc = refresh_panel32(A, s);
        if (rc) return rc;
    }
    if (A->panelbf) {
        int rc = refresh_panelbf(A, s);
        if (rc) return rc;
    }
    if (A->panelbp) {
        int rc = refresh_panelbp(A, s);
        if (rc) return rc;
    }
    if (A->paneldf) return refresh_paneldf(A, s);
    return VBCSR_OK;
}

// ---------------------------------------------------------------------------
// thresholded block sparse product (Eqs. 2-3)

namespace {
template <typename T>
struct DevVec {   // temporary device array freed on scope exit
    T *p = nullptr;
    ~DevVec() {
        if (p) cudaFree(p);
    }
    cudaError_t put(const std::vector<T> &v, cudaStream_t s) {
        cudaError_t e = cudaMalloc((void **)&p, std::max<size_t>(1, v.size()) * sizeof(T));
        if (e != cudaSuccess || v.empty()) return e;
        return cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc((void **)&p, std::max<size_t>(1, n) * sizeof(T)); }
};
}  // namespace

extern "C" int vbcsr_spgemm(const vbcsr_t *A, const vbcsr_t *B, double eps, vbcsr_t **Cout, void *stream) {
    if (!Cout) return fail(VBCSR_ERR_INVALID_ARG, "out is NULL");
    *Cout = nullptr;
    if (!A || !B) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (A->dtype != B->dtype) return fail(VBCSR_ERR_INVALID_ARG, "A and B have different dtypes");
    if (A->dtype == VBCSR_C128) return fail(VBCSR_ERR_UNSUPPORTED, "block product of complex operators");
    if (!(eps >= 0.0)) return fail(VBCSR_ERR_INVALID_ARG, "eps = %g", eps);
    if (A->n_bcols != B->n_brows) return fail(VBCSR_ERR_INVALID_ARG, "inner block counts differ");
    for (int64_t k = 0; k < A->n_bcols; ++k)
        if (A->col_b[k] != B->row_b[k]) return fail(VBCSR_ERR_INVALID_ARG, "inner block %lld sizes differ", (long long)k);
    cudaStream_t s = (cudaStream_t)stream;
    const bool f64 = A->dtype == VBCSR_F64;
    try {
        // block norms of both operands (plan order)
        const int64_t nbr = A->n_brows, nbc = B->n_bcols;
        DevVec<double> dA, dB;
        CUDA_TRY(dA.alloc(A->nblk), "alloc norms");
        CUDA_TRY(dB.alloc(B->nblk), "alloc norms");
        CUDA_TRY(launch_block_norms(f64, A->nblk, A->panel, A->fl_pbase, A->fl_kp, A->fl_bi, A->fl_w, dA.p, s),
                 "block norms");
        CUDA_TRY(launch_block_norms(f64, B->nblk, B->panel, B->fl_pbase, B->fl_kp, B->fl_bi, B->fl_w, dB.p, s),
                 "block norms");
        // symbolic stage on the device: pass 1 counts every block row (rows whose
        // candidates overflow the shared-memory table are counted again with a
        // workspace in device memory), the host scans the counts into row
        // offsets, pass 2 writes the kept pattern and the product lists
        DevVec<int32_t> d_acol, d_bcol, d_bcs, d_ovf;
        DevVec<int64_t> d_cnt;
        CUDA_TRY(d_acol.put(A->h_pcol, s), "upload");
        CUDA_TRY(d_bcol.put(B->h_pcol, s), "upload");
        CUDA_TRY(d_bcs.put(B->col_b, s), "upload");
        CUDA_TRY(d_ovf.alloc(nbr), "alloc");
        CUDA_TRY(d_cnt.alloc(3 * (size_t)nbr), "alloc");
        SymArgs y;
        memset(&y, 0, sizeof(y));
        y.n_rows = nbr;
        y.a_rowptr = A->prow_ptr;
        y.b_rowptr = B->prow_ptr;
        y.a_col = d_acol.p;
        y.b_col = d_bcol.p;
        y.a_norm = dA.p;
        y.b_norm = dB.p;
        y.a_w = A->fl_w;
        y.a_pbase = A->fl_pbase;
        y.b_pbase = B->fl_pbase;
        y.a_kp = A->fl_kp;
        y.b_kp = B->fl_kp;
        y.a_rowsize = A->d_row_b;
        y.b_colsize = d_bcs.p;
        y.eps = eps;
        y.overflow = d_ovf.p;
        y.cnt_out = d_cnt.p;
        y.cnt_prod = d_cnt.p + nbr;
        y.cnt_val = d_cnt.p + 2 * nbr;
        CUDA_TRY(launch_spgemm_symbolic(1, y, s), "symbolic stage");
        std::vector<int64_t> cnt(3 * (size_t)nbr);
        std::vector<int32_t> ovf(nbr);
        if (nbr) {
            CUDA_TRY(cudaMemcpyAsync(cnt.data(), d_cnt.p, cnt.size() * 8, cudaMemcpyDeviceToHost, s), "copy");
            CUDA_TRY(cudaMemcpyAsync(ovf.data(), d_ovf.p, ovf.size() * 4, cudaMemcpyDeviceToHost, s), "copy");
        }
        CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        // rows beyond the shared-memory table: a workspace sized by their product count
        std::vector<int64_t> big, ws_off(1, 0);
        std::vector<int32_t> ws_h, ws_cap;
        for (int64_t i = 0; i < nbr; ++i) {
            if (!ovf[i]) continue;
            int64_t np = 0;
            for (int64_t a = A->h_rowptr[i]; a < A->h_rowptr[i + 1]; ++a) {
                const int32_t k = A->h_pcol[a];
                np += B->h_rowptr[k + 1] - B->h_rowptr[k];
            }
            int64_t cap = 32;
            while (cap < np) cap <<= 1;
            if (cap > (1LL << 28)) return fail(VBCSR_ERR_UNSUPPORTED, "block row %lld: %lld candidate products",
                                               (long long)i, (long long)np);
            big.push_back(i);
            ws_cap.push_back((int32_t)cap);
            ws_h.push_back((int32_t)(2 * cap));
            ws_off.push_back(ws_off.back() + (int64_t)sym_ws_bytes((int)(2 * cap), (int)cap));
        }
        DevVec<int64_t> d_big, d_wsoff;
        DevVec<int32_t> d_wsh, d_wscap;
        DevVec<unsigned char> d_ws;
        SymArgs yb = y;
        if (!big.empty()) {
            CUDA_TRY(d_big.put(big, s), "upload");
            CUDA_TRY(d_wsoff.put(ws_off, s), "upload");
            CUDA_TRY(d_wsh.put(ws_h, s), "upload");
            CUDA_TRY(d_wscap.put(ws_cap, s), "upload");
            CUDA_TRY(d_ws.alloc((size_t)ws_off.back()), "alloc symbolic workspace");
            yb.n_rows = (int64_t)big.size();
            yb.rows = d_big.p;
            yb.global_ws = 1;
            yb.ws = d_ws.p;
            yb.ws_off = d_wsoff.p;
            yb.ws_h = d_wsh.p;
            yb.ws_cap = d_wscap.p;
            CUDA_TRY(launch_spgemm_symbolic(1, yb, s), "symbolic stage");
            CUDA_TRY(cudaMemcpyAsync(cnt.data(), d_cnt.p, cnt.size() * 8, cudaMemcpyDeviceToHost, s), "copy");
            CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        }
        // row offsets of the kept blocks, their products and their values
        std::vector<int64_t> out_ptr(nbr + 1, 0), off_prod(nbr + 1, 0), off_val(nbr + 1, 0);
        for (int64_t i = 0; i < nbr; ++i) {
            out_ptr[i + 1] = out_ptr[i] + cnt[i];
            off_prod[i + 1] = off_prod[i] + cnt[nbr + i];
            off_val[i + 1] = off_val[i] + cnt[2 * nbr + i];
        }
        const int64_t n_out = out_ptr[nbr], n_prod = off_prod[nbr], n_val = off_val[nbr];
        const size_t es = A->esize;
        DevVec<int64_t> d_optr, d_oprod, d_oval, d_pbeg, d_uoff, d_pa, d_pb;
        DevVec<int32_t> d_col, d_bi, d_bj, d_kpa, d_kpb, d_bk;
        DevVec<double> d_norm;
        DevVec<unsigned char> d_val;
        CUDA_TRY(d_optr.put(out_ptr, s), "upload");
        CUDA_TRY(d_oprod.put(off_prod, s), "upload");
        CUDA_TRY(d_oval.put(off_val, s), "upload");
        CUDA_TRY(d_pbeg.alloc(n_out + 1), "alloc");
        CUDA_TRY(d_uoff.alloc(n_out), "alloc");
        CUDA_TRY(d_col.alloc(n_out), "alloc");
        CUDA_TRY(d_bi.alloc(n_out), "alloc");
        CUDA_TRY(d_bj.alloc(n_out), "alloc");
        CUDA_TRY(d_pa.alloc(n_prod), "alloc product lists");
        CUDA_TRY(d_pb.alloc(n_prod), "alloc product lists");
        CUDA_TRY(d_kpa.alloc(n_prod), "alloc product lists");
        CUDA_TRY(d_kpb.alloc(n_prod), "alloc product lists");
        CUDA_TRY(d_bk.alloc(n_prod), "alloc product lists");
        CUDA_TRY(cudaMemcpyAsync(d_pbeg.p + n_out, &off_prod[nbr], 8, cudaMemcpyHostToDevice, s), "upload");
        for (SymArgs *q : {&y, &yb}) {
            q->off_out = d_optr.p;
            q->off_prod = d_oprod.p;
            q->off_val = d_oval.p;
            q->out_col = d_col.p;
            q->out_bi = d_bi.p;
            q->out_bj = d_bj.p;
            q->out_uoff = d_uoff.p;
            q->out_pbeg = d_pbeg.p;
            q->pa = d_pa.p;
            q->pb = d_pb.p;
            q->kpa = d_kpa.p;
            q->kpb = d_kpb.p;
            q->bk = d_bk.p;
        }
        CUDA_TRY(launch_spgemm_symbolic(2, y, s), "symbolic stage");
        if (!big.empty()) CUDA_TRY(launch_spgemm_symbolic(2, yb, s), "symbolic stage");

        // numeric stage
        CUDA_TRY(d_norm.alloc(n_out), "alloc norms");
        CUDA_TRY(d_val.alloc((size_t)n_val * es), "alloc product values");
        SpgemmArgs g;
        g.n_out = n_out;
        g.out_pbeg = d_pbeg.p;
        g.out_uoff = d_uoff.p;
        g.out_bi = d_bi.p;
        g.out_bj = d_bj.p;
        g.pa = d_pa.p;
        g.pb = d_pb.p;
        g.kpa = d_kpa.p;
        g.kpb = d_kpb.p;
        g.bk = d_bk.p;
        g.A = A->panel;
        g.B = B->panel;
        g.C = d_val.p;
        g.norms = d_norm.p;
        CUDA_TRY(launch_spgemm_numeric(f64, g, s), "numeric stage");
        // final filter on the computed block norms (Eq. 2)
        std::vector<double> norms(n_out);
        std::vector<int32_t> out_col(n_out);
        if (n_out) {
            CUDA_TRY(cudaMemcpyAsync(norms.data(), d_norm.p, n_out * 8, cudaMemcpyDeviceToHost, s), "copy");
            CUDA_TRY(cudaMemcpyAsync(out_col.data(), d_col.p, n_out * 4, cudaMemcpyDeviceToHost, s), "copy");
        }
        CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
        std::vector<int64_t> c_ptr(1, 0), keep_src, dst_off(1, 0);
        std::vector<int32_t> c_col, keep_size;
        c_ptr.reserve(nbr + 1);
        c_col.reserve(n_out);
        keep_src.reserve(n_out);
        keep_size.reserve(n_out);
        dst_off.reserve(n_out + 1);
        for (int64_t i = 0; i < nbr; ++i) {
            int64_t u = off_val[i];   // the block's offset in the unfiltered values
            for (int64_t o = out_ptr[i]; o < out_ptr[i + 1]; ++o) {
                const int32_t size = A->row_b[i] * B->col_b[out_col[o]];
                if (!(norms[o] < eps)) {
                    c_col.push_back(out_col[o]);
                    keep_src.push_back(u);
                    keep_size.push_back(size);
                    dst_off.push_back(dst_off.back() + size);
                }
                u += size;
            }
            c_ptr.push_back((int64_t)c_col.size());
        }
        DevVec<int64_t> d_keep, d_dst;
        DevVec<int32_t> d_size;
        DevVec<unsigned char> d_cval;
        CUDA_TRY(d_keep.put(keep_src, s), "upload");
        CUDA_TRY(d_dst.put(dst_off, s), "upload");
        CUDA_TRY(d_size.put(keep_size, s), "upload");
        CUDA_TRY(d_cval.alloc((size_t)dst_off.back() * es), "alloc result values");
        CUDA_TRY(launch_compact(f64, (int64_t)c_col.size(), d_keep.p, d_dst.p, d_size.p, d_val.p, d_cval.p, s),
                 "compaction");
        return vbcsr_create(Cout, nbr, nbc, A->row_b.data(), B->col_b.data(), c_ptr.data(), c_col.data(), d_cval.p,
                            A->dtype, 1, stream);
    } catch (const std::bad_alloc &) {
        return fail(VBCSR_ERR_NO_MEMORY, "host allocation in the block product");
    }
}

// ---------------------------------------------------------------------------
// inspection and control

extern "C" int vbcsr_get_info(const vbcsr_t *A, vbcsr_info_t *out) {
    if (!A || !out) return fail(VBCSR_ERR_INVALID_ARG, "NULL argument");
    out->n_brows = A->n_brows;
    out->n_bcols = A->n_bcols;
    out->n_rows = A->n_rows;
    out->n_cols = A->n_cols;
    out->nblk = A->nblk;
    out->nnz = A->nnz;
    out->panel_elems = A->panel_elems;
    out->device_bytes = A->device_bytes;
    out->dtype = A->dtype;
    out->n_shape_classes = (int32_t)A->cls_bi.size();
    out->n_row_classes = (int32_t)A->fwd_buckets.size();
    out->n_structs = A->n_structs;
    out->backend = A->backend;
    out->reserved = 0;
    return VBCSR_OK;
}

extern "C" int vbcsr_get_pattern(const vbcsr_t *A, int32_t *row_bsize, int32_t *col_bsize, int64_t *block_row_ptr,
                                 int32_t *block_col_idx) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (row_bsize) std::copy(A->row_b.begin(), A->row_b.end(), row_bsize);
    if (col_bsize) std::copy(A->col_b.begin(), A->col_b.end(), col_bsize);
    if (block_row_ptr) std::copy(A->h_rowptr.begin(), A->h_rowptr.end(), block_row_ptr);
    if (block_col_idx) std::copy(A->h_ucol.begin(), A->h_ucol.end(), block_col_idx);
    return VBCSR_OK;
}

extern "C" int vbcsr_shape_classes(const vbcsr_t *A, int32_t *bi, int32_t *bj, int64_t *count, int32_t cap) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (cap < 0 || (cap > 0 && (!bi || !bj || !count))) return fail(VBCSR_ERR_INVALID_ARG, "output arrays");
    const int32_t n = (int32_t)A->cls_bi.size();
    for (int32_t c = 0; c < n && c < cap; ++c) {
        bi[c] = A->cls_bi[c];
        bj[c] = A->cls_bj[c];
        count[c] = A->cls_count[c];
    }
    return n;
}

static bool valid_kc(int kc) { return kc == 0 || kc == 1 || kc == 2 || kc == 4 || kc == 8 || kc == 16 || kc == 32; }
static bool valid_warps(int w) { return w == 0 || w == 1 || w == 2 || w == 4 || w == 8; }

extern "C" int vbcsr_set_tuning(vbcsr_t *A, int32_t kc, int32_t warps) {
    return vbcsr_set_bucket_tuning(A, 0, kc, warps);
}

extern "C" int vbcsr_set_bucket_tuning(vbcsr_t *A, int32_t B, int32_t kc, int32_t warps) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (B < 0 || B > kMaxB) return fail(VBCSR_ERR_INVALID_ARG, "row count %d outside [0, %d]", B, kMaxB);
    if (!valid_kc(kc)) return fail(VBCSR_ERR_INVALID_ARG, "kc = %d", kc);
    if (!valid_warps(warps)) return fail(VBCSR_ERR_INVALID_ARG, "warps = %d", warps);
    for (int b = (B ? B : 1); b <= (B ? B : kMaxB); ++b) {
        A->kc_b[b] = kc;
        A->warps_b[b] = warps;
    }
    return VBCSR_OK;
}

extern "C" int vbcsr_set_schedule(vbcsr_t *A, int32_t schedule, int32_t persist_warps) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (schedule < 0 ||
        schedule > (VBCSR_SCHED_PERSISTENT | VBCSR_SCHED_MMA_STAGED | VBCSR_SCHED_NO_CSR | VBCSR_SCHED_NO_RING |
                    VBCSR_SCHED_NO_FPIPE))
        return fail(VBCSR_ERR_INVALID_ARG, "schedule %d", schedule);
    if (!valid_warps(persist_warps)) return fail(VBCSR_ERR_INVALID_ARG, "warps = %d", persist_warps);
    A->schedule = schedule;
    A->persist_warps = persist_warps;
    return VBCSR_OK;
}

extern "C" int vbcsr_get_tuning(const vbcsr_t *A, int32_t *kc_by_b, int32_t *warps_by_b, int32_t *schedule,
                                int32_t *persist_warps) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    for (int b = 0; b <= kMaxB; ++b) {
        if (kc_by_b) kc_by_b[b] = A->kc_b[b];
        if (warps_by_b) warps_by_b[b] = A->warps_b[b];
    }
    if (schedule) *schedule = A->schedule;
    if (persist_warps) *persist_warps = A->persist_warps;
    return VBCSR_OK;
}

// Mean device time of `reps` runs of one product configuration (ms), or < 0.
static double time_product(vbcsr_t *A, bool trans, int64_t k, const void *X, int64_t ldx, void *Y, int64_t ldy,
                           int precision, cudaStream_t s, int reps) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.0; }
    double ms = -1.0;
    if (run_product(A, trans, k, 1.0, X, ldx, 0.0, Y, ldy, nullptr, precision, s) == VBCSR_OK) {
        cudaEventRecord(e0, s);
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r)
            ok = run_product(A, trans, k, 1.0, X, ldx, 0.0, Y, ldy, nullptr, precision, s) == VBCSR_OK;
        cudaEventRecord(e1, s);
        float t = 0.f;
        if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
            ms = t / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

extern "C" int vbcsr_autotune(vbcsr_t *A, int transpose, int64_t k, const void *X, int64_t ldx, void *Y,
                              int64_t ldy, int precision, int32_t flags, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (transpose != 0 && transpose != 1) return fail(VBCSR_ERR_INVALID_ARG, "transpose must be 0 or 1");
    if (k < 1) return fail(VBCSR_ERR_INVALID_ARG, "k must be >= 1");
    if (precision != VBCSR_PREC_NATIVE &&
        !((precision == VBCSR_PREC_F32 || precision == VBCSR_PREC_DF32) && A->dtype == VBCSR_F64)) {
        // tensor-core kernels: no per-row-count tile; choose the forward variant
        if (precision < VBCSR_PREC_NATIVE || precision > VBCSR_PREC_DF32)
            return fail(VBCSR_ERR_INVALID_ARG, "precision %d", precision);
        if (transpose) return VBCSR_OK;
        cudaStream_t s = (cudaStream_t)stream;
        const int keep = A->schedule;
        A->schedule = keep & ~VBCSR_SCHED_MMA_STAGED;
        const double t_plain = time_product(A, false, k, X, ldx, Y, ldy, precision, s, 3);
        A->schedule = keep | VBCSR_SCHED_MMA_STAGED;
        const double t_staged = time_product(A, false, k, X, ldx, Y, ldy, precision, s, 3);
        if (t_plain < 0 || t_staged < 0) {
            A->schedule = keep;
            return fail(VBCSR_ERR_CUDA, "autotune trial failed: %s", g_detail.c_str());
        }
        A->schedule = t_staged < t_plain ? (keep | VBCSR_SCHED_MMA_STAGED) : (keep & ~VBCSR_SCHED_MMA_STAGED);
        return VBCSR_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool trans = transpose == 1;
    const int reps = 3;
    const int kcs[] = {1, 2, 4, 8, 16, 32};
    const int wss[] = {2, 4, 8};
    const int kc_auto = auto_kc(k);
    // 1) per row count: the column tile and CTA width of its bucket launch
    const int saved_schedule = A->schedule;
    // the tensor-core variant and the scalar-kernel opt-out are the caller's, not tuned here
    const int mma_bit =
        saved_schedule & (VBCSR_SCHED_MMA_STAGED | VBCSR_SCHED_NO_CSR | VBCSR_SCHED_NO_RING | VBCSR_SCHED_NO_FPIPE);
    A->schedule = VBCSR_SCHED_BUCKETED | mma_bit;
    const std::vector<Bucket> &buckets = trans ? A->adj_buckets : A->fwd_buckets;
    int keep_kc[kMaxB + 1], keep_w[kMaxB + 1];
    memcpy(keep_kc, A->kc_b, sizeof(keep_kc));
    memcpy(keep_w, A->warps_b, sizeof(keep_w));
    for (const Bucket &b : buckets) {
        double best = 1e30;
        int bkc = 0, bw = 0;
        // time this bucket alone: other buckets get an empty share by pointing their
        // tiles at the auto choice (their time is a constant offset)
        for (int kc : kcs) {
            if (kc > kc_auto) continue;
            for (int w : wss) {
                A->kc_b[b.B] = kc;
                A->warps_b[b.B] = w;
                const double ms = time_product(A, trans, k, X, ldx, Y, ldy, precision, s, reps);
                if (ms < 0) {
                    memcpy(A->kc_b, keep_kc, sizeof(keep_kc));
                    memcpy(A->warps_b, keep_w, sizeof(keep_w));
                    A->schedule = saved_schedule;
                    return fail(VBCSR_ERR_CUDA, "autotune trial failed: %s", g_detail.c_str());
                }
                if (ms < best) { best = ms; bkc = kc; bw = w; }
            }
        }
        A->kc_b[b.B] = bkc;
        A->warps_b[b.B] = bw;
    }
    const double t_bucketed = time_product(A, trans, k, X, ldx, Y, ldy, precision, s, reps);
    // 2) the persistent launch with those tiles: its CTA width, then the faster schedule
    int schedule = VBCSR_SCHED_BUCKETED, pw = 0;
    double best = t_bucketed;
    if (!(flags & VBCSR_TUNE_NO_PERSISTENT)) {
        A->schedule = VBCSR_SCHED_PERSISTENT | mma_bit;
        for (int w : wss) {
            A->persist_warps = w;
            const double ms = time_product(A, trans, k, X, ldx, Y, ldy, precision, s, reps);
            if (ms >= 0 && ms < best) { best = ms; schedule = VBCSR_SCHED_PERSISTENT; pw = w; }
        }
    }
    A->schedule = schedule | mma_bit;
    A->persist_warps = pw;
    return VBCSR_OK;
}

extern "C" int vbcsr_check(vbcsr_t *A, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamSynchronize(s), "synchronize");
    int h = 0;
    CUDA_TRY(cudaMemcpy(&h, A->err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (h != 0) {
        CUDA_TRY(cudaMemset(A->err, 0, sizeof(int)), "clear error word");
        return fail(VBCSR_ERR_DEVICE_CHECK, "device self-check code %d", h);
    }
    return VBCSR_OK;
}

// ---------------------------------------------------------------------------
// Chebyshev moments without a caller-provided work buffer
//
// For callers that cannot allocate device memory when they need the moments:
// code whose device memory is owned by another allocator (a host application
// or framework that reserves the free memory up front), or a loop that must
// not allocate once it runs. Such a caller creates the operator once at
// start-up and later calls this entry point, which allocates nothing: the two
// work panels of the recurrence live in the fixed array below, which every
// GPU that loads the library holds until the process exits. A mixed-precision
// mode also needs the handle's copies of the values and its converted-X
// buffers; those are built by an ordinary call, so this entry point only runs
// a mode whose buffers an earlier call on the handle already made large enough.

static constexpr int64_t kNoAllocPanelElems = int64_t(1) << 20;   // real elements per panel, at most
static __device__ __align__(256) double g_cheb_scratch[2 * kNoAllocPanelElems];   // 16 MiB

extern "C" int vbcsr_chebyshev_noalloc(vbcsr_t *A, int64_t k, const double *R, int64_t ldr, int64_t n_moments,
                                       double *moments, int precision, void *stream) {
    if (!A) return fail(VBCSR_ERR_INVALID_ARG, "handle is NULL");
    if (k < 1) return fail(VBCSR_ERR_INVALID_ARG, "k must be >= 1");
    if (A->dtype != VBCSR_F64 && A->dtype != VBCSR_C128)
        return fail(VBCSR_ERR_UNSUPPORTED, "the recurrence needs an FP64 or complex operator");
    if (precision < VBCSR_PREC_NATIVE || precision > VBCSR_PREC_DF32)
        return fail(VBCSR_ERR_INVALID_ARG, "precision %d", precision);
    // a complex panel holds two doubles per element
    const int64_t cw = A->dtype == VBCSR_C128 ? 2 : 1;
    if (A->n_rows > kNoAllocPanelElems / (k * cw))
        return fail(VBCSR_ERR_UNSUPPORTED,
                    "n_rows * k%s = %lld * %lld exceeds the fixed work area of %lld doubles per panel",
                    cw == 2 ? " * 2 (complex)" : "", (long long)A->n_rows, (long long)k,
                    (long long)kNoAllocPanelElems);
    if (precision != VBCSR_PREC_NATIVE && A->dtype == VBCSR_F64) {
        // the mode's value copy and converted-X buffers must exist already
        const ModePlan mp = plan_mode(A, false, k, precision);
        bool ready = mode_buffers_ready(A, mp, A->n_cols, k);
        if (ready && n_moments > 1 && fused_x_applies(A, mp)) {
            const size_t panel = (size_t)A->n_rows * (size_t)k;
            ready = (mp.xkind == kXPlanes || mp.xkind == kXF32P)
                        ? A->xbp_elems >= 4 * (size_t)A->n_rows * (size_t)pipe_ldp(k)
                  : mp.xkind == kXSplit  ? A->xbf_elems >= 2 * panel
                                         : A->xconv_elems >= 2 * panel;
        }
        if (!ready)
            return fail(VBCSR_ERR_UNSUPPORTED,
                        "precision %d needs buffers this handle has not built yet: make one vbcsr_chebyshev "
                        "call in this precision with at least %lld columns first",
                        precision, (long long)k);
    }
    // set-up, once per device: host code cannot use g_cheb_scratch as a device
    // address, so ask the runtime for it with that device current
    static std::mutex mu;
    static std::map<int, double *> addr;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    double *work = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = addr.find(dev);
        if (it == addr.end()) {
            void *p = nullptr;
            CUDA_TRY(cudaGetSymbolAddress(&p, g_cheb_scratch), "cudaGetSymbolAddress of the work area");
            it = addr.emplace(dev, static_cast<double *>(p)).first;
        }
        work = it->second;
    }
    // every element of the work panels that the recurrence reads is written
    // earlier in the same call, so nothing has to be cleared first
    return vbcsr_chebyshev(A, k, R, ldr, n_moments, moments, work, nullptr, 0, precision, stream);
}
