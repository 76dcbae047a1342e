// Internal declarations shared by the library's translation units.
//
// Device data layout of a handle (built once by the planner in api.cu):
//
//  * Value pages. Block row i is stored as one dense row-major "panel"
//    P_i of b_i rows and Kp_i columns: its stored blocks side by side in
//    increasing column order (K_i = sum_{j in J(i)} b_j columns, zero-padded
//    to Kp_i = roundup(K_i, 8) so that every panel row starts 64-byte aligned
//    in FP64 and 32-byte aligned in FP32; roundup(K_i, 4) for scalar operators,
//    16-byte aligned rows). Panels are laid out grouped by row
//    height b_i, so each row class is one contiguous page (the shape-grouped
//    pages of Sec. III.B). Then Y_i = P_i * X[g_i, :], where g_i lists the X
//    row of every panel column.
//  * Plan block list ("fl_*", one entry per stored block, row-major order with
//    columns sorted): X row c_j of its first column, its first panel column,
//    b_j, the user (packed-order) value offset, the panel element of its
//    (0, 0) entry, the panel stride and b_i.
//  * Transposed list ("tl_*", one entry per stored block, grouped by block
//    column, rows increasing): what the adjoint needs to walk column j.
//  * Work items: one warp task = up to 16 consecutive output rows of one block
//    row (forward) or block column (adjoint); items are bucketed by their row
//    count B so that each bucket runs as one launch of a kernel specialised
//    for B.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace vbcsr {

constexpr int kMaxB = 16;        // rows per work item
constexpr int kPadK = 8;         // panel width padding (elements)
constexpr int kPadKScalar = 4;   // the same for scalar (CSR-backend) operators
constexpr int kKMax = 512;       // virtual columns staged in shared memory per pass
constexpr int kPartialsCap = 1 << 16;
// tensor-core precision modes (the values of their vbcsr_precision codes), and
// the BF16X2 forward kernel on operands split once into packed bf16 (hi, lo)
// words (an internal launch mode, not a precision code)
constexpr int kTF32 = 2, kTF32X3 = 3, kBF16X2 = 4, kBF16X2Presplit = 16;
// below this many columns the tensor-core modes of an FP64 operator run their
// piece products on the CUDA cores (an MMA tile would be mostly padding)
constexpr int kSplitFmaMaxK = 2;

// One warp task.
struct WorkItem {
    int64_t vbase;   // forward: panel element of (first row of the item, column 0)
    int64_t yrow;    // first scalar output row
    int64_t lbegin;  // first entry in the plan block list (forward) / transposed list (adjoint)
    int32_t nlist;   // entries in that list
    int32_t K;       // virtual columns: K_i (forward) / sum of b_i over the column's blocks (adjoint)
    int32_t Kp;      // forward: panel row stride; adjoint: first row q0 inside the block column
    int32_t B;       // output rows of the item (1..16)
};

struct FwdList {
    const int32_t *xrow;   // c_j
    const int32_t *pcol;   // first panel column of the block
    const int32_t *w;      // b_j
};

struct AdjList {
    const int64_t *pbase;  // panel element of H_ij[0, 0]
    const int32_t *kp;     // panel stride of row i
    const int32_t *bi;     // b_i
    const int32_t *xrow;   // r_i
    const int32_t *vcol;   // first virtual column of the entry inside its block column
};

// Arguments of one product launch (one bucket of work items).
struct ProdArgs {
    const WorkItem *items;
    int64_t n_items;
    const void *values;     // panel values (FP64 or FP32 copy)
    FwdList fl;
    AdjList tl;
    int64_t k;
    int kc;                 // output columns per warp pass (power of two <= 32)
    double alpha, beta, gamma;
    float alpha32, beta32, gamma32;   // the same rounded to FP32 once on the host (FP32 epilogues)
    int beta_nz, gamma_nz;  // beta != 0, gamma != 0 (tested once on the host, not per element)
    const void *X; int64_t ldx;
    void *Y; int64_t ldy;
    const void *Z; int64_t ldz;
    const void *R; int64_t ldr;
    double *partials;       // per-CTA dot partials (NULL: no dot)
    double *item_partials;  // persistent launch: each item's dot written at its index (fixed-order
                            // reduction afterwards, whatever order the warps took the items in)
    int64_t x_rows;         // rows of X (bounds check)
    int *err;               // device error word
    int debug_checks;
    int grid;               // CTAs
    int warps;              // warps per CTA
    // persistent launch only
    long long *queue;       // device work counter, zero at launch (NULL: round-robin)
    uint64_t kc_log2_by_b;  // 3 bits per row count B = 1..16: log2 of its column tile
    int mma_staged;         // tensor-core forward: 1 = value panels staged in shared memory
    int value_ring;         // CUDA-core forward, FP32 values, k >= 4: read them through the ring
    void *xs_out;           // tensor-core forward (plain kernels) only, or NULL: every output
                            // element is also written here, in the form the kernel reads X
                            // (FP32 or the packed bf16 pieces of BF16X2, [rows of Y, k] with
                            // leading dimension k; the bf16 hi / lo planes of the pipelined
                            // BF16X2 kernel, leading dimension ldx, planes xs_plane apart), so
                            // that the next Chebyshev step needs no conversion pass
    int64_t xs_plane;       // pipelined BF16X2 kernel: elements between the hi and lo planes of xs_out
    int64_t v_plane;        //   ... of the value planes
    int64_t x_plane;        //   ... of the X planes (X row stride: ldx)
    __host__ __device__ int kc_of(int B) const { return 1 << ((kc_log2_by_b >> (3 * B)) & 7); }
};

// alpha, beta, gamma in an epilogue's type: the FP32 copies for FP32 outputs,
// so that no element pays an FP64 conversion
template <typename TX>
struct EpiScalars {
    TX alpha, beta, gamma;
};
template <typename TX>
__device__ __forceinline__ EpiScalars<TX> epi_scalars(const ProdArgs &a) {
    if constexpr (std::is_same<TX, float>::value) return {a.alpha32, a.beta32, a.gamma32};
    else return {(TX)a.alpha, (TX)a.beta, (TX)a.gamma};
}

// Kernel families (defined in spmm_fma_*.cu and spmm_mma.cu). B = 0 selects
// the persistent launch over items of every row count.
// value/accumulate/X types: f64 = <double,double,double>; f32 = <float,float,float>;
// f32_on_f64 = <float,float,double> (FP32 arithmetic on an FP64 operator).
cudaError_t launch_fma_f64(int B, bool trans, const ProdArgs &a, cudaStream_t s);
cudaError_t launch_fma_f32(int B, bool trans, const ProdArgs &a, cudaStream_t s);
cudaError_t launch_fma_f32_on_f64(int B, bool trans, const ProdArgs &a, cudaStream_t s);
// double-FP32 arithmetic on (hi, lo) FP32 pairs of an FP64 operator and X, FP64 epilogue
// narrow: the persistent forward kernel with two columns per lane for every row
// count (for operators with many row counts)
cudaError_t launch_fma_df(int B, bool trans, const ProdArgs &a, cudaStream_t s, bool narrow);
cudaError_t launch_split_df(int64_t rows, int64_t k, const double *in, int64_t ld, float2 *out, cudaStream_t s);
// mode: 2 = TF32, 3 = TF32X3, 4 = BF16X2 (vbcsr_precision values); xdouble: X/Y are FP64
cudaError_t launch_mma(int mode, bool xdouble, bool trans, const ProdArgs &a, cudaStream_t s);
// Tensor-core forward of an FP64 operator pipelined through shared memory (spmm_mma_pipe.cu):
// mode kBF16X2: values and X as bf16 hi / lo planes; kTF32 / kTF32X3: the FP32 copy of the
// values and X as FP32; X rows pipe_ldp(k) elements apart in either form
cudaError_t launch_mma_pipe(int mode, const ProdArgs &a, cudaStream_t s);
const void *mma_pipe_kernel_ptr(int mode, int64_t k);
size_t mma_pipe_smem_bytes(int mode, int64_t k, int warps);
int64_t pipe_ldp(int64_t k);
// FP32-value forward product on the CUDA cores pipelined through shared memory (k >= 8;
// X rows 16-byte aligned: ldx a multiple of 4); ydouble: FP64 Y (the F32 mode of an FP64 operator)
cudaError_t launch_fma32_pipe(bool ydouble, const ProdArgs &a, cudaStream_t s);
const void *fma32_pipe_kernel_ptr(int64_t k, bool ydouble);
size_t fma32_pipe_smem_bytes(int64_t k, int warps);

// Scalar (all 1 x 1 blocks) operators: L lanes per row (2, 4 or 8 for the
// FP64 and double-FP32 kinds, 4, 8, 16 or 32 for the FP32 ones; csr_lane_class
// 0 and 1).
enum CsrKind {
    kCsrF64 = 0, kCsrF32 = 1, kCsrF32OnF64 = 2, kCsrDF = 3,
    kCsrSplitTF32 = 4, kCsrSplitTF32X3 = 5, kCsrSplitBF16X2 = 6   // split.cuh, FP64 Y
};
int csr_lane_class(int kind);
cudaError_t launch_csr(int kind, int L, const ProdArgs &a, cudaStream_t s);
const void *csr_kernel_ptr(int kind, int L, int64_t k);

// Thresholded block sparse product (spgemm.cu)
struct SpgemmArgs {
    int64_t n_out;              // output blocks
    const int64_t *out_pbeg;    // [n_out + 1] range of each output block in the product list
    const int64_t *out_uoff;    // packed-order offset of each output block
    const int32_t *out_bi, *out_bj;
    const int64_t *pa, *pb;     // panel element of A_ik[0,0] / B_kj[0,0] of every product
    const int32_t *kpa, *kpb;   // their panel strides
    const int32_t *bk;          // inner block size b_k
    const void *A, *B;          // panels
    void *C;                    // packed-order output
    double *norms;              // [n_out] Frobenius norm of every output block
};
// Symbolic stage of the block product on the device (Eq. 3). Per block row i
// of A, the candidates C_ij reached by A_ik B_kj, their norm bounds
// sum_k |A_ik| |B_kj| accumulated in increasing plan order of k, the kept set
// (bound >= eps, in increasing j), and for each kept block its product list
// ordered by inner size b_k, then by k. Pass 1 counts (per row: kept blocks,
// products, values); pass 2 writes at the row offsets the host scanned.
struct SymArgs {
    int64_t n_rows;             // rows to process: rows[t] when given, else t
    const int64_t *rows;
    const int64_t *a_rowptr, *b_rowptr;   // plan block range of every block row
    const int32_t *a_col, *b_col;         // block column of every plan block
    const double *a_norm, *b_norm;        // Frobenius norm of every plan block
    const int32_t *a_w;                   // b_k of every plan block of A
    const int64_t *a_pbase, *b_pbase;     // panel element [0, 0] of every plan block
    const int32_t *a_kp, *b_kp;           // panel stride of every plan block
    const int32_t *a_rowsize;             // b_i of every block row of A
    const int32_t *b_colsize;             // b_j of every block column of B
    double eps;
    // workspace: a shared-memory table per warp (global == 0), or a global slice
    // per listed row at ws_off[t] with table size ws_h[t] and capacity ws_cap[t]
    int global_ws;
    unsigned char *ws;
    const int64_t *ws_off;
    const int32_t *ws_h, *ws_cap;
    // pass 1 outputs
    int64_t *cnt_out, *cnt_prod, *cnt_val;   // per block row
    int32_t *overflow;                       // per block row: more candidates than the table holds
    // pass 2: row offsets (inputs) and the lists (outputs)
    const int64_t *off_out, *off_prod, *off_val;
    int32_t *out_col, *out_bi, *out_bj;
    int64_t *out_uoff, *out_pbeg;
    int64_t *pa, *pb;
    int32_t *kpa, *kpb, *bk;
};
constexpr int kSymHash = 2048;   // shared-memory table slots per warp
constexpr int kSymCap = 512;     // candidates per row the shared-memory table holds
// workspace bytes of one row: bound (8 B), key and slot (4 B each) per table
// slot, candidate, kept index and cursor (4 B each) per candidate
__host__ __device__ constexpr size_t sym_ws_bytes(int h, int cap) {
    return (size_t)8 * cap + (size_t)8 * h + (size_t)12 * cap;
}
cudaError_t launch_spgemm_symbolic(int pass, const SymArgs &g, cudaStream_t s);
cudaError_t launch_block_norms(bool f64, int64_t nblk, const void *panel, const int64_t *pbase, const int32_t *kp,
                               const int32_t *bi, const int32_t *bj, double *out, cudaStream_t s);
cudaError_t launch_spgemm_numeric(bool f64, const SpgemmArgs &g, cudaStream_t s);
cudaError_t launch_compact(bool f64, int64_t n, const int64_t *keep_src, const int64_t *dst_off, const int32_t *size,
                           const void *src, void *dst, cudaStream_t s);

// Occupancy-derived CTA count cap (SMs x resident CTAs per SM); -1 when a CUDA
// query failed (the error stays pending for the caller to read).
int max_resident_ctas(const void *kernel, int threads, size_t smem);

// value ring of the FP32-value forward kernel: stages of kRingCols panel columns
// of up to 16 rows, per warp
constexpr int kRingStages = 3, kRingCols = 32;
constexpr int kRingBytes = kRingStages * 16 * kRingCols * 4;
size_t fma_smem_bytes(bool trans, int warps, bool ring = false);
// forward products of an FP64 operator in a tensor-core mode on the CUDA cores
cudaError_t launch_fma_split(int mode, const ProdArgs &a, cudaStream_t s);
const void *fma_split_kernel(int mode);
size_t mma_smem_bytes(bool trans, bool staged, int warps);

// Misc kernels (misc.cu).
struct SddmmArgs {
    const WorkItem *items;      // the forward work items (rows of a block row), in descending cost
    int64_t n_items;
    long long *queue;           // device work counter (zeroed by the launch)
    const int32_t *fl_xrow;     // c_j
    const int32_t *fl_pcol;     // first panel column of the block
    const int32_t *fl_w;        // b_j
    const int64_t *fl_uoff;     // packed-order offset of the block
    const int64_t *fl_pbase;    // panel element [0, 0] of the block
    int64_t k;
    double alpha, beta;
    const void *A; int64_t lda;
    const void *B; int64_t ldb;
    void *D;
};
cudaError_t launch_sddmm(bool f64, const SddmmArgs &a, cudaStream_t s);

// scatter (to_panel = true) or gather packed-order values <-> panels
// reciprocal-space sampling (Eq. 4) of a k-space handle into packed complex values
cudaError_t launch_ksample(int64_t nblk, int64_t n_edges, const int64_t *ks_ptr, const double *ks_shift,
                           const int64_t *ks_voff, const double *ks_vals, const int64_t *uoff, const int32_t *ub_n,
                           const double *kfrac, double2 *phase, double2 *out, cudaStream_t s);
// complex FP64 products (VBCSR_C128)
cudaError_t launch_fma_c128(int B, bool trans, const ProdArgs &a, cudaStream_t s);
const void *fma_c128_kernel(bool trans, bool persistent, int B);
// esize: 4 (FP32), 8 (FP64) or 16 (complex FP64) bytes per element
cudaError_t launch_permute_values(int esize, bool to_panel, int64_t nblk, const int64_t *uoff,
                                  const int64_t *pbase, const int32_t *kp, const int32_t *bi,
                                  const int32_t *bj, const void *user, void *panel, cudaStream_t s);
cudaError_t launch_convert_f64_to_f32(const double *in, float *out, int64_t n, cudaStream_t s);
// FP64 -> FP32 v -> one 32-bit word: bf16_rn(v) in the low half, bf16_rn(v - that) in the high half
cudaError_t launch_split_bf16(const double *in, uint32_t *out, int64_t n, cudaStream_t s);
// the same pieces as two planes: hi[i], lo[i] (values), and hi / lo[r * ldp + c] of an
// [rows, k] panel with leading dimension ld (X)
cudaError_t launch_split_bf16_planes(const double *in, uint16_t *hi, uint16_t *lo, int64_t n, cudaStream_t s);
cudaError_t launch_split_bf16_planes_panel(int64_t rows, int64_t k, const double *in, int64_t ld, uint16_t *hi,
                                           uint16_t *lo, int64_t ldp, cudaStream_t s);
cudaError_t launch_split_bf16_panel(int64_t rows, int64_t k, const double *in, int64_t ld, uint32_t *out,
                                    cudaStream_t s);
// out[rows, k] (leading dimension k) = FP32 of the FP64 panel in (leading dimension ld)
cudaError_t launch_convert_panel_f64_to_f32(int64_t rows, int64_t k, const double *in, int64_t ld, float *out,
                                            int64_t ldo,
                                            cudaStream_t s);
// out[0] = scale * sum(partials[0..n)) in a fixed order (set by n alone); long sums
// go through `scratch` (kDotScratch doubles, or NULL for the one-CTA sum)
constexpr int64_t kDotOneStage = 16384, kDotChunk = 4096, kDotScratch = 1024;
cudaError_t launch_finalize_dot(const double *partials, int64_t n, double scale, double *out, double *scratch,
                                cudaStream_t s);
// partials[b] = sum over CTA b of A .* B ([rows, k] panels); returns CTAs used in *n_used
cudaError_t launch_dot_panels(bool f64, int64_t rows, int64_t k, const void *A, int64_t lda,
                              const void *B, int64_t ldb, double *partials, int64_t cap,
                              int64_t *n_used, cudaStream_t s);
// Y = alpha X + beta Y on [rows, k] FP64 panels (beta == 0: Y not read)
cudaError_t launch_axpby(int64_t rows, int64_t k, double alpha, const double *X, int64_t ldx, double beta,
                         double *Y, int64_t ldy, cudaStream_t s);
// Gershgorin bounds over the forward items: out[0] = min, out[1] = max (device)
// real (FP64) or complex Hermitian (cplx) operators
cudaError_t launch_gershgorin(bool cplx, const WorkItem *items, int64_t n_items, const void *panel,
                              const int32_t *xrow, const int32_t *pcol, const int32_t *wd, double *partials,
                              int64_t cap, double *out, cudaStream_t s);
// panel <- (panel - c I) / d in place
cudaError_t launch_shift_scale(bool cplx, const WorkItem *items, int64_t n_items, void *panel, const int32_t *xrow,
                               const int32_t *pcol, const int32_t *wd, double c, double d, cudaStream_t s);
// kernel polynomial method
cudaError_t launch_kpm_fixup(double *mu, int64_t M, cudaStream_t s);
cudaError_t launch_kpm_dos(const double *mu, int64_t M, int jackson, const double *x, int64_t nx, double *out,
                           cudaStream_t s);
// out = {E[lo], E[hi]} of the below-threshold run around the grid point nearest ref, or NaN, NaN
cudaError_t launch_kpm_gap(const double *E, const double *D, int64_t n, double ref, double thr, double *out,
                           cudaStream_t s);
// dst[rows, k] (ld ldd) = src (ld lds), FP64
cudaError_t launch_copy_panel(int64_t rows, int64_t k, const double *src, int64_t lds, double *dst,
                              int64_t ldd, cudaStream_t s);

}  // namespace vbcsr
