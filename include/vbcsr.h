/*
 * vbcsr.h -- C ABI of the GB300 (sm_103a) variable-block sparse library.
 *
 * A VBCSR operator H has n_brows block rows and n_bcols block columns. Block
 * row i holds b_i = row_bsize[i] scalar rows starting at r_i = sum_{i'<i} b_i';
 * block column j holds b_j = col_bsize[j] scalar columns starting at
 * c_j = sum_{j'<j} b_j'. The stored blocks of row i are the columns
 * J(i) = block_col_idx[block_row_ptr[i] .. block_row_ptr[i+1]); block (i, j) is a
 * dense b_i x b_j matrix (the variable-block CSR format of Sec. II.A of the
 * paper "Accelerating Atom Simulations with Variable-Block Sparse Matrix
 * Library").
 *
 * User value order ("packed order"): blocks in block_row_ptr / block_col_idx
 * order, each block row-major. Panels X and Y are row-major [rows, k] with a
 * leading dimension ld >= k, in the matrix dtype.
 *
 * Conventions shared by every entry point:
 *  - Return value: VBCSR_OK (0) or a negative vbcsr_status. On error a
 *    thread-local message is available from vbcsr_last_error_detail().
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Compute calls
 *    are asynchronous on that stream and never synchronise the host, except
 *    vbcsr_check and the host-buffer calls that say so.
 *  - Every argument is validated on the host before anything is launched;
 *    an invalid call launches nothing and leaves its outputs untouched.
 *  - Pointers are borrowed for the duration of the call only. Device pointers
 *    must belong to the device that was current at vbcsr_create.
 *  - A handle may be used from one host thread at a time, and its compute
 *    calls must not overlap on the GPU (issue them on one stream, or order the
 *    streams): the handle's work counter, converted-X buffers and dot partials
 *    are shared by its calls.
 */
#ifndef VBCSR_H
#define VBCSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vbcsr_matrix vbcsr_t;

typedef enum {
    VBCSR_OK = 0,
    VBCSR_ERR_INVALID_ARG = -1,   /* null pointer, negative size, ld < k, bad enum   */
    VBCSR_ERR_PATTERN = -2,       /* bad block_row_ptr, column out of range, duplicate
                                     block in a row, block size < 1 or too large     */
    VBCSR_ERR_CUDA = -3,          /* a CUDA runtime call failed                       */
    VBCSR_ERR_NO_MEMORY = -4,     /* device or host allocation failed                 */
    VBCSR_ERR_UNSUPPORTED = -5,   /* valid request outside what the library supports */
    VBCSR_ERR_DEVICE_CHECK = -6,  /* a kernel's self-check recorded an error          */
    VBCSR_ERR_ALIAS = -7          /* output overlaps an input that it may not alias   */
} vbcsr_status;

typedef enum {
    VBCSR_F64 = 0,                /* values, X and Y are double */
    VBCSR_F32 = 1,                /* values, X and Y are float  */
    VBCSR_C128 = 2                /* complex double: values, X and Y are interleaved
                                     (re, im) double pairs, leading dimensions count
                                     complex elements; alpha and beta stay real; the
                                     adjoint is the conjugate transpose (the dagger
                                     of Eq. 1); NATIVE precision only               */
} vbcsr_dtype;

/*
 * Arithmetic of the block products. X, Y, alpha, beta and the epilogue stay in
 * the matrix dtype in every mode; the mixed modes keep a copy of the values in
 * their own format (FP32; for BF16X2 on an FP64 operator one 32-bit word per
 * value holding its bf16 hi and lo pieces; for DF32 FP32 pairs), built on
 * first use and refreshed by vbcsr_set_values and vbcsr_shift_scale, and, for
 * an FP64 operator, convert X the same way once per call into a buffer the
 * handle owns (allocated on first use and grown when a call needs more;
 * growing it synchronises the stream). Mixed-mode calls on one handle
 * therefore must not overlap on the GPU.
 *  NATIVE  products and accumulation in the matrix dtype (FP64 FMA / FP32 FMA)
 *  F32     values and X rounded to FP32, FP32 FMA, FP32 accumulation
 *  TF32    one TF32 tensor-core product per block product, FP32 accumulation
 *  TF32X3  v = hi + lo with hi = tf32(v), lo = tf32(v - hi) for values and X;
 *          hi*hi + hi*lo + lo*hi on the tensor cores, FP32 accumulation
 *  BF16X2  the same split with bf16 pieces, FP32 accumulation
 *  DF32    FP64-accurate: values and X carried as pairs hi + lo of FP32
 *          numbers (48 significand bits), products with an exact leading
 *          part (fused multiply-add) and TwoSum accumulation on the FP32
 *          units; relative error a few 2^-48 of sum |h x|. FP64 operators
 *          only; operands must lie inside the FP32 exponent range
 *          (|v| in about [1e-30, 1e38]) for that accuracy.
 */
typedef enum {
    VBCSR_PREC_NATIVE = 0,
    VBCSR_PREC_F32 = 1,
    VBCSR_PREC_TF32 = 2,
    VBCSR_PREC_TF32X3 = 3,
    VBCSR_PREC_BF16X2 = 4,
    VBCSR_PREC_DF32 = 5
} vbcsr_precision;

/* Launch schedules of the CUDA-core products (vbcsr_set_schedule). */
typedef enum {
    VBCSR_SCHED_BUCKETED = 0,     /* one launch per work-item row count                */
    VBCSR_SCHED_PERSISTENT = 1,   /* one launch over all items, costliest first, warps
                                     taking items from a device work counter (default:
                                     no per-launch tail, which at large k is ~1 item
                                     per warp and dominates a launch of few waves)     */
    VBCSR_SCHED_MMA_STAGED = 2,   /* flag: the tensor-core forward kernel stages value
                                     panels in shared memory with bulk async copies   */
    VBCSR_SCHED_NO_CSR = 4,       /* flag: a CSR-backend operator uses the block-row
                                     kernels instead of the scalar kernel (which
                                     otherwise serves its forward products under
                                     either schedule)                                  */
    VBCSR_SCHED_NO_RING = 8,      /* flag: the CUDA-core forward kernel on FP32 values
                                     (FP32 operators, the F32 mode) reads them directly
                                     instead of through its ring of asynchronous
                                     shared-memory copies, which it otherwise uses at
                                     k >= 8 (one launch per row count, or with
                                     VBCSR_SCHED_NO_FPIPE)                             */
    VBCSR_SCHED_NO_FPIPE = 16     /* flag: the persistent launch on FP32 values at
                                     k >= 8 uses the CUDA-core kernel with per-lane
                                     output columns instead of the pipelined one (each
                                     lane a 4-row register tile fed from a ring of
                                     shared-memory stages of values and gathered X),
                                     which it otherwise uses when X rows are 16-byte
                                     aligned                                           */
} vbcsr_schedule;

/* Flags of vbcsr_autotune. */
#define VBCSR_TUNE_NO_PERSISTENT 1   /* keep the bucketed schedule */

typedef struct {
    int64_t n_brows, n_bcols;     /* block rows / block columns                      */
    int64_t n_rows, n_cols;       /* scalar rows / columns                           */
    int64_t nblk;                 /* stored blocks                                   */
    int64_t nnz;                  /* stored scalar entries (sum of b_i * b_j)        */
    int64_t panel_elems;          /* device value elements incl. alignment padding   */
    int64_t device_bytes;         /* device memory held by the handle                */
    int32_t dtype;                /* vbcsr_dtype                                     */
    int32_t n_shape_classes;      /* distinct (b_i, b_j) pairs among stored blocks   */
    int32_t n_row_classes;        /* distinct work heights used by the forward plan  */
    int32_t n_structs;            /* independent structures (1 unless batched)      */
    int32_t backend;              /* vbcsr_backend chosen from the block sizes       */
    int32_t reserved;
} vbcsr_info_t;

/*
 * Backend chosen at creation from the block sizes (Sec. II.B: scalar operators
 * map to CSR, a uniform basis to BSR, species-dependent bases to VBCSR):
 *  CSR    every block 1 x 1: the forward product (FP64 / FP32 arithmetic) runs
 *         a scalar kernel with several rows per warp
 *  BSR    every block b x b for one b > 1: the block-row kernels specialised
 *         for that b
 *  VBCSR  otherwise
 * Values, X and Y are laid out the same way for every backend.
 */
typedef enum {
    VBCSR_BACKEND_CSR = 0,
    VBCSR_BACKEND_BSR = 1,
    VBCSR_BACKEND_VBCSR = 2
} vbcsr_backend;

/* Optional fused epilogue of vbcsr_spmm_ex (all fields may be zero/NULL). */
typedef struct {
    double gamma;                 /* Y += gamma * Z after the product (Z ignored if 0) */
    const void *Z;                /* device, [rows of Y, k], may equal neither X nor Y */
    int64_t ldz;
    const void *R;                /* device, [rows of Y, k]; with dot_out set, the call
                                     also writes *dot_out = sum(R .* Y_new) in FP64    */
    int64_t ldr;
    double *dot_out;              /* device pointer to one double, or NULL             */
} vbcsr_epilogue_t;

/* ---- status -------------------------------------------------------------- */

/* Static, thread-safe description of a status code. */
const char *vbcsr_error_string(int status);
/* Message of the last failing call on this host thread ("" if none). */
const char *vbcsr_last_error_detail(void);

/* ---- construction -------------------------------------------------------- */

/*
 * Builds a handle from a VBCSR pattern and packed values (Sec. II.A; the
 * shape-class registry and shape-grouped value pages of Sec. III.B are built
 * here, once).
 *  n_brows, n_bcols  >= 0
 *  row_bsize[n_brows], col_bsize[n_bcols]   host, block sizes in [1, 4096]
 *  block_row_ptr[n_brows+1]   host, block_row_ptr[0] = 0, non-decreasing
 *  block_col_idx[nblk]        host, in [0, n_bcols), no duplicate in a row
 *                             (any order inside a row)
 *  values     packed order, nnz elements of `dtype`; host memory when
 *             values_on_device = 0, device memory when 1
 * The library copies everything it needs; the caller keeps ownership of its
 * buffers. The scalar sizes must stay below 2^31. Errors: INVALID_ARG,
 * PATTERN, NO_MEMORY, CUDA. The call synchronises `stream` before returning.
 */
int vbcsr_create(vbcsr_t **out, int64_t n_brows, int64_t n_bcols,
                 const int32_t *row_bsize, const int32_t *col_bsize,
                 const int64_t *block_row_ptr, const int32_t *block_col_idx,
                 const void *values, int dtype, int values_on_device, void *stream);

/*
 * Builds one handle over n_structs independent structures (a block-diagonal
 * operator), so that one launch serves all of them.
 *  struct_brow_offsets[n_structs+1], struct_bcol_offsets[n_structs+1]  host,
 *      first block row / block column of every structure (offsets[0] = 0,
 *      offsets[n_structs] = n_brows / n_bcols)
 *  block_col_idx holds column indices LOCAL to the structure of the row
 *  (0 .. its block-column count - 1); everything else as in vbcsr_create with
 *  global block rows. X and Y are the concatenated panels of all structures.
 */
int vbcsr_create_batched(vbcsr_t **out, int64_t n_structs,
                         const int64_t *struct_brow_offsets, const int64_t *struct_bcol_offsets,
                         const int32_t *row_bsize, const int32_t *col_bsize,
                         const int64_t *block_row_ptr, const int32_t *block_col_idx,
                         const void *values, int dtype, int values_on_device, void *stream);

/* Frees every device and host resource of the handle; NULL is accepted. The
   caller must make sure no work using the handle is still in flight. */
int vbcsr_destroy(vbcsr_t *A);

/* ---- values ---------------------------------------------------------------- */

/* Replaces all values (packed order, nnz elements of the matrix dtype; host
   when on_device = 0, else device) on the fixed pattern. Asynchronous on
   `stream` for device input; host input is staged and the call synchronises. */
int vbcsr_set_values(vbcsr_t *A, const void *values, int on_device, void *stream);

/* Copies all values out in packed order (host when on_device = 0, else device).
   Host output synchronises `stream`. */
int vbcsr_get_values(const vbcsr_t *A, void *values, int on_device, void *stream);

/* ---- products ---------------------------------------------------------------- */

/*
 * Y = alpha * H * X + beta * Y   (Sec. III.B, "Matrix multiplication": every
 * block row accumulates A_ij X_j over j in J(i)).
 *  X  device [n_cols, k], leading dimension ldx >= k
 *  Y  device [n_rows, k], leading dimension ldy >= k; Y must not overlap X
 *  beta == 0: Y is not read (NaN in Y does not propagate)
 *  alpha == 0: H and X are not read
 *  k == 0 or n_rows == 0: nothing is launched
 * Each output row block is written exactly once (no atomics).
 * Errors: INVALID_ARG, ALIAS, UNSUPPORTED (precision), NO_MEMORY, CUDA.
 */
int vbcsr_spmm(vbcsr_t *A, int64_t k, double alpha, const void *X, int64_t ldx,
               double beta, void *Y, int64_t ldy, int precision, void *stream);

/*
 * Y = alpha * H^T * X + beta * Y   (Eq. 1: Y_j += A_ij^dagger X_i for j in J(i);
 * values are real, so the dagger is a transpose). X is [n_rows, k], Y is
 * [n_cols, k]; otherwise as vbcsr_spmm. A transposed index of the pattern
 * (no value copy) lets every output row block be written once, without atomics.
 */
int vbcsr_spmm_adjoint(vbcsr_t *A, int64_t k, double alpha, const void *X, int64_t ldx,
                       double beta, void *Y, int64_t ldy, int precision, void *stream);

/*
 * vbcsr_spmm (transpose = 0) or vbcsr_spmm_adjoint (transpose = 1) with a
 * fused epilogue (may be NULL):
 *   Y = alpha * op(H) X + beta * Y + gamma * Z,   *dot_out = sum(R .* Y)
 * This is one step of the Chebyshev recurrence and of its reverse (adjoint)
 * recurrence in the kernel polynomial method of Sec. V. The dot product is
 * reduced in a fixed order (per work item under the persistent schedule, per
 * CTA otherwise), so repeated calls with the same tuning give the same bits.
 */
int vbcsr_spmm_ex(vbcsr_t *A, int transpose, int64_t k, double alpha, const void *X,
                  int64_t ldx, double beta, void *Y, int64_t ldy,
                  const vbcsr_epilogue_t *epilogue, int precision, void *stream);

/*
 * Pattern-sampled dense product, the gradient of <G, H X> with respect to the
 * stored values:
 *   D_ij[p, q] = alpha * sum_c Aop[r_i + p, c] * Bop[c_j + q, c] + beta * D_ij[p, q]
 * for every stored block (i, j), written in packed order.
 *  Aop  device [n_rows, k], lda >= k;  Bop  device [n_cols, k], ldb >= k
 *  D    device, nnz elements of the matrix dtype; beta == 0: D is not read
 * (This operation has no counterpart in the paper.)
 */
int vbcsr_sddmm(vbcsr_t *A, int64_t k, double alpha, const void *Aop, int64_t lda,
                const void *Bop, int64_t ldb, double beta, void *D, void *stream);

/*
 * Chebyshev moments of the kernel polynomial method (Sec. V) for an operator
 * already shifted and scaled to H~ with spectrum inside [-1, 1]:
 *   t_0 = R,  t_1 = H~ R,  t_{n+1} = 2 H~ t_n - t_{n-1},
 *   moments[n] = sum(R .* t_n) / (n_rows * k),   n = 0 .. n_moments - 1.
 * The recurrence and the moments are FP64 (matrix dtype F64, or C128 for a
 * complex Hermitian operator: R, work and the checkpoints are then complex,
 * the moment is Re sum(conj(R) .* t_n) / (n_rows * k), NATIVE precision); the
 * block products use `precision`.
 *  R        device [n_rows, k], ldr >= k (square operator: n_rows == n_cols)
 *  moments  device, n_moments doubles
 *  work     device, 2 * n_rows * k doubles (scratch panels)
 *  ckpt     device or NULL; when given with ckpt_every >= 1, the pairs
 *           (t_m, t_{m+1}) for m = 0, ckpt_every, 2*ckpt_every, ... (m+1 <
 *           n_moments) are stored consecutively, each panel n_rows * k doubles
 *           with leading dimension k: ceil((n_moments - 1) / ckpt_every) pairs.
 */
int vbcsr_chebyshev(vbcsr_t *Ht, int64_t k, const double *R, int64_t ldr, int64_t n_moments,
                    double *moments, double *work, double *ckpt, int64_t ckpt_every,
                    int precision, void *stream);

/*
 * Reverse-mode gradient of the moments of vbcsr_chebyshev with respect to the
 * stored values of H~ (packed order), given dL/dmu_n = grad_mu[n]:
 *   g_n = grad_mu[n] R / (n_rows * k),
 *   lam_{M-1} = g_{M-1},  lam_n = g_n + 2 H~^T lam_{n+1} - lam_{n+2}  (n >= 1),
 *   dL/dH~ = lam_1 t_0^T + sum_{n=1}^{M-2} 2 lam_{n+1} t_n^T   on the stored blocks,
 *   dvalues = dL/dH~ / d_scale.
 * When the handle holds H~ = (H - c I) / d made from an operator H by
 * vbcsr_shift_scale, d_scale = d gives the gradient with respect to the
 * stored values of H itself (the shift c is a constant and drops out);
 * d_scale = 1 gives dL/dH~.
 * The t_n are recomputed segment by segment from the checkpoint pairs that
 * vbcsr_chebyshev stored with the same ckpt_every, so memory stays at
 * O(ckpt_every) panels.
 *  grad_mu  device, n_moments doubles (copied to the host: the call
 *           synchronises `stream` once at its start)
 *  ckpt     device, as written by vbcsr_chebyshev
 *  d_scale  finite and nonzero
 *  dvalues  device, nnz doubles, overwritten
 *  work     device, (2 + 2 * ckpt_every) * n_rows * k doubles
 * (The adjoint recurrence has no counterpart in the paper; it differentiates
 * the kernel-polynomial moments of Sec. V.)
 */
int vbcsr_chebyshev_backward(vbcsr_t *Ht, int64_t k, const double *R, int64_t ldr, int64_t n_moments,
                             const double *grad_mu, const double *ckpt, int64_t ckpt_every, double d_scale,
                             double *dvalues, double *work, int precision, void *stream);

/* Damping kernels of vbcsr_kpm_dos. */
#define VBCSR_KPM_NO_KERNEL 0
#define VBCSR_KPM_JACKSON 1

/*
 * Kernel-polynomial moments mu_0 .. mu_{M-1} (Sec. V: the DOS of the InP
 * particles comes from KPM moments) for a SYMMETRIC operator already scaled
 * to H~, with half the products of vbcsr_chebyshev: t_0 = R, t_1 = H~ R,
 * t_{n+1} = 2 H~ t_n - t_{n-1} up to n = ceil(M/2) - 1 or so, and
 *   mu_0 = <R, R> / (N k),  mu_1 = <t_1, R> / (N k),
 *   mu_{2n} = 2 <t_n, t_n> / (N k) - mu_0,  mu_{2n+1} = 2 <t_{n+1}, t_n> / (N k) - mu_1,
 * from T_{2n} = 2 T_n^2 - T_0 and T_{2n+1} = 2 T_{n+1} T_n - T_1 (these need
 * H~ = H~^T, or H~ = H~^dagger for a C128 operator; for a non-symmetric operator
 * use vbcsr_chebyshev). Arguments as
 * vbcsr_chebyshev: R device [n_rows, k] (ldr), moments device [M], work device
 * 2 * n_rows * k doubles; recurrence and moments FP64, products in `precision`.
 */
int vbcsr_kpm_moments(vbcsr_t *Ht, int64_t k, const double *R, int64_t ldr, int64_t n_moments,
                      double *moments, double *work, int precision, void *stream);

/*
 * Density of states from KPM moments at scaled energies x in (-1, 1):
 *   dos[i] = [g_0 mu_0 + 2 sum_{n>=1} g_n mu_n T_n(x_i)] / (pi sqrt(1 - x_i^2)),
 * g the Jackson damping factors (kernel = VBCSR_KPM_JACKSON,
 *   g_n = [(M - n + 1) cos(pi n / (M + 1)) + sin(pi n / (M + 1)) cot(pi / (M + 1))] / (M + 1))
 * or 1 (VBCSR_KPM_NO_KERNEL). In the energy of H = c + d H~, the density is
 * dos / d at E = c + d x. moments, x, dos: device arrays of n_moments, n_x,
 * n_x doubles. Needs no handle.
 */
int vbcsr_kpm_dos(const double *moments, int64_t n_moments, int kernel, const double *x, int64_t n_x,
                  double *dos, void *stream);

/*
 * Band gap read off a density of states (Sec. V takes the band gaps of the
 * InP particles from their KPM densities of states; the criterion is a DOS
 * threshold). On an energy grid energies[0 .. n) (increasing) with densities
 * dos[0 .. n): i0 is the grid point nearest `reference` (the smallest index
 * on a tie), and the gap is the widest run lo <= i0 <= hi of consecutive grid
 * points whose DOS is below `threshold` (dos < threshold; NaN is not below):
 *   out[0] = energies[lo], out[1] = energies[hi],
 * where lo - 1 and hi + 1 are outside the grid or not below the threshold;
 * out = {NaN, NaN} when dos[i0] is not below the threshold (the reference
 * lies inside a band). energies, dos: device arrays of n >= 1 doubles (the
 * grid and vbcsr_kpm_dos's output); out: device array of 2 doubles. One CTA,
 * asynchronous on `stream`. Errors: INVALID_ARG (n < 1, NULL, NaN reference
 * or threshold), CUDA.
 */
int vbcsr_kpm_gap(const double *energies, const double *dos, int64_t n, double reference, double threshold,
                  double *out, void *stream);

/*
 * Spectral bounds for the kernel polynomial method (Sec. V needs H scaled so
 * that its spectrum lies in [-1, 1]): Gershgorin discs over scalar rows,
 *   bounds[0] = min_r (H_rr - sum_{c != r} |H_rc|),
 *   bounds[1] = max_r (H_rr + sum_{c != r} |H_rc|),
 * written to the device array `bounds` (2 doubles). Square FP64 operator, or
 * C128 for a complex Hermitian one (H_rr its real part, |H_rc| the modulus).
 */
int vbcsr_gershgorin(vbcsr_t *A, double *bounds, void *stream);

/*
 * Replaces the stored values by those of H~ = (H - c I) / d (c subtracted on
 * the scalar diagonal, every entry divided by d), in place, for the Chebyshev
 * recurrence; with c = (E+ + E-)/2 and d slightly above (E+ - E-)/2 from
 * vbcsr_gershgorin the spectrum of H~ lies inside [-1, 1]. Square FP64 or
 * C128 operator (c comes off the real part of the diagonal); d must be
 * nonzero and finite.
 */
int vbcsr_shift_scale(vbcsr_t *A, double c, double d, void *stream);

/*
 * vbcsr_chebyshev without the `work` argument (and without checkpoints), for
 * callers that cannot allocate device memory at the point where they need
 * the moments: code whose device memory belongs to another allocator (a host
 * application or framework that reserves the free memory up front) or a loop
 * that must not allocate once it runs. Such a caller creates the operator at
 * start-up; this call then allocates nothing (no cudaMalloc or cudaFree): the
 * recurrence's two work panels live in a fixed 16 MiB device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits.
 *  Limit: n_rows * k <= 1,048,576 (2^20); larger requests return
 *         VBCSR_ERR_UNSUPPORTED and launch nothing.
 *  The first call on a device looks up the array's device address (with
 *  that device current); make that first call before any stream capture.
 *  All calls share the one array: calls whose work overlaps on the GPU (on
 *  different streams, or from several threads) race and give wrong moments.
 *  Nothing in the array needs to start at zero: each call writes every element
 *  it reads before reading it.
 * Arguments, moments and errors as in vbcsr_chebyshev. (This entry point has
 * no counterpart in the paper.)
 */
int vbcsr_chebyshev_noalloc(vbcsr_t *Ht, int64_t k, const double *R, int64_t ldr, int64_t n_moments,
                            double *moments, int precision, void *stream);

/*
 * Thresholded block sparse product C = A * B (Sec. III.B, Eqs. 2-3), a new
 * handle in *C. A's block columns must be B's block rows (same count and
 * sizes); same dtype. With Frobenius block norms:
 *  symbolic stage  a candidate block (i, j) is kept when the bound
 *                  sum_k ||A_ik|| ||B_kj|| (Eq. 3, summed over k in
 *                  increasing column order) is >= eps; on the GPU, one warp
 *                  per block row;
 *  numeric stage   C_ij = sum_k A_ik B_kj over every k with both blocks stored
 *                  (products grouped by output block, equal inner sizes b_k
 *                  adjacent), on the GPU;
 *  final filter    blocks with ||C_ij|| < eps are removed.
 * eps = 0 keeps every block reached by a product path. The per-row counts of
 * the symbolic stage, the block columns and norms of the candidates and the
 * filtered pattern pass through host memory; the call synchronises `stream`.
 * Errors: INVALID_ARG, NO_MEMORY, CUDA; UNSUPPORTED when one block row has
 * more than 2^28 candidate products.
 */
int vbcsr_spgemm(const vbcsr_t *A, const vbcsr_t *B, double eps, vbcsr_t **C, void *stream);

/*
 * Periodic operator at a reciprocal-space point (Eq. 4). The real-space images
 * O(R) of a periodic operator are given as edges (i, j, R), each with a real
 * b_i x b_j block; the result is a VBCSR_C128 handle on the union pattern (every
 * (i, j) that some edge has, columns increasing inside a row) whose values
 * vbcsr_set_kpoint fills with
 *     O_ij(k) = sum over the edges (i, j, R) of exp(-2 pi i k . s) O_ij(R),
 * s = R (tau == NULL: the "R" convention) or s = R + tau_j - tau_i (the "R+tau"
 * convention), k in fractional reciprocal coordinates. Until the first
 * vbcsr_set_kpoint the values are zero.
 *  n_atoms, bsize[n_atoms]   block size of every atom (square blocks: rows = columns)
 *  n_edges                   >= 0; edge_i, edge_j host int32 [n_edges] atoms in [0, n_atoms)
 *  edge_R                    host int32 [n_edges][3] lattice translations
 *  edge_values               host double, the edges' blocks packed in edge order, each
 *                            row-major b_i x b_j
 *  tau                       host double [n_atoms][3] fractional positions, or NULL
 * The images stay on the device (FP64) so that vbcsr_set_kpoint can sample many k.
 * Edges that repeat (i, j, R) are summed. Errors: INVALID_ARG, PATTERN, NO_MEMORY, CUDA.
 */
int vbcsr_create_kspace(vbcsr_t **out, int64_t n_atoms, const int32_t *bsize, int64_t n_edges,
                        const int32_t *edge_i, const int32_t *edge_j, const int32_t *edge_R,
                        const double *edge_values, const double *tau, void *stream);

/* Fill a vbcsr_create_kspace handle with O(k); kfrac: host double[3]. Asynchronous on
   `stream`. Errors: INVALID_ARG (NULL, or a handle not made by vbcsr_create_kspace), CUDA. */
int vbcsr_set_kpoint(vbcsr_t *H, const double *kfrac, void *stream);

/* ---- inspection ---------------------------------------------------------- */

int vbcsr_get_info(const vbcsr_t *A, vbcsr_info_t *out);

/* Copies the pattern out (host arrays of n_brows, n_bcols, n_brows + 1 and
   nblk elements, as vbcsr_get_info reports them; any pointer may be NULL),
   block columns in the order the handle was created with. */
int vbcsr_get_pattern(const vbcsr_t *A, int32_t *row_bsize, int32_t *col_bsize, int64_t *block_row_ptr,
                      int32_t *block_col_idx);

/*
 * Shape-class registry (Sec. III.B: every distinct (b_i, b_j) of a stored
 * block is registered as a shape class). Writes up to `cap` classes sorted by
 * (b_i, b_j) into bi[], bj[], count[] and returns the number of classes (>= 0)
 * or a negative status.
 */
int vbcsr_shape_classes(const vbcsr_t *A, int32_t *bi, int32_t *bj, int64_t *count, int32_t cap);

/*
 * Tuning of the CUDA-core products. Work items are bucketed by their row
 * count B (1..16); each bucket has a column tile kc (output columns per warp
 * pass: 1, 2, 4, 8, 16 or 32; 0 = the smallest power of two >= k, capped at
 * 32) and a CTA width (warps per CTA: 1, 2, 4 or 8; 0 = 4). A tile larger than
 * k's automatic choice is clamped to it.
 *  vbcsr_set_tuning         the same kc and warps for every bucket
 *  vbcsr_set_bucket_tuning  one bucket (B = 0: every bucket)
 *  vbcsr_set_schedule       VBCSR_SCHED_BUCKETED or VBCSR_SCHED_PERSISTENT, optionally
 *                           OR VBCSR_SCHED_MMA_STAGED, VBCSR_SCHED_NO_CSR and
 *                           VBCSR_SCHED_NO_RING, and the CTA width of the
 *                           persistent launch (0 = 4)
 *  vbcsr_get_tuning         reads them back: kc_by_b[17], warps_by_b[17] (index = B;
 *                           any pointer may be NULL)
 * They apply to later calls on this handle. The tensor-core modes ignore them.
 */
int vbcsr_set_tuning(vbcsr_t *A, int32_t kc, int32_t warps_per_cta);
int vbcsr_set_bucket_tuning(vbcsr_t *A, int32_t B, int32_t kc, int32_t warps_per_cta);
int vbcsr_set_schedule(vbcsr_t *A, int32_t schedule, int32_t persist_warps);
int vbcsr_get_tuning(const vbcsr_t *A, int32_t *kc_by_b, int32_t *warps_by_b, int32_t *schedule,
                     int32_t *persist_warps);

/*
 * Autotuner: times the product (transpose = 0 forward, 1 adjoint) at width k
 * for every bucket's candidate (kc, warps) pairs, keeps the fastest per
 * bucket, then times the persistent schedule at each CTA width and keeps
 * whichever schedule is faster (unless flags has VBCSR_TUNE_NO_PERSISTENT).
 * X and Y are device panels of the product's shapes; Y is overwritten. The
 * call synchronises `stream` repeatedly (a set-up step: do not capture it in
 * a CUDA graph). For the tensor-core precisions it only chooses, for the
 * forward product, between the plain and the shared-memory-staged kernel.
 * (The per-shape-group tuning of tiles has no counterpart in the paper.)
 */
int vbcsr_autotune(vbcsr_t *A, int transpose, int64_t k, const void *X, int64_t ldx, void *Y, int64_t ldy,
                   int precision, int32_t flags, void *stream);

/* Synchronises `stream`, then reads and clears the handle's device error
   word: VBCSR_OK, or VBCSR_ERR_DEVICE_CHECK with the recorded code in the
   detail message. */
int vbcsr_check(vbcsr_t *A, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VBCSR_H */
