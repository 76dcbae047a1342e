/*
 * VBCSR oracle: plain, slow, scalar-expanded FP64 loops.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links this file;
 * only the tests, the repository smoke check and the benchmark's CPU-baseline
 * leg call it. It shares no code with the CUDA path.
 *
 * Storage (Sec. II.A, Sec. III.B): block row i has b_i = row_bsize[i] scalar
 * rows starting at scalar row r_i = sum_{i'<i} b_{i'}; block column j has
 * b_j = col_bsize[j] scalar columns starting at c_j = sum_{j'<j} b_{j'}. The
 * stored blocks of row i are block_col_idx[block_row_ptr[i] .. block_row_ptr[i+1]),
 * the set J(i). Block values are packed in that order, each block row-major
 * b_i x b_j. Panels X, Y are row-major with leading dimension ld >= k.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* scalar offsets r_i (size n+1) */
static int64_t *prefix_sizes(int64_t n, const int32_t *bsize) {
    int64_t *off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!off) return NULL;
    off[0] = 0;
    for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + bsize[i];
    return off;
}

/* packed value offset of every block (size nblk+1) */
static int64_t *value_offsets(int64_t n_brows, const int32_t *row_bsize, const int32_t *col_bsize,
                              const int64_t *block_row_ptr, const int32_t *block_col_idx) {
    int64_t nblk = block_row_ptr[n_brows];
    int64_t *off = (int64_t *)malloc((size_t)(nblk + 1) * sizeof(int64_t));
    if (!off) return NULL;
    off[0] = 0;
    for (int64_t i = 0; i < n_brows; ++i)
        for (int64_t b = block_row_ptr[i]; b < block_row_ptr[i + 1]; ++b)
            off[b + 1] = off[b] + (int64_t)row_bsize[i] * col_bsize[block_col_idx[b]];
    return off;
}

/*
 * Forward product (Sec. III.B, "Matrix multiplication": for each block row,
 * accumulate A_ij X_j over j in J(i)), in scalar form:
 *
 *   Y[r_i+p, c] = alpha * sum_{j in J(i)} sum_{q<b_j} H_ij[p,q] X[c_j+q, c]
 *                 + beta * Y[r_i+p, c]
 *
 * for block rows i in [row_begin, row_end). beta == 0 means Y is not read.
 * nthreads > 1 splits the block rows over OpenMP threads (rows are independent).
 * Returns 0, or -1 on allocation failure.
 */
int oracle_spmm(int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize, const int32_t *col_bsize,
                const int64_t *block_row_ptr, const int32_t *block_col_idx, const double *values,
                int64_t k, double alpha, const double *X, int64_t ldx, double beta, double *Y,
                int64_t ldy, int64_t row_begin, int64_t row_end, int nthreads) {
    int64_t *r = prefix_sizes(n_brows, row_bsize);
    int64_t *cj = prefix_sizes(n_bcols, col_bsize);
    int64_t *voff = value_offsets(n_brows, row_bsize, col_bsize, block_row_ptr, block_col_idx);
    if (!r || !cj || !voff) { free(r); free(cj); free(voff); return -1; }
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t i = row_begin; i < row_end; ++i) {
        const int bi = row_bsize[i];
        for (int p = 0; p < bi; ++p) {
            for (int64_t c = 0; c < k; ++c) {
                double s = 0.0;
                for (int64_t b = block_row_ptr[i]; b < block_row_ptr[i + 1]; ++b) {
                    const int64_t j = block_col_idx[b];
                    const int bj = col_bsize[j];
                    const double *h = values + voff[b];
                    for (int q = 0; q < bj; ++q)
                        s += h[p * bj + q] * X[(cj[j] + q) * ldx + c];
                }
                double *y = &Y[(r[i] + p) * ldy + c];
                *y = (beta == 0.0) ? alpha * s : alpha * s + beta * (*y);
            }
        }
    }
    free(r); free(cj); free(voff);
    return 0;
}

/*
 * Adjoint product, Eq. (1) (Y_j += A_ij^dagger X_i for j in J(i); real values,
 * so the dagger is a transpose), in scalar form:
 *
 *   Y[c_j+q, c] = alpha * sum_{i : j in J(i)} sum_{p<b_i} H_ij[p,q] X[r_i+p, c]
 *                 + beta * Y[c_j+q, c]
 *
 * Y has n_cols = sum_j b_j rows, X has n_rows = sum_i b_i rows. beta == 0
 * means Y is not read. Single-threaded (the scatter is not partitioned).
 */
int oracle_spmm_adjoint(int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize,
                        const int32_t *col_bsize, const int64_t *block_row_ptr,
                        const int32_t *block_col_idx, const double *values, int64_t k, double alpha,
                        const double *X, int64_t ldx, double beta, double *Y, int64_t ldy) {
    int64_t *r = prefix_sizes(n_brows, row_bsize);
    int64_t *cj = prefix_sizes(n_bcols, col_bsize);
    int64_t *voff = value_offsets(n_brows, row_bsize, col_bsize, block_row_ptr, block_col_idx);
    int64_t ncols = cj ? cj[n_bcols] : 0;
    double *acc = (double *)calloc((size_t)(ncols * k + 1), sizeof(double));
    if (!r || !cj || !voff || !acc) { free(r); free(cj); free(voff); free(acc); return -1; }
    for (int64_t i = 0; i < n_brows; ++i) {
        const int bi = row_bsize[i];
        for (int64_t b = block_row_ptr[i]; b < block_row_ptr[i + 1]; ++b) {
            const int64_t j = block_col_idx[b];
            const int bj = col_bsize[j];
            const double *h = values + voff[b];
            for (int p = 0; p < bi; ++p)
                for (int q = 0; q < bj; ++q)
                    for (int64_t c = 0; c < k; ++c)
                        acc[(cj[j] + q) * k + c] += h[p * bj + q] * X[(r[i] + p) * ldx + c];
        }
    }
    for (int64_t row = 0; row < ncols; ++row)
        for (int64_t c = 0; c < k; ++c) {
            double *y = &Y[row * ldy + c];
            *y = (beta == 0.0) ? alpha * acc[row * k + c] : alpha * acc[row * k + c] + beta * (*y);
        }
    free(r); free(cj); free(voff); free(acc);
    return 0;
}

/*
 * Block-sampled dense-dense product on the stored pattern (the gradient of
 * Y = H X with respect to the stored values):
 *
 *   D_ij[p,q] = alpha * sum_c A[r_i+p, c] B[c_j+q, c] + beta * D_ij[p,q]
 *
 * for every stored block (i, j); D is in the packed value order. beta == 0
 * means D is not read.
 */
int oracle_sddmm(int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize, const int32_t *col_bsize,
                 const int64_t *block_row_ptr, const int32_t *block_col_idx, int64_t k, double alpha,
                 const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *D,
                 int nthreads) {
    int64_t *r = prefix_sizes(n_brows, row_bsize);
    int64_t *cj = prefix_sizes(n_bcols, col_bsize);
    int64_t *voff = value_offsets(n_brows, row_bsize, col_bsize, block_row_ptr, block_col_idx);
    if (!r || !cj || !voff) { free(r); free(cj); free(voff); return -1; }
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t i = 0; i < n_brows; ++i) {
        const int bi = row_bsize[i];
        for (int64_t b = block_row_ptr[i]; b < block_row_ptr[i + 1]; ++b) {
            const int64_t j = block_col_idx[b];
            const int bj = col_bsize[j];
            double *d = D + voff[b];
            for (int p = 0; p < bi; ++p)
                for (int q = 0; q < bj; ++q) {
                    double s = 0.0;
                    for (int64_t c = 0; c < k; ++c)
                        s += A[(r[i] + p) * lda + c] * B[(cj[j] + q) * ldb + c];
                    d[p * bj + q] = (beta == 0.0) ? alpha * s : alpha * s + beta * d[p * bj + q];
                }
        }
    }
    free(r); free(cj); free(voff);
    return 0;
}

/*
 * Gershgorin bounds over scalar rows of a square operator: every eigenvalue
 * lies in [min_r (H_rr - R_r), max_r (H_rr + R_r)], R_r = sum_{c != r} |H_rc|.
 * Writes out[0] = lower bound, out[1] = upper bound. Plain loops, O(nnz) time
 * and O(n_rows) memory.
 */
int oracle_gershgorin(int64_t n_brows, int64_t n_bcols, const int32_t *row_bsize, const int32_t *col_bsize,
                      const int64_t *block_row_ptr, const int32_t *block_col_idx, const double *values,
                      double *out) {
    int64_t *r = prefix_sizes(n_brows, row_bsize);
    int64_t *cj = prefix_sizes(n_bcols, col_bsize);
    int64_t *voff = value_offsets(n_brows, row_bsize, col_bsize, block_row_ptr, block_col_idx);
    if (!r || !cj || !voff) { free(r); free(cj); free(voff); return -1; }
    double lo = 0.0, hi = 0.0;
    int first = 1;
    for (int64_t i = 0; i < n_brows; ++i) {
        const int bi = row_bsize[i];
        for (int p = 0; p < bi; ++p) {
            const int64_t row = r[i] + p;
            double diag = 0.0, off = 0.0;
            for (int64_t b = block_row_ptr[i]; b < block_row_ptr[i + 1]; ++b) {
                const int64_t j = block_col_idx[b];
                const int bj = col_bsize[j];
                const double *h = values + voff[b];
                for (int q = 0; q < bj; ++q) {
                    const double v = h[p * bj + q];
                    if (cj[j] + q == row) diag += v;
                    else off += v < 0 ? -v : v;
                }
            }
            const double a = diag - off, c = diag + off;
            if (first || a < lo) lo = a;
            if (first || c > hi) hi = c;
            first = 0;
        }
    }
    out[0] = lo;
    out[1] = hi;
    free(r); free(cj); free(voff);
    return 0;
}
