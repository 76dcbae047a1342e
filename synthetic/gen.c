/*
 * Seeded synthetic input generator (host C, OpenMP).
 *
 * This file draws the random numbers that make up the synthetic operators
 * and panels; it holds none of the sparse-product arithmetic. Every value is
 * a pure function of (seed, stream, counter) through SplitMix64 (Steele, Lea
 * & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
 * so the result does not depend on thread count or traversal order.
 *
 *   hash(key, n)   = mix(key + (n + 1) * 0x9E3779B97F4A7C15)
 *   normal(key, n) = Box-Muller on the two 32-bit halves of hash(key, n)
 *   sign(key, n)   = +1 / -1 from the top bit of hash(key, n)
 */
#include <math.h>
#include <stdint.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t syn_stream_key(uint64_t seed, uint64_t stream) {
    return mix64(mix64(seed + GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL));
}

static inline uint64_t hash_at(uint64_t key, uint64_t n) {
    return mix64(key + (n + 1ULL) * GOLDEN);
}

static inline double normal_at(uint64_t key, uint64_t n) {
    uint64_t h = hash_at(key, n);
    double u1 = ((double)(h >> 32) + 1.0) * (1.0 / 4294967296.0);   /* (0, 1] */
    double u2 = (double)(h & 0xFFFFFFFFULL) * (1.0 / 4294967296.0); /* [0, 1) */
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* out[i] = normal(key, counter[i]) */
void syn_normal_at(uint64_t key, int64_t n, const uint64_t *counter, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = normal_at(key, counter[i]);
}

/* Dense row-major panel P[r*ld + c] = normal(key, r*ncols + c). */
void syn_normal_panel(uint64_t key, int64_t nrows, int64_t ncols, int64_t ld, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; ++r)
        for (int64_t c = 0; c < ncols; ++c)
            out[r * ld + c] = normal_at(key, (uint64_t)(r * ncols + c));
}

/* Dense row-major panel of +1/-1 (Rademacher) entries. */
void syn_sign_panel(uint64_t key, int64_t nrows, int64_t ncols, int64_t ld, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; ++r)
        for (int64_t c = 0; c < ncols; ++c)
            out[r * ld + c] = (hash_at(key, (uint64_t)(r * ncols + c)) >> 63) ? -1.0 : 1.0;
}

/*
 * Values of a symmetric block operator, H_ji = H_ij^T, packed block by block
 * (blocks in block_row_ptr / block_col_idx order, each block row-major b_i x b_j).
 *
 * The entry (p, q) of block (i, j) with i < j is scale[blk] * G_ij[p, q]; with
 * i > j it is scale[blk] * G_ji[q, p]; a diagonal block is
 * scale[blk] * (G_ii[p, q] + G_ii[q, p]) / sqrt(2). G_lo,hi[p, q] is the normal
 * draw at counter ((lo * n_atoms + hi) << 10) | (p << 5) | q, so block sizes are
 * limited to 32. scale[] must itself be symmetric in (i, j).
 */
int syn_symmetric_values(uint64_t key, int64_t n_atoms, const int32_t *bsize,
                         const int64_t *block_row_ptr, const int32_t *block_col_idx,
                         const int64_t *value_offset, const double *scale, double *out) {
    for (int64_t a = 0; a < n_atoms; ++a)
        if (bsize[a] < 1 || bsize[a] > 32) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_atoms; ++i) {
        const int bi = bsize[i];
        for (int64_t b = block_row_ptr[i]; b < block_row_ptr[i + 1]; ++b) {
            const int64_t j = block_col_idx[b];
            const int bj = bsize[j];
            const double s = scale[b];
            double *blk = out + value_offset[b];
            for (int p = 0; p < bi; ++p) {
                for (int q = 0; q < bj; ++q) {
                    double v;
                    if (i < j) {
                        uint64_t c = ((uint64_t)(i * n_atoms + j) << 10) | ((uint64_t)p << 5) | (uint64_t)q;
                        v = normal_at(key, c);
                    } else if (i > j) {
                        uint64_t c = ((uint64_t)(j * n_atoms + i) << 10) | ((uint64_t)q << 5) | (uint64_t)p;
                        v = normal_at(key, c);
                    } else {
                        uint64_t base = (uint64_t)(i * n_atoms + i) << 10;
                        double g1 = normal_at(key, base | ((uint64_t)p << 5) | (uint64_t)q);
                        double g2 = normal_at(key, base | ((uint64_t)q << 5) | (uint64_t)p);
                        v = (g1 + g2) * 0.70710678118654752440;
                    }
                    blk[p * bj + q] = s * v;
                }
            }
        }
    }
    return 0;
}
