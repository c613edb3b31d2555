/*
 * FP64 CPU oracle for rpCholesky-QR (Garrison & Ipsen, "A randomized preconditioned Cholesky-QR
 * algorithm", arXiv 2406.11751).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct restatement of the
 * method that the CUDA library is checked against.  It shares no code, header, table or helper
 * with the CUDA path.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  The product path never calls into it.
 *
 * It follows Algorithm alg_2 ("rpCholesky-QR", Section 4) step by step:
 *   sample        A_s = S A            c rows drawn uniformly, independently, with replacement and
 *                                      scaled by sqrt(m/c) as in Remark r_exp (Section 5); or, with
 *                                      smoothing, A_s = S F A with F = F_T D (Walsh-Hadamard F_T,
 *                                      Rademacher D; the Blendenpik remark of Section 4)
 *   factor        A_s = Q_s R_s        Householder QR, R_s only
 *   precondition  A_1 = A R_s^{-1}     m row-wise lower-triangular solves R_s^T a1_i^T = a_i^T
 *   Gram          G_1 = A_1^T A_1
 *   Cholesky      G_1 = R_2^T R_2
 *   solve         Q   = A_1 R_2^{-1}   m row-wise solves
 *   recover       R   = R_2 R_s
 * and Algorithm alg_0 ("Basic Cholesky-QR", Section 2.1) for Cholesky-QR, Cholesky-QR2 and the shifted
 * Cholesky-QR3 cited in Section 1.
 *
 * Readings where the paper is silent (each stated at the function that implements it):
 *   - the random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), key (seed, stream),
 *     counter block k = (k,0,0,0), sample j takes word j mod 4 of block j/4, index = high 64 bits
 *     of word * m;
 *   - R_s is sign-normalised to a positive diagonal (rows with a negative diagonal are negated),
 *     which makes (Q, R) the unique thin QR with diag(R) > 0 (Lemma l_r1r2, Section 2.1);
 *   - the sketch is "singular" only when a diagonal element of R_s is zero, subnormal or not finite;
 *   - Cholesky fails when a pivot is not > 0 (this includes NaN).
 *
 * Compiled with -O2 -ffp-contract=off so every a*b+c is two rounded operations, sums run left
 * to right, and the Gram sums 4096-row blocks left to right and then combines the block sums in a
 * fixed pairwise tree, so results do not depend on the OpenMP thread count.
 *
 * "variant" = 1 reverses every inner summation order (the oracle' used to measure how far two
 * equally valid roundings of the same algorithm drift apart).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NONFINITE = 2, ORC_ERR_SINGULAR_SKETCH = 3,
       ORC_ERR_NOT_SPD = 4 };

#define ORC_GRAM_BLOCK 4096

/* ---------------------------------------------------------------------------------------------
 * Philox4x64-10.  Round function from Salmon et al. (SC'11), Section 4: two 64x64->128-bit
 * products of the even words with the multipliers, the odd words and the key xor-ed into the high
 * halves, with the words permuted; the key is bumped by the Weyl constants between rounds.
 * ------------------------------------------------------------------------------------------- */
static const uint64_t ORC_PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t ORC_PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t ORC_PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t ORC_PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1 */

static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += ORC_PHILOX_W0; k1 += ORC_PHILOX_W1; }
        uint64_t hi0, lo0, hi1, lo1;
        orc_mulhilo64(ORC_PHILOX_M0, x0, &hi0, &lo0);
        orc_mulhilo64(ORC_PHILOX_M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Sampling matrix S of Section 4 (c rows of [1, m], uniform, independent, with replacement),
 * as 0-based row indices.  Reading: Philox words mapped to [0, m) by the high half of w * m. */
void oracle_sample_indices(uint64_t seed, uint64_t stream, int64_t m, int64_t s, int64_t* idx) {
    uint64_t key[2] = {seed, stream};
    for (int64_t blk = 0; blk * 4 < s; ++blk) {
        uint64_t ctr[4] = {(uint64_t)blk, 0, 0, 0}, w[4];
        oracle_philox4x64_10(ctr, key, w);
        for (int q = 0; q < 4 && blk * 4 + q < s; ++q) {
            uint64_t hi, lo;
            orc_mulhilo64(w[q], (uint64_t)m, &hi, &lo);
            idx[blk * 4 + q] = (int64_t)hi;
        }
    }
}

/* A_s = sqrt(m/c) * A(idx, :) (Remark r_exp, Section 5).  The scale is computed once with sqrt(). */
void oracle_gather_scale(const double* A, int64_t m, int64_t n, int64_t lda, const int64_t* idx,
                         int64_t s, double* As) {
    double scale = sqrt((double)m / (double)s);
    for (int64_t j = 0; j < s; ++j)
        for (int64_t c = 0; c < n; ++c) As[j * n + c] = scale * A[idx[j] * lda + c];
}

/* ---------------------------------------------------------------------------------------------
 * Householder QR of the s x n sample (Algorithm alg_2, step 'factor A_s = Q_s R_s'), textbook column-by-column form
 * (Golub & Van Loan, Householder vector with beta = -sign(alpha)||x||, v(1) = 1,
 * tau = (beta - alpha)/beta).  W is overwritten.  Only R_s (n x n, row-major, upper) is kept;
 * afterwards each row with a negative diagonal is negated.
 * Returns ORC_ERR_SINGULAR_SKETCH if a diagonal of R_s is 0, subnormal or not finite.
 * ------------------------------------------------------------------------------------------- */
int oracle_householder_r(double* W, int64_t s, int64_t n, double* Rs, int variant) {
    if (s < n || n < 1) return ORC_ERR_ARG;
    double* v = (double*)malloc(sizeof(double) * (size_t)s);
    for (int64_t j = 0; j < n; ++j) {
        double alpha = W[j * n + j];
        double sigma = 0.0;
        if (!variant) {
            for (int64_t i = j + 1; i < s; ++i) sigma += W[i * n + j] * W[i * n + j];
        } else {
            for (int64_t i = s - 1; i > j; --i) sigma += W[i * n + j] * W[i * n + j];
        }
        double beta, tau;
        if (sigma == 0.0) {
            beta = alpha; tau = 0.0;      /* already triangular in this column: no reflection */
            for (int64_t i = j; i < s; ++i) v[i] = 0.0;
        } else {
            double nrm = sqrt(alpha * alpha + sigma);
            beta = (alpha >= 0.0) ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            double inv = 1.0 / (alpha - beta);
            v[j] = 1.0;
            for (int64_t i = j + 1; i < s; ++i) v[i] = W[i * n + j] * inv;
        }
        W[j * n + j] = beta;
        for (int64_t i = j + 1; i < s; ++i) W[i * n + j] = 0.0;
        if (tau != 0.0) {
            for (int64_t k = j + 1; k < n; ++k) {
                double w = 0.0;
                if (!variant) {
                    for (int64_t i = j; i < s; ++i) w += v[i] * W[i * n + k];
                } else {
                    for (int64_t i = s - 1; i >= j; --i) w += v[i] * W[i * n + k];
                }
                double tw = tau * w;
                for (int64_t i = j; i < s; ++i) W[i * n + k] -= v[i] * tw;
            }
        }
    }
    free(v);
    int status = ORC_OK;
    for (int64_t i = 0; i < n; ++i) {
        double d = W[i * n + i];
        double sgn = (d < 0.0) ? -1.0 : 1.0;
        for (int64_t k = 0; k < n; ++k) Rs[i * n + k] = (k < i) ? 0.0 : sgn * W[i * n + k];
        if (!isfinite(d) || fabs(d) < DBL_MIN) status = ORC_ERR_SINGULAR_SKETCH;
    }
    return status;
}

/* Row-wise forward substitution X = B T^{-1} for upper-triangular T (n x n), i.e. the m lower
 * triangular systems T^T x_i^T = b_i^T (the row-wise view stated in Section 2.1; used for
 * A_1 = A R_s^{-1} and Q = A_1 R_2^{-1} of Algorithm alg_2):
 *   x_i[j] = (b_i[j] - sum_{k<j} x_i[k] T[k][j]) / T[j][j]. */
void oracle_trsm_rows(const double* B, int64_t m, int64_t n, int64_t ldb, const double* T,
                      double* X, int64_t ldx, int variant) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const double* b = B + i * ldb;
        double* x = X + i * ldx;
        for (int64_t j = 0; j < n; ++j) {
            double t = b[j];
            if (!variant) {
                for (int64_t k = 0; k < j; ++k) t -= x[k] * T[k * n + j];
            } else {
                for (int64_t k = j - 1; k >= 0; --k) t -= x[k] * T[k * n + j];
            }
            x[j] = t / T[j * n + j];
        }
    }
}

/* Gram matrix G = X^T X (Algorithm alg_2, step 'multiply G_1 = A_1^T A_1'), upper triangle, lower triangle mirrored.
 * Fixed order: each 4096-row block summed row by row, then the block sums combined in a pairwise
 * tree over block index.  variant 1 walks rows inside each block backwards. */
void oracle_gram(const double* X, int64_t m, int64_t n, int64_t ldx, double* G, int variant) {
    int64_t nb = (m + ORC_GRAM_BLOCK - 1) / ORC_GRAM_BLOCK;
    if (nb < 1) nb = 1;
    size_t nn = (size_t)n * (size_t)n;
    double* part = (double*)calloc((size_t)nb * nn, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        double* P = part + (size_t)b * nn;
        int64_t r0 = b * ORC_GRAM_BLOCK, r1 = r0 + ORC_GRAM_BLOCK;
        if (r1 > m) r1 = m;
        for (int64_t t = 0; t < r1 - r0; ++t) {
            int64_t r = variant ? (r1 - 1 - t) : (r0 + t);
            const double* x = X + r * ldx;
            for (int64_t p = 0; p < n; ++p) {
                double xp = x[p];
                for (int64_t q = p; q < n; ++q) P[p * n + q] += xp * x[q];
            }
        }
    }
    for (int64_t stride = 1; stride < nb; stride *= 2) {
#pragma omp parallel for schedule(static)
        for (int64_t b = 0; b < nb; b += 2 * stride) {
            if (b + stride < nb) {
                double* D = part + (size_t)b * nn;
                const double* S = part + (size_t)(b + stride) * nn;
                for (size_t e = 0; e < nn; ++e) D[e] += S[e];
            }
        }
    }
    for (int64_t p = 0; p < n; ++p)
        for (int64_t q = 0; q < n; ++q) G[p * n + q] = (q >= p) ? part[p * n + q] : part[q * n + p];
    free(part);
}

/* Upper Cholesky G = R^T R (Algorithm alg_2, step 'factor G_1 = R_2^T R_2'), unblocked:
 *   R[j][j] = sqrt(G[j][j] - sum_{k<j} R[k][j]^2),
 *   R[j][l] = (G[j][l] - sum_{k<j} R[k][j] R[k][l]) / R[j][j],  l > j.
 * Returns ORC_ERR_NOT_SPD (and *pivot = j) when a pivot is not > 0 (NaN included). */
int oracle_cholesky_upper(const double* G, int64_t n, double* R, int64_t* pivot, int variant) {
    memset(R, 0, sizeof(double) * (size_t)n * (size_t)n);
    if (pivot) *pivot = -1;
    for (int64_t j = 0; j < n; ++j) {
        double d = G[j * n + j];
        if (!variant) {
            for (int64_t k = 0; k < j; ++k) d -= R[k * n + j] * R[k * n + j];
        } else {
            for (int64_t k = j - 1; k >= 0; --k) d -= R[k * n + j] * R[k * n + j];
        }
        if (!(d > 0.0)) {
            if (pivot) *pivot = j;
            return ORC_ERR_NOT_SPD;
        }
        double rjj = sqrt(d);
        R[j * n + j] = rjj;
        for (int64_t l = j + 1; l < n; ++l) {
            double t = G[j * n + l];
            if (!variant) {
                for (int64_t k = 0; k < j; ++k) t -= R[k * n + j] * R[k * n + l];
            } else {
                for (int64_t k = j - 1; k >= 0; --k) t -= R[k * n + j] * R[k * n + l];
            }
            R[j * n + l] = t / rjj;
        }
    }
    return ORC_OK;
}

/* R = R2 R_s for upper-triangular factors (Algorithm alg_2, step 'recover R'):
 *   R[i][j] = sum_{k=i..j} R2[i][k] R_s[k][j]. */
void oracle_triu_mul(const double* R2, const double* Rs, int64_t n, double* R, int variant) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double t = 0.0;
            if (j >= i) {
                if (!variant) {
                    for (int64_t k = i; k <= j; ++k) t += R2[i * n + k] * Rs[k * n + j];
                } else {
                    for (int64_t k = j; k >= i; --k) t += R2[i * n + k] * Rs[k * n + j];
                }
            }
            R[i * n + j] = t;
        }
}

static int orc_all_finite(const double* A, int64_t m, int64_t n, int64_t lda) {
    int ok = 1;
#pragma omp parallel for schedule(static) reduction(&& : ok)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) ok = ok && isfinite(A[i * lda + j]);
    return ok;
}

/* ---------------------------------------------------------------------------------------------
 * Smoothing F = F_T D.  Algorithm alg_2 samples rows of F A; the remark after Theorem t_prob
 * (Section 4) takes F_T a Walsh-Hadamard, discrete cosine or Hartley transform and D a diagonal of
 * independent Rademacher signs.  Readings:
 *   - F_T is the Walsh-Hadamard transform of order m' = 2^ceil(log2 m) in natural (Sylvester)
 *     order, normalised to be orthogonal: F_T[k][i] = (-1)^popcount(k & i) / sqrt(m');
 *     it acts on A padded with m' - m zero rows (same R factor as A);
 *   - D_i = -1 when bit 63 of word (i mod 4) of Philox block i/4 under key (seed, stream + 1) is
 *     set, else +1;
 *   - the c sampled rows are drawn from [0, m') and scaled by sqrt(m'/c).
 * ------------------------------------------------------------------------------------------- */
int64_t oracle_smooth_order(int64_t m) {
    int64_t p = 1;
    while (p < m) p <<= 1;
    return p;
}

void oracle_rademacher(uint64_t seed, uint64_t stream, int64_t m, double* d) {
    uint64_t key[2] = {seed, stream};
    for (int64_t blk = 0; blk * 4 < m; ++blk) {
        uint64_t ctr[4] = {(uint64_t)blk, 0, 0, 0}, w[4];
        oracle_philox4x64_10(ctr, key, w);
        for (int q = 0; q < 4 && blk * 4 + q < m; ++q) d[blk * 4 + q] = (w[q] >> 63) ? -1.0 : 1.0;
    }
}

/* out (nrows x n) = rows `rows` of F_T D [A; 0] (m' = mp rows), each a plain sum over i < m of
 * (-1)^popcount(k & i) d_i A[i, :], times 1/sqrt(m'). */
void oracle_smooth_rows(const double* A, int64_t m, int64_t n, int64_t lda, const double* d, int64_t mp,
                        const int64_t* rows, int64_t nrows, double* out) {
    const double inv = 1.0 / sqrt((double)mp);
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nrows; ++j) {
        const uint64_t k = (uint64_t)rows[j];
        double* o = out + j * n;
        for (int64_t c = 0; c < n; ++c) o[c] = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            const double sg = (__builtin_popcountll(k & (uint64_t)i) & 1) ? -d[i] : d[i];
            const double* a = A + i * lda;
            for (int64_t c = 0; c < n; ++c) o[c] += sg * a[c];
        }
        for (int64_t c = 0; c < n; ++c) o[c] *= inv;
    }
}

/* The discrete cosine transform (the paper's MATLAB dct, Remark r_exp) as F_T: the orthonormal DCT-II
 * of order m', F_T[k][i] = w_k cos(pi (2i + 1) k / (2 m')), w_0 = sqrt(1/m'), w_k = sqrt(2/m') for
 * k > 0, on D [A; 0].  out (nrows x n) = rows `rows`, each a plain sum over i < m; the cosine argument
 * is reduced exactly as the integer (2i + 1) k mod 4m' before it is scaled by pi / (2m'). */
void oracle_smooth_rows_dct(const double* A, int64_t m, int64_t n, int64_t lda, const double* d, int64_t mp,
                            const int64_t* rows, int64_t nrows, double* out) {
    const double pi = 3.14159265358979323846;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < nrows; ++j) {
        const uint64_t k = (uint64_t)rows[j];
        const double w = k == 0 ? sqrt(1.0 / (double)mp) : sqrt(2.0 / (double)mp);
        double* o = out + j * n;
        for (int64_t c = 0; c < n; ++c) o[c] = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            const uint64_t r = ((2 * (uint64_t)i + 1) * k) % (4 * (uint64_t)mp);
            const double cs = cos(pi * (double)r / (2.0 * (double)mp)) * d[i];
            const double* a = A + i * lda;
            for (int64_t c = 0; c < n; ++c) o[c] += cs * a[c];
        }
        for (int64_t c = 0; c < n; ++c) o[c] *= w;
    }
}

/* The smoothed sample A_s = sqrt(m'/c) (F A)(idx, :), idx drawn from [0, m') (key (seed, stream));
 * kind 1: Walsh-Hadamard F_T, kind 2: cosine F_T. */
void oracle_smoothed_sample(const double* A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                            uint64_t stream, int kind, int64_t* idx, double* As) {
    const int64_t mp = oracle_smooth_order(m);
    double* d = (double*)malloc(sizeof(double) * (size_t)m);
    oracle_rademacher(seed, stream + 1, m, d);
    oracle_sample_indices(seed, stream, mp, s, idx);
    if (kind == 2) oracle_smooth_rows_dct(A, m, n, lda, d, mp, idx, s, As);
    else oracle_smooth_rows(A, m, n, lda, d, mp, idx, s, As);
    const double scale = sqrt((double)mp / (double)s);
    for (int64_t e = 0; e < s * n; ++e) As[e] *= scale;
    free(d);
}

/* ---------------------------------------------------------------------------------------------
 * rpCholesky-QR (Algorithm alg_2, Section 4).  Q: m x n (ldq), R: n x n.  smoothing = 0: A_s = S A;
 * 1 / 2: A_s = S F A with the Walsh-Hadamard / cosine smoothing above (idx then indexes the m' rows
 * of F A).
 * Optional outputs (may be NULL): idx (s), Rs (n x n), A1 (m x n, ld n), G1 (n x n), R1 (n x n).
 * Status order: ARG, NONFINITE (a sampled row; with smoothing any row, since every row enters the
 * sample), SINGULAR_SKETCH, NONFINITE (any row), NOT_SPD.
 * ------------------------------------------------------------------------------------------- */
int oracle_rpcholqr(const double* A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                    uint64_t stream, double* Q, int64_t ldq, double* R, int64_t* idx_out,
                    double* Rs_out, double* A1_out, double* G1_out, double* R1_out,
                    int64_t* pivot, int variant, int smoothing) {
    if (pivot) *pivot = -1;
    if (n < 1 || s < n || m < s || lda < n || ldq < n || smoothing < 0 || smoothing > 2) return ORC_ERR_ARG;
    size_t nn = (size_t)n * (size_t)n;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)s);
    double* As = (double*)malloc(sizeof(double) * (size_t)s * (size_t)n);
    double* Rs = (double*)malloc(sizeof(double) * nn);
    double* A1 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* G1 = (double*)malloc(sizeof(double) * nn);
    double* R1 = (double*)malloc(sizeof(double) * nn);
    int status = ORC_OK;

    if (smoothing) {
        if (!orc_all_finite(A, m, n, lda)) { status = ORC_ERR_NONFINITE; goto done; }
        oracle_smoothed_sample(A, m, n, lda, s, seed, stream, smoothing, idx, As);
    } else {
        oracle_sample_indices(seed, stream, m, s, idx);
        oracle_gather_scale(A, m, n, lda, idx, s, As);
    }
    if (idx_out) memcpy(idx_out, idx, sizeof(int64_t) * (size_t)s);
    if (!orc_all_finite(As, s, n, n)) { status = ORC_ERR_NONFINITE; goto done; }
    status = oracle_householder_r(As, s, n, Rs, variant);
    if (Rs_out) memcpy(Rs_out, Rs, sizeof(double) * nn);
    if (status != ORC_OK) goto done;
    if (!orc_all_finite(A, m, n, lda)) { status = ORC_ERR_NONFINITE; goto done; }
    oracle_trsm_rows(A, m, n, lda, Rs, A1, n, variant);
    if (A1_out) memcpy(A1_out, A1, sizeof(double) * (size_t)m * (size_t)n);
    oracle_gram(A1, m, n, n, G1, variant);
    if (G1_out) memcpy(G1_out, G1, sizeof(double) * nn);
    status = oracle_cholesky_upper(G1, n, R1, pivot, variant);
    if (R1_out) memcpy(R1_out, R1, sizeof(double) * nn);
    if (status != ORC_OK) goto done;
    oracle_trsm_rows(A1, m, n, n, R1, Q, ldq, variant);
    oracle_triu_mul(R1, Rs, n, R, variant);
done:
    free(idx); free(As); free(Rs); free(A1); free(G1); free(R1);
    return status;
}

/* Basic Cholesky-QR (Algorithm alg_0, Section 2.1): G = A^T A, G = R^T R, Q = A R^{-1}. */
int oracle_cholqr(const double* A, int64_t m, int64_t n, int64_t lda, double* Q, int64_t ldq,
                  double* R, int64_t* pivot, int variant) {
    if (n < 1 || m < n || lda < n || ldq < n) return ORC_ERR_ARG;
    double* G = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* Ac = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    for (int64_t i = 0; i < m; ++i) memcpy(Ac + i * n, A + i * lda, sizeof(double) * (size_t)n);
    oracle_gram(Ac, m, n, n, G, variant);
    int st = oracle_cholesky_upper(G, n, R, pivot, variant);
    if (st == ORC_OK) oracle_trsm_rows(Ac, m, n, n, R, Q, ldq, variant);
    free(G); free(Ac);
    return st;
}

/* Cholesky-QR2 (Yamamoto et al., the comparison method of Section 5.3): Cholesky-QR applied to A,
 * then to the first Q; R = R_b R_a. */
int oracle_cholqr2(const double* A, int64_t m, int64_t n, int64_t lda, double* Q, int64_t ldq,
                   double* R, int64_t* pivot, int variant) {
    size_t nn = (size_t)n * (size_t)n;
    double* Q1 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* Ra = (double*)malloc(sizeof(double) * nn);
    double* Rb = (double*)malloc(sizeof(double) * nn);
    int st = oracle_cholqr(A, m, n, lda, Q1, n, Ra, pivot, variant);
    if (st == ORC_OK) st = oracle_cholqr(Q1, m, n, n, Q, ldq, Rb, pivot, variant);
    if (st == ORC_OK) oracle_triu_mul(Rb, Ra, n, R, variant);
    free(Q1); free(Ra); free(Rb);
    return st;
}

/* Shifted Cholesky-QR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020;
 * the remedy for Cholesky-QR2's breakdown cited in Section 1): G = A^T A + sigma I with
 * sigma = 11 (m n + n (n + 1)) u ||A||^2, R_1 = chol(G), Q_1 = A R_1^{-1}; then Cholesky-QR2 of Q_1;
 * R = R_3 R_2 R_1.  Reading: u = 2^-53 and ||A||^2 bounded by ||A||_F^2 = trace(A^T A), summed in
 * index order. */
double oracle_scholqr3_shift(const double* G, int64_t m, int64_t n) {
    double tr = 0.0;
    for (int64_t i = 0; i < n; ++i) tr += G[i * n + i];
    return 11.0 * ((double)m * (double)n + (double)n * (double)(n + 1)) * ldexp(1.0, -53) * tr;
}

int oracle_scholqr3(const double* A, int64_t m, int64_t n, int64_t lda, double* Q, int64_t ldq, double* R,
                    int64_t* pivot, int variant) {
    if (pivot) *pivot = -1;
    if (n < 1 || m < n || lda < n || ldq < n) return ORC_ERR_ARG;
    size_t nn = (size_t)n * (size_t)n;
    double* Ac = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* Q1 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* G = (double*)malloc(sizeof(double) * nn);
    double* R1 = (double*)malloc(sizeof(double) * nn);
    double* R23 = (double*)malloc(sizeof(double) * nn);
    for (int64_t i = 0; i < m; ++i) memcpy(Ac + i * n, A + i * lda, sizeof(double) * (size_t)n);
    int st = ORC_OK;
    if (!orc_all_finite(Ac, m, n, n)) { st = ORC_ERR_NONFINITE; goto done; }
    oracle_gram(Ac, m, n, n, G, variant);
    {
        const double sigma = oracle_scholqr3_shift(G, m, n);
        for (int64_t i = 0; i < n; ++i) G[i * n + i] += sigma;
    }
    st = oracle_cholesky_upper(G, n, R1, pivot, variant);
    if (st != ORC_OK) goto done;
    oracle_trsm_rows(Ac, m, n, n, R1, Q1, n, variant);
    st = oracle_cholqr2(Q1, m, n, n, Q, ldq, R23, pivot, variant);
    if (st != ORC_OK) goto done;
    oracle_triu_mul(R23, R1, n, R, variant);
done:
    free(Ac); free(Q1); free(G); free(R1); free(R23);
    return st;
}

/* ---------------------------------------------------------------------------------------------
 * Accurate error metrics.  Dot2 of Ogita, Rump & Oishi (SIAM J. Sci. Comput. 2005, Algorithm 5.3)
 * with TwoSum (Knuth) and TwoProduct via Dekker's splitting (no fused multiply-add needed).
 * ------------------------------------------------------------------------------------------- */
static inline void orc_two_sum(double a, double b, double* x, double* y) {
    double s = a + b;
    double z = s - a;
    *x = s;
    *y = (a - (s - z)) + (b - z);
}
static inline void orc_split(double a, double* hi, double* lo) {
    const double factor = 134217729.0; /* 2^27 + 1 */
    double c = factor * a;
    double h = c - (c - a);
    *hi = h;
    *lo = a - h;
}
static inline void orc_two_product(double a, double b, double* x, double* y) {
    double p = a * b;
    double ah, al, bh, bl;
    orc_split(a, &ah, &al);
    orc_split(b, &bh, &bl);
    *x = p;
    *y = al * bl - (((p - ah * bh) - al * bh) - ah * bl);
}

/* E = Q^T Q - I (n x n, full), every entry a Dot2 sum over the m rows. */
void oracle_orth_matrix(const double* Q, int64_t m, int64_t n, int64_t ldq, double* E) {
#pragma omp parallel for schedule(dynamic)
    for (int64_t p = 0; p < n; ++p) {
        for (int64_t q = p; q < n; ++q) {
            double s = (p == q) ? -1.0 : 0.0, c = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double h, r, t;
                orc_two_product(Q[i * ldq + p], Q[i * ldq + q], &h, &r);
                orc_two_sum(s, h, &s, &t);
                c += t + r;
            }
            E[p * n + q] = s + c;
            E[q * n + p] = s + c;
        }
    }
}

/* Residual rows D = A - Q R (m x n, ld n), every entry a Dot2 sum. */
void oracle_residual_matrix(const double* A, int64_t m, int64_t n, int64_t lda, const double* Q,
                            int64_t ldq, const double* R, double* D) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double s = A[i * lda + j], c = 0.0;
            for (int64_t k = 0; k <= j; ++k) {
                double h, r, t;
                orc_two_product(-Q[i * ldq + k], R[k * n + j], &h, &r);
                orc_two_sum(s, h, &s, &t);
                c += t + r;
            }
            D[i * n + j] = s + c;
        }
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
