// Steps of a row-sharded factorisation, where each process holds a contiguous block of rows of A
// (Algorithm alg_2 with A partitioned by rows: the row solves of both passes and the Gram partials
// are row-local, so the only exchanges are the s x n sample, before the sketch QR, and the n x n Gram
// matrix, before the Cholesky factorisation):
//
//   k_gather_owned_rows   sample row j = sqrt(m/s) A[idx_j, :] if this block owns global row idx_j,
//                         else a row of zeros (summing the blocks' samples gives the full sample
//                         exactly: every sample row has one owner);
//   k_sample_to_colmajor  a row-major s x n sample into the column-major, padded layout of the
//                         Householder kernel;
//   k_sum_parts           G = sum_k parts[k] in k order (deterministic for a fixed number of parts).
#include "common.cuh"
#include "philox.cuh"

namespace rpq {

__global__ void k_gather_owned_rows(const double* __restrict__ A, int64_t m_local, int32_t n, int64_t lda,
                                    int64_t row_offset, int64_t m, int32_t s, uint64_t seed, uint64_t stream_id,
                                    double scale, double* __restrict__ As, int64_t ld_as, int32_t* info) {
    __shared__ int64_t row_s;
    const int j = blockIdx.x;
    if (threadIdx.x == 0) row_s = sample_row(seed, stream_id, m, j) - row_offset;
    __syncthreads();
    const int64_t r = row_s;
    const bool owned = r >= 0 && r < m_local;
    bool bad = false;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double v = 0.0;
        if (owned) {
            const double a = A[r * lda + c];
            bad |= !isfinite(a);
            v = scale * a;
        }
        As[static_cast<int64_t>(j) * ld_as + c] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
}

// dst (column-major, ld lds, np columns, zero padding) = src (row-major s x n, ld ld_src)
__global__ void k_sample_to_colmajor(const double* __restrict__ src, int64_t ld_src, int32_t s, int32_t n,
                                     int32_t np, double* __restrict__ dst, int64_t lds) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= static_cast<int64_t>(s) * np) return;
    const int c = static_cast<int>(e / s), j = static_cast<int>(e - static_cast<int64_t>(c) * s);
    dst[static_cast<int64_t>(c) * lds + j] = c < n ? src[static_cast<int64_t>(j) * ld_src + c] : 0.0;
}

__global__ void k_sum_parts(const double* __restrict__ parts, int32_t nparts, int32_t n, double* __restrict__ G) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nn = static_cast<int64_t>(n) * n;
    if (e >= nn) return;
    double sum = 0.0;
    for (int k = 0; k < nparts; ++k) sum += parts[k * nn + e];
    G[e] = sum;
}

void launch_gather_owned_rows(const double* A, int64_t m_local, int32_t n, int64_t lda, int64_t row_offset,
                              int64_t m, int32_t s, uint64_t seed, uint64_t stream_id, double scale, double* As,
                              int64_t ld_as, int32_t* info, cudaStream_t st) {
    k_gather_owned_rows<<<s, 128, 0, st>>>(A, m_local, n, lda, row_offset, m, s, seed, stream_id, scale, As,
                                           ld_as, info);
}

void launch_sample_to_colmajor(const double* src, int64_t ld_src, int32_t s, int32_t n, int32_t np, double* dst,
                               int64_t lds, cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(s) * np;
    k_sample_to_colmajor<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(src, ld_src, s, n, np, dst,
                                                                                       lds);
}

void launch_sum_parts(const double* parts, int32_t nparts, int32_t n, double* G, cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(n) * n;
    k_sum_parts<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(parts, nparts, n, G);
}

}  // namespace rpq
