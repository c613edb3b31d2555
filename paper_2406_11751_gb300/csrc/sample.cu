// Step 'sample' of Algorithm alg_2 (Section 4): A_s = sqrt(m/s) * A(idx, :), with idx drawn
// uniformly, independently and with replacement (the sampling matrix S; scale from Remark r_exp).
// Random numbers: Philox4x64-10 (philox.cuh).
#include "common.cuh"
#include "philox.cuh"

namespace rpq {

__global__ void k_sample_indices(uint64_t seed, uint64_t stream_id, int64_t m, int32_t s, int64_t* idx) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j < s) idx[j] = sample_row(seed, stream_id, m, j);
}

// One CTA per sampled row j: As (column-major, ld = lds, np columns) gets sqrt(m/s) * A[idx_j, :]
// in columns < n and 0 in the padding columns.  A non-finite sampled entry sets NONFINITE.
template <typename TA>
__global__ void k_sample_gather(const TA* __restrict__ A, int64_t m, int32_t n, int64_t lda,
                                int32_t s, uint64_t seed, uint64_t stream_id, double scale,
                                double* __restrict__ As, int64_t lds, int32_t np,
                                int64_t* __restrict__ idx_out, int32_t* info) {
    __shared__ int64_t row_s;
    const int j = blockIdx.x;
    if (threadIdx.x == 0) {
        const int64_t r = sample_row(seed, stream_id, m, j);
        row_s = r;
        if (idx_out) idx_out[j] = r;
    }
    __syncthreads();
    const TA* src = A + row_s * lda;
    bool bad = false;
    for (int c = threadIdx.x; c < np; c += blockDim.x) {
        double v = 0.0;
        if (c < n) {
            const double a = static_cast<double>(src[c]);
            bad |= !isfinite(a);
            v = scale * a;
        }
        As[static_cast<int64_t>(c) * lds + j] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
}

// The same sample from rows already gathered in sample order (rows: s x n row-major, ld n): As gets
// sqrt(m/s) * rows[j, :] exactly as k_sample_gather would from A[idx_j, :].
__global__ void k_sample_rows(const double* __restrict__ rows, int32_t n, double scale, double* __restrict__ As,
                              int64_t lds, int32_t np, int32_t* info) {
    const int j = blockIdx.x;
    const double* src = rows + static_cast<int64_t>(j) * n;
    bool bad = false;
    for (int c = threadIdx.x; c < np; c += blockDim.x) {
        double v = 0.0;
        if (c < n) {
            const double a = src[c];
            bad |= !isfinite(a);
            v = scale * a;
        }
        As[static_cast<int64_t>(c) * lds + j] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
}

// A[i] = a uniform value in [-1, 1) from Philox word i mod 4 of block i / 4 under key (seed, 7): the
// synthetic matrices the autotuner times (any full-rank A serves; it is never a result).
__global__ void k_fill_uniform(double* __restrict__ A, int64_t count, uint64_t seed) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint64_t x[4] = {static_cast<uint64_t>(i >> 2), 0ull, 0ull, 0ull};
    philox4x64_10_dev(x, seed, 7ull);
    const int q = static_cast<int>(i & 3);
    const uint64_t w = q == 0 ? x[0] : q == 1 ? x[1] : q == 2 ? x[2] : x[3];
    A[i] = static_cast<double>(static_cast<int64_t>(w) >> 11) * 0x1.0p-52;
}

void launch_fill_uniform(double* A, int64_t count, uint64_t seed, cudaStream_t st) {
    k_fill_uniform<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(A, count, seed);
}

void launch_sample_rows(const double* rows, int32_t n, int32_t s, double scale, double* As, int64_t lds,
                        int32_t np, int32_t* info, cudaStream_t st) {
    k_sample_rows<<<s, 128, 0, st>>>(rows, n, scale, As, lds, np, info);
}

void launch_sample_indices(uint64_t seed, uint64_t stream_id, int64_t m, int32_t s, int64_t* idx,
                           cudaStream_t st) {
    k_sample_indices<<<(s + 127) / 128, 128, 0, st>>>(seed, stream_id, m, s, idx);
}

void launch_sample_gather(const double* A, int64_t m, int32_t n, int64_t lda, int32_t s, uint64_t seed,
                          uint64_t stream_id, double scale, double* As, int64_t lds, int32_t np,
                          int64_t* idx_out, int32_t* info, cudaStream_t st) {
    k_sample_gather<double><<<s, 128, 0, st>>>(A, m, n, lda, s, seed, stream_id, scale, As, lds, np,
                                               idx_out, info);
}

// FP32 input (the FP32 mode): the sampled rows are widened to FP64 before the scale.
void launch_sample_gather_f32(const float* A, int64_t m, int32_t n, int64_t lda, int32_t s, uint64_t seed,
                              uint64_t stream_id, double scale, double* As, int64_t lds, int32_t np,
                              int64_t* idx_out, int32_t* info, cudaStream_t st) {
    k_sample_gather<float><<<s, 128, 0, st>>>(A, m, n, lda, s, seed, stream_id, scale, As, lds, np,
                                              idx_out, info);
}

}  // namespace rpq
