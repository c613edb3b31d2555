// Step 'sample' of Algorithm alg_2 (Section 4): A_s = sqrt(m/s) * A(idx, :), with idx drawn
// uniformly, independently and with replacement (the sampling matrix S; scale from Remark r_exp).
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11), written from that paper: each of the 10 rounds multiplies counter words 0 and 2
// by the two round multipliers (full 128-bit products), xors the high halves with the odd counter
// words and the key, and permutes; the key advances by the two Weyl increments between rounds.
// Key = (seed, stream_id); counter block k = (k,0,0,0); sample j uses word j%4 of block j/4 and
// maps it to a row by the high 64 bits of word * m.
#include "common.cuh"

namespace rpq {

__device__ __forceinline__ void philox4x64_10_dev(uint64_t (&x)[4], uint64_t k0, uint64_t k1) {
    constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ull;
    constexpr uint64_t kMulB = 0xCA5A826395121157ull;
    constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ull;
    constexpr uint64_t kWeylB = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += kWeylA; k1 += kWeylB; }
        const uint64_t pa_hi = __umul64hi(kMulA, x[0]), pa_lo = kMulA * x[0];
        const uint64_t pb_hi = __umul64hi(kMulB, x[2]), pb_lo = kMulB * x[2];
        const uint64_t n0 = pb_hi ^ x[1] ^ k0;
        const uint64_t n2 = pa_hi ^ x[3] ^ k1;
        x[0] = n0; x[1] = pb_lo; x[2] = n2; x[3] = pa_lo;
    }
}

__device__ __forceinline__ int64_t sample_row(uint64_t seed, uint64_t stream_id, int64_t m, int64_t j) {
    uint64_t x[4] = {static_cast<uint64_t>(j >> 2), 0ull, 0ull, 0ull};
    philox4x64_10_dev(x, seed, stream_id);
    const int q = static_cast<int>(j & 3);
    const uint64_t w = q == 0 ? x[0] : q == 1 ? x[1] : q == 2 ? x[2] : x[3];
    return static_cast<int64_t>(__umul64hi(w, static_cast<uint64_t>(m)));
}

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
