// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11)
// and the sample-row map of the sampling matrix S (Section 4), shared by the sample kernels.
// Each of the 10 rounds multiplies counter words 0 and 2 by the two round multipliers (full 128-bit
// products), xors the high halves with the odd counter words and the key, and permutes; the key
// advances by the two Weyl increments between rounds.  Key = (seed, stream_id); counter block
// k = (k,0,0,0); sample j uses word j%4 of block j/4 and maps it to a row by the high 64 bits of
// word * m.
#pragma once
#include <cstdint>

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

}  // namespace rpq
