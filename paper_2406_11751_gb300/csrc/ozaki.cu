// Split-precision (Ozaki-style) FP64 products on the GB300 BF16 tensor cores (tcgen05).
//
// Used by the SPLIT64 mode for the well-conditioned products of Algorithm alg_2 (Section 4):
//   Gram          G_1 = A_1^T A_1               (k_ozaki_gram; above 128 columns k_ozaki_gram_db)
//   solve         Q   = A_1 R_1^{-1}            (k_ozaki_gemm_ws with the explicit R_1^{-1}; above 128
//                                                columns k_ozaki_gemm_db; kappa(R_1) = kappa(A_1) is
//                                                small, Lemma l_31)
//   precondition  the off-diagonal block update A[:,J] - A_1[:,<J] R_s[<J,J] of the blocked row solve
//                                               (k_ozaki_update for K <= 32, else k_ozaki_gemm_ws /
//                                                k_ozaki_gemm_db, subtract form; the diagonal blocks stay
//                                                FP64 substitution)
// Above 128 columns the left operand is sliced beforehand into stage images (k_slice_images,
// k_slice_block_images, k_slice_col_images) that the *_db kernels stream in by TMA bulk copies.
//
// Splitting (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication and its applications", Numer. Algorithms 2012, restated): every
// FP64 value x of a row (or column) with the shared power-of-two bound 2^E > max|x| is cut into eight
// 7-bit signed integer slices, x = 2^E sum_{a=1..8} s_a 2^{-7a} + O(2^{E-56}), |s_a| <= 127 (exact in
// BF16).  A product of two such operands is sum_{a,b} 2^{-7(a+b)} S_a S_b; the 36 slice pairs with
// a + b <= 9 are kept (the dropped ones are below 2^-53 of the scale).  Pairs with the same d = a + b
// share one FP32 accumulator in tensor memory: with K <= 128 every partial sum is an integer below
// 8 * 127^2 * 128 < 2^24, so the FP32 accumulation is exact.  The eight accumulators (d = 2..9) are
// combined exactly in int64, I = sum_{d<=6} M_d 2^{7(6-d)} + rint(sum_{d>6} M_d 2^{7(6-d)}), and the
// result is 2^{E_x + E_y - 42} I.
//
// Tiles: M = 128 output rows (TMEM lanes) x N = 64 output columns, 8 groups x 64 columns = the 512 TMEM
// columns of the SM (k_ozaki_update: N = 32, two tiles in TMEM).  K is staged 32 at a time in shared
// memory (core-matrix K-major layout, no swizzle), two stages in flight: while the tensor core works on
// one stage the CTA slices the next.  One thread issues the 72 tcgen05.mma of a stage and commits them
// to the stage's mbarrier.  Every mbarrier wait is bounded: the pipeline waits by the caller's spin limit
// (a plan option), the final wait for the kernel's own MMAs by kSpinLimit; on timeout the kernel records
// RPCHOLQR_ERR_TIMEOUT, waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include <climits>

#include "common.cuh"

namespace rpq {
namespace oz {

constexpr int kSlices = 8;
constexpr int kGroups = 8;                 // d = 2..9
constexpr int kTileM = 128;
constexpr int kTileN = 64;
constexpr int kKW = 32;                    // K per stage
constexpr int kThreads = 512;            // 16 warps: 4 threads per tile row (TMEM lane), one per K chunk
// Per-thread shares for a CTA of NT threads (NT/128 threads per tile row):
template <int NT> struct Share {
    static constexpr int kRowThreads = NT / 128;
    static constexpr int kChunks = (32 / 8) / kRowThreads;   // 8-value K chunks sliced per stage
    static constexpr int kDrainCols = 64 / kRowThreads;      // output columns drained
};
// The windowed GEMM (K > 128) keeps int64 accumulators live across stages (16 columns per thread with 512
// threads, drained 4 columns at a time to fit the 120 registers a 544-thread CTA allows).
constexpr int kThreadsWin = 512;
constexpr int kSBO = (kKW * 2 / 16) * 128; // 512 B between 8-row core-matrix groups
constexpr int kLBO = 128;                  // 128 B between K-adjacent core matrices
constexpr int kASlice = kTileM * kKW * 2;  // 8 KB
constexpr int kBSlice = kTileN * kKW * 2;  // 4 KB
constexpr int kAStage = kSlices * kASlice; // 64 KB
constexpr int kBStage = kSlices * kBSlice; // 32 KB
// k_ozaki_gemm_ws shared memory: two stages (A slices, then B slices: 96 KB each), then the raw FP64 X
// rows of the next stage (row stride kRawLd doubles: 16-byte reads of one row per thread are
// conflict-free).  At a tile end the drained stage's 96 KB stage the 128 x 64 output tile (row stride
// kEpiLd doubles) so that B is read and C written in whole rows.
constexpr int kStageBytes = kAStage + kBStage;
constexpr int kRawLd = kKW + 2;
constexpr int kRawBytes = kTileM * kRawLd * 8;
constexpr int kEpiLd = kTileN + 1;
constexpr int kGemmSmem = 2 * kStageBytes + kRawBytes;
static_assert(kTileM * kEpiLd * 8 <= kStageBytes, "output tile must fit in one stage");
static_assert(kGemmSmem + 1024 <= 232448, "k_ozaki_gemm_ws exceeds the 227 KB shared-memory limit");
constexpr int kTmemCols = 512;
constexpr long kSpinLimit = 1L << 24;
// BF16 x BF16 -> FP32, A and B K-major, M = 128, N = 64
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte offset of (row r, K byte kb) inside one slice of a stage (8-row x 16-byte core matrices)
__device__ __forceinline__ uint32_t core_off(int r, int kb) {
    return (r >> 3) * kSBO + (kb >> 4) * kLBO + (r & 7) * 16 + (kb & 15);
}
// tcgen05 shared-memory matrix descriptor: start, LBO, SBO (>>4), version 1 at bit 46, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return static_cast<uint64_t>((addr >> 4) & 0x3FFF) | (static_cast<uint64_t>(kLBO >> 4) << 16) |
           (static_cast<uint64_t>(kSBO >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}
// Instruction descriptor: BF16 x BF16 -> FP32, A and B K-major, M = 128, N = n (a multiple of 16, <= 256)
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
           (static_cast<uint32_t>(kTileM >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16_n(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
        smem_u32(bar)));
}
__device__ __forceinline__ uint32_t mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
    return done;
}
// The outcome of a wait is made uniform over the lanes that take part in it: once any of them saw the
// phase complete it stays complete (its next completion needs arrivals this warp has not made yet), so
// the others poll again until they see it too (acquire for every lane).  A lane can therefore never
// leave a wait that its warp-mates passed, whatever the poll limit.
__device__ __forceinline__ bool mbar_uniform(uint64_t* bar, uint32_t parity, uint32_t done) {
    if (__any_sync(__activemask(), done != 0)) {
        for (long it = 0; it < kSpinLimit && !done; ++it) done = mbar_try(bar, parity);
    }
    return done != 0;
}
// Polls the phase up to `limit` times (the plan's spin limit for pipeline waits; kSpinLimit for a
// kernel's final wait for its own MMAs, which must complete before the tensor memory is released).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long limit = kSpinLimit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it) done = mbar_try(bar, parity);
    return mbar_uniform(bar, parity, done);
}
// mbar_wait that also gives up once *abort is set (by the other side of a warp-specialised pipeline).
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, const volatile int* abort,
                                             long limit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it) {
        done = mbar_try(bar, parity);
        if (!done && (it & 255) == 255 && *abort) break;
    }
    return mbar_uniform(bar, parity, done);
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// Pre-sliced stages arrive by bulk copies (the TMA engine, no tensor map): the issuing thread arms the
// stage's load barrier with the byte count, and each copy completes its share of the transaction on it.
// Sizes are multiples of 16 bytes and both addresses 16-byte aligned (64 KB / 4 KB / 32 KB images at
// 1 KB-aligned stage buffers).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// A hint to bring `bytes` (a multiple of 16, 16-byte aligned source) into L2 ahead of a bulk copy: with two
// stage buffers a stage's copy is issued only when the MMAs two stages back are done, so a stage coming
// cold from HBM would leave the tensor core waiting for the whole DRAM latency.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
}
// Stages prefetched into L2 ahead of the stage being copied (64 KB each: 152 SMs x 4 x 64 KB = 39 MB of L2).
constexpr int kPrefetchAhead = 4;

// Before a kernel that issued bulk copies returns (also after a timeout): the last copy issued into each
// stage buffer has landed (parity of its phase), bounded like every wait.
__device__ __forceinline__ bool bulk_drain(uint64_t* load_bar, const int64_t (&issued)[2]) {
    bool ok = true;
    for (int b = 0; b < 2; ++b)
        if (issued[b] > 0) {
            const uint32_t par = static_cast<uint32_t>((issued[b] - 1) & 1);
            uint32_t done = 0;
            for (long it = 0; it < kSpinLimit && !done; ++it) done = mbar_try(&load_bar[b], par);
            ok = ok && done;
        }
    return ok;
}

// Barrier 1 over the n producer threads only (the MMA warp does not take part).
__device__ __forceinline__ void prod_sync(int n) { asm volatile("bar.sync 1, %0;\n" ::"r"(n) : "memory"); }
__device__ __forceinline__ bool prod_sync_or(bool v, int n) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(addr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t addr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// 56-bit fixed-point magnitude F = floor(|x| 2^{56-E}) of x relative to the bound 2^E > |x|, split in
// two 28-bit halves (hi: slices 1..4, lo: slices 5..8).  0 for zero, subnormal, non-finite or unknown E.
// Branch-free: F = (mantissa 2^3) >> (3 - sh) with sh = ex - 1019 - E <= 3 for a valid bound (a larger
// sh, |x| >= 2^E, saturates).
__device__ __forceinline__ void fixed56(double x, int E, uint32_t& fhi, uint32_t& flo) {
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
    const int ex = static_cast<int>((bits >> 52) & 0x7FF);
    const unsigned long long mant8 = ((bits & ((1ull << 52) - 1)) | (1ull << 52)) << 3;   // < 2^56
    const int r = E + 1022 - ex;
    unsigned long long F = mant8 >> (r < 63 ? (r > 0 ? r : 0) : 63);
    F = r < 0 ? (1ull << 56) - 1 : F;
    F = (ex != 0 && ex != 0x7FF && E > kNoExp) ? F : 0ull;
    fhi = static_cast<uint32_t>(F >> 28);
    flo = static_cast<uint32_t>(F) & 0x0FFFFFFFu;
}

// Two 7-bit fields (bits pos..pos+6 of u0 and u1) as a packed BF16 pair (u0 in the low half), signed:
// the pair of BF16 numbers 128 + v (exponent 7, mantissa v) goes through one packed BF16 FMA,
// (128 + v) s - 128 s = s v, exact.  sgn2: the BF16 pair (s0, s1), s = +-1; off2: (-128 s0, -128 s1).
__device__ __forceinline__ uint32_t bf16x2_field(uint32_t u0, uint32_t u1, int pos, uint32_t sgn2, uint32_t off2) {
    const uint32_t t = ((u0 >> pos) & 0x7Fu) | (((u1 >> pos) & 0x7Fu) << 16) | 0x43004300u;
    uint32_t r;
    asm("fma.rn.bf16x2 %0, %1, %2, %3;\n" : "=r"(r) : "r"(t), "r"(sgn2), "r"(off2));
    return r;
}

// Slice the 8 values x[0..7] (consecutive K) and store slice a of all eight as one 16-byte core-matrix
// row at dst + a * slice_bytes (x[i] in BF16 lane i).  Every slice carries the sign of its value.
__device__ __forceinline__ void slice_store8(const double (&x)[8], int E, uint8_t* dst, int slice_bytes) {
    uint32_t fh[8], fl[8], sgn2[4], off2[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) fixed56(x[i], E, fh[i], fl[i]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool n0 = __double_as_longlong(x[2 * j]) < 0, n1 = __double_as_longlong(x[2 * j + 1]) < 0;
        sgn2[j] = (n0 ? 0xBF80u : 0x3F80u) | ((n1 ? 0xBF80u : 0x3F80u) << 16);    // -1 / +1
        off2[j] = (n0 ? 0x4300u : 0xC300u) | ((n1 ? 0x4300u : 0xC300u) << 16);    // +128 / -128
    }
#pragma unroll
    for (int a = 0; a < kSlices; ++a) {
        const int pos = 21 - 7 * (a & 3);
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            w[j] = a < 4 ? bf16x2_field(fh[2 * j], fh[2 * j + 1], pos, sgn2[j], off2[j])
                         : bf16x2_field(fl[2 * j], fl[2 * j + 1], pos, sgn2[j], off2[j]);
        *reinterpret_cast<uint4*>(dst + a * slice_bytes) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Exact combination of the eight group sums M_d (d = 2..9) of one output element:
//   I = sum_{d=2..6} M_d 2^{7(6-d)}  (units of 2^-42 of the operand scale, |I| < 2^50),
//   L = sum_{d=7..9} M_d 2^{7(9-d)}  (units of 2^-63, |L| < 2^39).
__device__ __forceinline__ void combine_groups(const float (&m)[kGroups], long long& I, long long& L) {
    I = (static_cast<long long>(__float2int_rn(m[0])) << 28) +
        (static_cast<long long>(__float2int_rn(m[1])) << 21) +
        (static_cast<long long>(__float2int_rn(m[2])) << 14) +
        (static_cast<long long>(__float2int_rn(m[3])) << 7) + static_cast<long long>(__float2int_rn(m[4]));
    L = (static_cast<long long>(__float2int_rn(m[5])) << 14) +
        (static_cast<long long>(__float2int_rn(m[6])) << 7) + static_cast<long long>(__float2int_rn(m[7]));
}
// For K <= 32 every group sum is below 8 * 127^2 * 32 < 2^22 in magnitude, so M + 1.5 2^23 holds M
// exactly in its low mantissa bits: the integer is read from the bit pattern (no conversion
// instruction), and pairs of neighbouring groups fit one int32 (M_d 2^7 + M_{d+1} < 2^30), leaving
// three 32 x 32 -> 64-bit multiply-adds for the int64 part.
__device__ __forceinline__ long long combine_units53_k32(const float (&m)[kGroups]) {
    int v[kGroups];
#pragma unroll
    for (int g = 0; g < kGroups; ++g) v[g] = __float_as_int(m[g] + 12582912.0f) - 0x4B400000;
    const int u = v[1] * 128 + v[2], t = v[3] * 128 + v[4], w = v[6] * 128 + v[7];
    const long long I = static_cast<long long>(v[0]) * (1ll << 28) +
                        (static_cast<long long>(u) * (1ll << 14) + static_cast<long long>(t));
    const long long L = static_cast<long long>(v[5]) * (1ll << 14) + static_cast<long long>(w);
    return I * 2048 + ((L + 512) >> 10);
}
// the value in units of 2^-53 (rounded), for a single-window product: |result| < 2^61
__device__ __forceinline__ long long combine_units53(const float (&m)[kGroups]) {
    long long I, L;
    combine_groups(m, I, L);
    return (I << 11) + ((L + 512) >> 10);
}
// the value in units of 2^-49 (rounded), accumulated across windows
__device__ __forceinline__ long long combine_units49(const float (&m)[kGroups]) {
    long long I, L;
    combine_groups(m, I, L);
    return (I << 7) + ((L + (1ll << 13)) >> 14);
}

// I * 2^e: I converted to FP64 (rounded to nearest above 2^53), exponent added in the bit pattern
// when the result stays normal (the usual case), ldexp otherwise.
__device__ __forceinline__ double scale_pow2(long long I, int e) {
    if (I == 0) return 0.0;
    const double v = static_cast<double>(I);
    const long long bits = __double_as_longlong(v);
    const int ex = static_cast<int>((bits >> 52) & 0x7FF);
    if (ex + e > 0 && ex + e < 0x7FF) return __longlong_as_double(bits + (static_cast<long long>(e) << 52));
    return ldexp(v, e);
}

// Add the eight TMEM group sums of this thread's row and its NC columns (col0.. of the 64-column tile,
// read CW at a time) to int64 accumulators in units of 2^-53 (U53) or 2^-49 of the operand scale.
// The sliced operands are below 0.51 of their power-of-two bounds, so a K-term sum stays below
// 0.26 K scale: units of 2^-53 hold K < 2^10 / 0.26 (about 3900) terms -- the products take K <= 2048,
// a factor 2 below -- and units of 2^-49 hold 2^14 (a 64-window flush of the Gram).
template <bool U53, int NC, int CW = 8>
__device__ __forceinline__ void drain_acc(uint32_t tmem, int warp, int col0, long long (&acc)[NC]) {
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += CW) {
        float mg[kGroups][CW];
#pragma unroll
        for (int g = 0; g < kGroups; ++g)
            if constexpr (CW == 8) tmem_ld8(tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + g * kTileN + col0 + c0, mg[g]);
            else tmem_ld4(tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + g * kTileN + col0 + c0, mg[g]);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            float grp[kGroups];
#pragma unroll
            for (int g = 0; g < kGroups; ++g) grp[g] = mg[g][j];
            acc[c0 + j] += U53 ? combine_units53(grp) : combine_units49(grp);
        }
    }
}

// Issue the 72 MMAs of one stage: all pairs (a, b), a + b <= 9, for the two K=16 steps, one N = 64 MMA
// per pair (any slice stride of B: used when B's slices are not stored back to back).
// first_window: the stage starts an exactness window (the first MMA into each accumulator clears it).
// The descriptors of the stage's two base addresses are formed once; every MMA adds its (constant)
// offset to the 14-bit start field, which cannot carry (shared memory < 256 KB).
__device__ __forceinline__ void issue_stage_pairs(uint32_t tmem, uint32_t a_base, uint32_t b_base,
                                                  uint32_t b_slice_bytes, bool first_window) {
    const uint64_t a0 = sdesc(a_base), b0 = sdesc(b_base);
    const uint32_t bstep = b_slice_bytes >> 4;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int d = 2; d <= 9; ++d) {
            const int alo = d - 8 > 1 ? d - 8 : 1, ahi = d - 1 < 8 ? d - 1 : 8;
#pragma unroll
            for (int a = alo; a <= ahi; ++a) {
                const int b = d - a;
                const uint64_t ad = a0 + static_cast<uint32_t>(((a - 1) * kASlice + kk * 256) >> 4);
                const uint64_t bd = b0 + (static_cast<uint32_t>(b - 1) * bstep + static_cast<uint32_t>(kk * 16));
                const uint32_t acc = (first_window && kk == 0 && a == alo) ? 0u : 1u;
                mma_bf16(tmem + (d - 2) * kTileN, ad, bd, acc);
            }
        }
    }
}

// The same 36 pairs per K = 16 step in 12 MMAs, for B slices stored back to back (kBSlice apart: the
// eight 64-row slices form one 512-row operand in the same core-matrix layout).  For slice a of X the
// pairs (a, b), b = 1 .. 9 - a, go to the groups d = a + b, whose accumulators are adjacent 64-column
// ranges of tensor memory: one MMA with N = 64 nb multiplies slice a by nb consecutive B slices at once
// (N <= 256, so slices 1-4 and 5-8 are two MMAs).  Same products, same exact integer sums.
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t a_base, uint32_t b_base, bool first_window) {
    const uint64_t a0 = sdesc(a_base), b0 = sdesc(b_base);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int a = 1; a <= 8; ++a) {
            const int nb = 9 - a;
            const int n1 = nb < 4 ? nb : 4;
            const uint64_t ad = a0 + static_cast<uint32_t>(((a - 1) * kASlice + kk * 256) >> 4);
            const uint32_t acc = (first_window && kk == 0 && a == 1) ? 0u : 1u;
            mma_bf16_n(tmem + (a - 1) * kTileN, ad, b0 + static_cast<uint32_t>(kk * 16), idesc_bf16(kTileN * n1),
                       acc);
            if (nb > 4)
                mma_bf16_n(tmem + (a + 3) * kTileN, ad,
                           b0 + static_cast<uint32_t>((4 * kBSlice) >> 4) + static_cast<uint32_t>(kk * 16),
                           idesc_bf16(kTileN * (nb - 4)), acc);
        }
    }
}

struct TmemState {
    uint32_t base;
};

// ---- column slices of a small K x N matrix Y (the B operand of k_ozaki_gemm_ws and k_ozaki_update) --
// yexp[q] = exponent bound of column q over its K rows; blocks[(tn*nkw + kw)*8 + b] (4 KB each) hold
// slice b of columns 64tn..64tn+63 and rows 32kw..32kw+31 in the core-matrix K-major layout.
// Y rows >= K and columns >= N read as 0.  One CTA per (tn, kw), 256 threads: (column, 8-row chunk).
__global__ void __launch_bounds__(256) k_ozaki_slice_cols(const double* __restrict__ Y, int64_t ldy, int K,
                                                          int N, uint8_t* __restrict__ blocks,
                                                          int32_t* __restrict__ yexp, const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int tn = blockIdx.x, kw = blockIdx.y, nkw = gridDim.y;
    const int q = threadIdx.x & 63, c = threadIdx.x >> 6;   // 64 columns x 4 chunks of 8 rows
    const int col = tn * kTileN + q;
    int E = kNoExp;
    if (col < N)
        for (int k = 0; k < K; ++k) {
            const int e = exp_bound(Y[static_cast<int64_t>(k) * ldy + col]);
            E = e > E ? e : E;
        }
    if (kw == 0 && c == 0 && col < N) yexp[col] = E;
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = kw * kKW + 8 * c + i;
        x[i] = (col < N && k < K) ? Y[static_cast<int64_t>(k) * ldy + col] : 0.0;
    }
    uint8_t* blk = blocks + static_cast<size_t>((tn * nkw + kw) * kSlices) * kBSlice;
    slice_store8(x, E, blk + core_off(q, 16 * c), kBSlice);
}

// ---- stage images of X's row slices ------------------------------------------------------------------
// img[(tm * nkw + kw) * kAStage ..] = the eight 8 KB slices of rows 128 tm .. 128 tm + 127, K values
// 32 kw .. 32 kw + 31 of X, in the core-matrix layout of a k_ozaki_gemm_ws stage buffer, against the row
// bounds xexp: exactly what that kernel's producers would slice for the stage (zeros outside X).  One
// CTA per (row tile, K stage), one thread per (row, 8-value chunk).  Skipped when *info != 0.
__global__ void __launch_bounds__(512) k_slice_images(const double* __restrict__ X, int64_t ldx, int64_t m, int K,
                                                      const int32_t* __restrict__ xexp, uint8_t* __restrict__ img,
                                                      const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int nkw = (K + kKW - 1) / kKW;
    const int64_t tm = blockIdx.x;
    const int kw = blockIdx.y;
    const int lr = threadIdx.x & (kTileM - 1), c = threadIdx.x >> 7;
    const int64_t row = tm * kTileM + lr;
    const int E = row < m ? xexp[row] : kNoExp;
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = kw * kKW + 8 * c + i;
        x[i] = (row < m && k < K) ? X[row * ldx + k] : 0.0;
    }
    slice_store8(x, E, img + static_cast<size_t>(tm * nkw + kw) * kAStage + core_off(lr, 16 * c), kASlice);
}

// ---- stage images of X's column slices (the split Gram's operands) -------------------------------------
// img[(blk * nst + st) * kAStage ..] = the eight 8 KB slices of columns 128 blk .. 128 blk + 127 (the
// tile's M dimension) over rows 32 st .. 32 st + 31 (K) of X, against the column bounds colexp, in the
// layout k_ozaki_gram's producers would slice them (zeros outside X); nst = ceil(m / 32).
__global__ void __launch_bounds__(512) k_slice_col_images(const double* __restrict__ X, int64_t ldx, int64_t m,
                                                          int n, const int32_t* __restrict__ colexp,
                                                          uint8_t* __restrict__ img, const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int64_t nst = (m + kKW - 1) / kKW;
    const int blk = blockIdx.y;
    const int64_t st = blockIdx.x;
    const int lr = threadIdx.x & (kTileM - 1), c = threadIdx.x >> 7;
    const int p = 128 * blk + lr;
    const int E = p < n ? colexp[p] : kNoExp;
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = st * kKW + 8 * c + i;
        x[i] = (row < m && p < n) ? X[row * ldx + p] : 0.0;
    }
    slice_store8(x, E, img + static_cast<size_t>(blk * nst + st) * kAStage + core_off(lr, 16 * c), kASlice);
}

// ---- stage images of up to 128 finished columns, against their own row bounds --------------------------
// The left-looking wide first pass slices its finished 64-column blocks in pairs: columns c0 .. c0 + nc - 1
// of X (nc <= 128: one block, or a pair) become stages kw0 .. kw0 + ceil(nc / 32) - 1 of row tile tm's
// image (img_nkw stages per row tile), sliced against the row's bound over those columns alone, written
// to bexp[row].  The products that read the image take each such group of up to 128 columns as one
// exactness window with its own row bound.  One CTA per 64 rows (half a 128-row tile): the rows are
// copied into shared memory in whole rows (consecutive lanes, consecutive columns), then thread (row, q)
// takes stage kw0 + q (values 32 q .. 32 q + 31 of its row); the row bound is the maximum over the four.
constexpr int kSbRows = 64;
constexpr int kSbLd = 129;   // odd row stride (doubles): 8-byte reads of 32 consecutive rows hit distinct banks
constexpr int kSbSmem = kSbRows * kSbLd * 8;
__global__ void __launch_bounds__(256) k_slice_block_images(const double* __restrict__ X, int64_t ldx, int64_t m,
                                                            int nc, uint8_t* __restrict__ img, int img_nkw, int kw0,
                                                            int32_t* __restrict__ bexp, const int32_t* info) {
    extern __shared__ double sb_tile[];
    __shared__ int red[4][kSbRows];
    if (info && load_status(info) != 0) return;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kSbRows;
    const int tid = threadIdx.x;
    for (int e = tid; e < kSbRows * nc; e += 256) {
        const int r = e / nc, c = e - r * nc;
        const bool ok = r0 + r < m;
        cp_async8(&sb_tile[r * kSbLd + c], ok ? X + (r0 + r) * ldx + c : X, ok);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const int lr = tid & (kSbRows - 1), q = tid >> 6;
    const int64_t row = r0 + lr;
    const double* xr = sb_tile + lr * kSbLd;
    int e = kNoExp;
    if (row < m) {
#pragma unroll 8
        for (int i = 0; i < 32; ++i) {
            const int k = 32 * q + i;
            const int ek = exp_bound(k < nc ? xr[k] : 0.0);
            e = ek > e ? ek : e;
        }
    }
    red[q][lr] = e;
    __syncthreads();
    int E = red[0][lr];
#pragma unroll
    for (int j = 1; j < 4; ++j) E = red[j][lr] > E ? red[j][lr] : E;
    if (q == 0 && row < m) bexp[row] = E;
    if (32 * q >= nc) return;   // no stage of this group
    const int64_t tm = r0 / kTileM;
    const int tr = static_cast<int>(r0 - tm * kTileM) + lr;   // row inside the 128-row stage tile
    uint8_t* dst = img + static_cast<size_t>(tm * img_nkw + kw0 + q) * kAStage;
    for (int c = 0; c < 4; ++c) {
        double x8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = 32 * q + 8 * c + i;
            x8[i] = (row < m && k < nc) ? xr[k] : 0.0;
        }
        slice_store8(x8, E, dst + core_off(tr, 16 * c), kASlice);
    }
}

// ---- C = X Y, warp-specialised: helpers ------------------------------------------------------------
// 128 rows x 32 K values of X (rows row0.., columns k0..) into R, one 8-byte cp.async per value, zero
// outside the matrix; the 32 lanes of a warp copy one row.
template <int NT>
__device__ __forceinline__ void prefetch_x(const double* X, int64_t ldx, int64_t m, int K, int64_t row0, int k0,
                                           double* R, int tid) {
#pragma unroll
    for (int i = 0; i < kTileM * kKW / NT; ++i) {
        const int e = tid + i * NT;
        const int r = e >> 5, k = e & 31;
        const int64_t row = row0 + r;
        const bool ok = row < m && k0 + k < K;
        cp_async8(R + r * kRawLd + k, ok ? X + row * ldx + k0 + k : X, ok);
    }
}

// Write the finished tile (rows row0 + 0..127, columns 64 tn + 0..63) of C = X Y through the staging
// buffer W (run by the NT producer threads): each thread puts its row's NC values into W, then the tile
// is written in whole rows.  The values come from the TMEM accumulators (single window) or from acc (WIN).
template <bool WIN, bool SUB, int NT, int NC>
__device__ __forceinline__ void gemm_store_tile(uint32_t tmem, int warp, int tid, int64_t row0, int tn, int E,
                                                int N, const int32_t* __restrict__ yexp, const double* B,
                                                int64_t ldb, double* C, int64_t ldc, int64_t m, double* W,
                                                long long (&acc)[NC]) {
    const int lr = tid & (kTileM - 1), rq = tid / kTileM;
    const int col0 = tn * kTileN;
    const int ncols = N - col0 < kTileN ? N - col0 : kTileN;
    double* wr = W + lr * kEpiLd + NC * rq;
    if (WIN) {
        drain_acc<true, NC, 4>(tmem, warp, NC * rq, acc);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const int col = col0 + NC * rq + j;
            const int ey = col < N ? yexp[col] : kNoExp;
            const double v = (E > kNoExp && ey > kNoExp) ? scale_pow2(acc[j], E + ey - 53) : 0.0;
            wr[j] = v;
        }
    } else {
#pragma unroll 1
        for (int c0 = 0; c0 < NC; c0 += 8) {
            float mg[kGroups][8];
#pragma unroll
            for (int g = 0; g < kGroups; ++g)
                tmem_ld8(tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + g * kTileN + NC * rq + c0, mg[g]);
            tmem_wait_ld();
            if (col0 + NC * rq + c0 >= N) continue;   // (warp-uniform) no valid column in this chunk
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = col0 + NC * rq + c0 + j;
                float grp[kGroups];
#pragma unroll
                for (int g = 0; g < kGroups; ++g) grp[g] = mg[g][j];
                if (col < N) {
                    const long long I = combine_units53(grp);
                    const int ey = yexp[col];
                    const double v = (E > kNoExp && ey > kNoExp) ? scale_pow2(I, E + ey - 53) : 0.0;
                    wr[c0 + j] = v;
                }
            }
        }
    }
    prod_sync(NT);
#pragma unroll 8
    for (int i = 0; i < kTileM * kTileN / NT; ++i) {
        const int e = tid + i * NT;
        const int r = e >> 6, c = e & 63;
        const int64_t row = row0 + r;
        if (row < m && c < ncols) {
            // SUB: C = B - X Y, B read in whole rows like C is written (B may be C itself)
            if (SUB) C[row * ldc + col0 + c] = B[row * ldb + col0 + c] - W[r * kEpiLd + c];
            else C[row * ldc + col0 + c] = W[r * kEpiLd + c];
        }
    }
    fence_async_smem();   // the next bulk copy into this buffer (async proxy) follows these accesses
    prod_sync(NT);        // W (a stage buffer) is free again
}

// ---- C = X Y (SUB = false: pass 2, Q = A_1 R_1^{-1}) or C = B - X Y (SUB = true: the off-diagonal block
// updates of the wide first pass), warp-specialised ---------------------------------------------------
// X: m x K FP64 (ldx) with row exponent bounds xexp[m] (max over the K columns used);
// Y: pre-sliced by k_ozaki_slice_cols (K x N, column bounds yexp[N]);
// B, C: m x N FP64 (ldb, ldc); C may equal B.  Persistent grid over 128-row x 64-column tiles.
// WIN (128 < K <= 1024): the K range is cut into exactness windows of 128, each drained into int64
// accumulators in units of 2^-53 of the scale (the same resolution as a single window).
// The CTA's (tile, K-stage) sequence is one stream of stages over two shared-memory buffers: stage g is
// sliced while the MMAs of stage g - 1 run; when stage g opens a new exactness window (or a new tile)
// the previous window's accumulators are drained (into int64, or out to C at a tile end) before its
// MMAs are issued.  The raw X rows of stage g + 1 are copied (cp.async, whole rows per warp) while
// stage g is sliced, and the finished tile is written (B read) in whole rows through a free stage
// buffer.  Warp roles: NT producer
// threads (warps 0 .. NT/32 - 1) copy, slice and drain; the last warp issues the MMAs.  full[s]: the
// producer warps filled stage buffer s (one arrival per warp); empty[s]: the MMAs of the stage in
// buffer s are done (tcgen05.commit).  A drain waits for empty of the stage before and
// arrives on full of the next stage only after it, so the next tile's MMAs start once TMEM is read out.
// The K stages the output tile of column tile tn needs: all nkw, or, with an upper-triangular Y (tri),
// those up to the last K row its columns reach (k < 64 (tn + 1)); the stages after it multiply zeros.
__device__ __forceinline__ int tile_stages(int tn, int nkw, bool tri) {
    if (!tri) return nkw;
    const int last = ((tn + 1) * kTileN + kKW - 1) / kKW;
    return last < nkw ? last : nkw;
}

// Column tile of tile t (row tile t / ntn).  With a triangular Y the tiles' costs differ (2 (tn + 1)
// stages), and a grid that is a multiple of ntn would give every CTA one fixed tn: the column tile is
// rotated by the row tile, so a CTA's tiles t, t + gridDim.x, ... cycle through all tn, while the ntn
// tiles of one row tile still run side by side (their A stages shared in L2).
__device__ __forceinline__ int tile_col(int64_t t, int ntn, bool tri) {
    const int j = static_cast<int>(t % ntn);
    return tri ? static_cast<int>((j + t / ntn) % ntn) : j;
}

// Walks the stages of the output tiles one CTA owns (tiles t = blockIdx.x, + gridDim.x, ...; stages
// kw = 0 .. tile_stages - 1 of each).
struct StageWalk {
    int64_t t;
    int tn, kw, nk, ntn, nkw;
    bool tri;
    __device__ __forceinline__ StageWalk(int ntn_, int nkw_, bool tri_)
        : t(blockIdx.x), kw(0), ntn(ntn_), nkw(nkw_), tri(tri_) {
        tn = tile_col(t, ntn, tri);
        nk = tile_stages(tn, nkw, tri);
    }
    __device__ __forceinline__ void advance() {
        if (++kw == nk) {
            kw = 0;
            t += gridDim.x;
            tn = tile_col(t, ntn, tri);
            nk = tile_stages(tn, nkw, tri);
        }
    }
};

template <bool WIN, bool SUB>
__global__ void __launch_bounds__((WIN ? kThreadsWin : kThreads) + 32, 1)
k_ozaki_gemm_ws(const double* X, int64_t ldx, const int32_t* __restrict__ xexp, int K,
                const uint8_t* __restrict__ yblocks, const int32_t* __restrict__ yexp, int N, const double* B,
                int64_t ldb, double* C, int64_t ldc, int64_t m, int32_t* info, long spin, int tri) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t empty_bar[2], full_bar[2], done_bar;
    __shared__ uint32_t tslot;
    __shared__ int abort_s;
    if (load_status(info) != 0) return;
    constexpr int NT = WIN ? kThreadsWin : kThreads;
    constexpr int NC = Share<NT>::kDrainCols, NCH = Share<NT>::kChunks;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* stA[2] = {sm, sm + kStageBytes};
    uint8_t* stB[2] = {sm + kAStage, sm + kStageBytes + kAStage};
    double* R = reinterpret_cast<double*>(sm + 2 * kStageBytes);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tslot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty_bar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&full_bar[i])), "r"(NT / 32));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        abort_s = 0;
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tslot;

    const int nkw = (K + kKW - 1) / kKW;
    const int ntn = (N + kTileN - 1) / kTileN;
    const int64_t ntm = (m + kTileM - 1) / kTileM;
    const int64_t ntiles = ntm * ntn;
    const int64_t my_tiles =
        static_cast<int64_t>(blockIdx.x) < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    int64_t nstages = 0;
    if (tri) {
        for (int64_t u = 0; u < my_tiles; ++u)
            nstages += tile_stages(tile_col(blockIdx.x + u * gridDim.x, ntn, true), nkw, true);
    } else {
        nstages = my_tiles * nkw;
    }

    if (warp == NT / 32) {
        // MMA warp: one lane issues every stage once the producers have filled it
        if (lane == 0) {
            uint32_t fphase[2] = {0u, 0u};
            StageWalk wk(ntn, nkw, tri != 0);
            for (int64_t g = 0; g < nstages; ++g, wk.advance()) {
                const int s = static_cast<int>(g & 1);
                if (!mbar_wait_ab(&full_bar[s], fphase[s], &abort_s, spin)) {
                    abort_s = 1;
                    break;
                }
                fphase[s] ^= 1u;
                tc_after_sync();
                issue_stage(tmem, smem_u32(stA[s]), smem_u32(stB[s]), (wk.kw & 3) == 0);
                mma_commit(&empty_bar[s]);
            }
            // every MMA issued here is complete before the tensor memory is released
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0u)) abort_s = 1;
        }
        __syncwarp();
    } else {
        const int lr = tid & (kTileM - 1);  // tile row: producer row and drain row (TMEM lane)
        const int rq = tid >> 7;            // producer K chunk(s) NCH*rq..; drain columns NC*rq..
        uint32_t phase[2] = {0u, 0u};
        bool pending[2] = {false, false};
        bool timed_out = false;
        long long acc[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = 0;
        int64_t cur_row0 = 0;               // the tile whose accumulators are in TMEM
        int cur_tn = 0, cur_E = kNoExp;
        StageWalk wk(ntn, nkw, tri != 0);   // stage g
        if (nstages > 0) prefetch_x<NT>(X, ldx, m, K, (wk.t / ntn) * kTileM, wk.kw * kKW, R, tid);
        cp_async_commit();

        for (int64_t g = 0; g < nstages; ++g, wk.advance()) {
            const int s = static_cast<int>(g & 1);
            const int64_t t = wk.t;
            const int kw = wk.kw;
            const int64_t tm = t / ntn;
            const int tn = wk.tn;
            const int64_t row = tm * kTileM + lr;
            const int E = row < m ? xexp[row] : kNoExp;
            // buffer s is free once the MMAs of stage g - 2 are done
            if (pending[s]) {
                const bool ok = mbar_wait_ab(&empty_bar[s], phase[s], &abort_s, spin);
                if (prod_sync_or(!ok, NT)) { timed_out = true; break; }
                phase[s] ^= 1u;
                pending[s] = false;
            }
            // B slices of stage g: one contiguous 32 KB block
            const uint8_t* src = yblocks + static_cast<size_t>((tn * nkw + kw) * kSlices) * kBSlice;
            {
                for (int e = tid; e < kBStage / 16; e += NT) {
                    const unsigned dst = smem_u32(stB[s] + 16 * e);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + 16 * e));
                }
                cp_async_commit();
                // the raw X rows of stage g (copied during stage g - 1) are complete: slice this thread's row
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                prod_sync(NT);
#pragma unroll
                for (int cc = 0; cc < NCH; ++cc) {
                    const int c = NCH * rq + cc;
                    const double2* rp = reinterpret_cast<const double2*>(R + lr * kRawLd + 8 * c);
                    double x[8];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const double2 v = rp[i];
                        x[2 * i] = v.x;
                        x[2 * i + 1] = v.y;
                    }
                    slice_store8(x, E, stA[s] + core_off(lr, 16 * c), kASlice);
                }
                // R is free: copy the raw X rows of stage g + 1
                prod_sync(NT);
                if (g + 1 < nstages) {
                    StageWalk nx = wk;
                    nx.advance();
                    prefetch_x<NT>(X, ldx, m, K, (nx.t / ntn) * kTileM, nx.kw * kKW, R, tid);
                }
                cp_async_commit();
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // the B slices of stage g
            }
            fence_async_smem();
            // stage g opens an exactness window: drain the previous window's accumulators first
            if (g > 0 && (kw & 3) == 0) {
                const int sp = s ^ 1;
                if (pending[sp]) {
                    const bool ok = mbar_wait_ab(&empty_bar[sp], phase[sp], &abort_s, spin);
                    if (prod_sync_or(!ok, NT)) { timed_out = true; break; }
                    phase[sp] ^= 1u;
                    pending[sp] = false;
                }
                tc_after_sync();
                if (kw == 0) {
                    // every MMA so far is complete: stage sp's buffer stages the output tile
                    gemm_store_tile<WIN, SUB, NT, NC>(tmem, warp, tid, cur_row0, cur_tn, cur_E, N, yexp, B, ldb, C, ldc, m,
                                                 reinterpret_cast<double*>(stA[sp]), acc);
#pragma unroll
                    for (int j = 0; j < NC; ++j) acc[j] = 0;
                } else if (WIN) {
                    drain_acc<true, NC, 4>(tmem, warp, NC * rq, acc);
                }
            }
            if (kw == 0) {
                cur_row0 = tm * kTileM;
                cur_tn = tn;
                cur_E = E;
            }
            // stage g is ready (and TMEM drained if it opens a window): hand it to the MMA warp
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[s]);
            pending[s] = true;
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        // the last tile
        if (!timed_out && nstages > 0) {
            for (int s = 0; s < 2 && !timed_out; ++s)
                if (pending[s]) {
                    const bool ok = mbar_wait_ab(&empty_bar[s], phase[s], &abort_s, spin);
                    if (prod_sync_or(!ok, NT)) { timed_out = true; break; }
                    phase[s] ^= 1u;
                    pending[s] = false;
                }
            if (!timed_out) {
                tc_after_sync();
                gemm_store_tile<WIN, SUB, NT, NC>(tmem, warp, tid, cur_row0, cur_tn, cur_E, N, yexp, B, ldb, C, ldc, m,
                                             reinterpret_cast<double*>(stA[0]), acc);
            }
        }
        if (timed_out) abort_s = 1;
    }

    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0 && abort_s) set_status(info, RPCHOLQR_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// ---- C = X Y / C = B - X Y from stage images, with the accumulators double-buffered ------------------------
// The product over pre-sliced X (k_slice_images) for the wide passes: pass 2 (Q = A_1 R_1^{-1}, Y upper
// triangular) and the left-looking block updates of the first pass (C = B - X Y, K up to 2048).  Output
// tiles of 128 rows x 32 columns, so that one exactness window's eight group accumulators take 256 TMEM
// columns and two sets fit: consecutive windows of a CTA (within a tile and across its tiles) alternate
// between the sets, so a window's drain (the eight FP32 group sums into int64, or the tile's result out
// to C) runs while the tensor core fills the other set.  Warp roles: warps 0-7 drain (two threads per
// tile row, 16 columns each: warp w reads TMEM lanes 32 (w % 4)..), warp 8 lane 0 streams the stages
// (one 64 KB bulk copy of X's stage image, eight 2 KB copies of Y's slices, on the stage's load barrier),
// warp 9 lane 0 issues the MMAs (8 per K = 16 step: Y's eight 32-column slices are stacked, N = 32 (9 - a)
// for slice a of X).  Barriers: load[s] (bytes landed) and empty[s] (MMAs of the stage done) per stage
// buffer; acc_full[b] (the window's MMAs done) and acc_empty[b] (the set read out) per accumulator set.
// The arithmetic is that of k_ozaki_gemm_ws: the same slices, exact group sums per window of 128, the
// same int64 combination in units of 2^-53, so the results are the same bits.
constexpr int kDbN = 32;
constexpr int kDbBSlice = kDbN * kKW * 2;            // 2 KB: one slice of a 32-column tile's stage
constexpr int kDbBStage = kSlices * kDbBSlice;       // 16 KB
constexpr int kDbStage = kAStage + kDbBStage;        // 80 KB
constexpr int kDbEpiWarps = 8;
constexpr int kDbEpi = 32 * kDbEpiWarps;             // 256 drain threads
constexpr int kDbThreads = kDbEpi + 64;              // + the copy warp and the MMA warp
constexpr int kDbCols = kDbN / (kDbEpi / kTileM);    // 16 columns per drain thread
constexpr int kDbEpiLd = kDbN + 1;
constexpr int kDbSmem = 2 * kDbStage + kTileM * kDbEpiLd * 8;
static_assert(kDbSmem + 1024 <= 232448, "k_ozaki_gemm_db exceeds the 227 KB shared-memory limit");

// K stages an output tile of 32-column tile tn needs (tri: those up to the last K row its columns reach).
__device__ __forceinline__ int db_tile_stages(int tn, int nkw, bool tri) {
    if (!tri) return nkw;
    const int last = ((tn + 1) * kDbN + kKW - 1) / kKW;
    return last < nkw ? last : nkw;
}

// The 36 slice pairs of one 32-wide K stage into accumulator set `tset` (group d at columns (d - 2) 32):
// 8 MMAs per K = 16 step; `first`: the stage opens a window (the a = 1 MMA clears all eight groups).
__device__ __forceinline__ void issue_stage_n32(uint32_t tset, uint32_t a_base, uint32_t b_base, bool first) {
    const uint64_t a0 = sdesc(a_base), b0 = sdesc(b_base);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int a = 1; a <= 8; ++a) {
            const uint64_t ad = a0 + static_cast<uint32_t>(((a - 1) * kASlice + kk * 256) >> 4);
            mma_bf16_n(tset + (a - 1) * kDbN, ad, b0 + static_cast<uint32_t>(kk * 16), idesc_bf16(kDbN * (9 - a)),
                       (first && kk == 0 && a == 1) ? 0u : 1u);
        }
    }
}

// I 2^-sh rounded to nearest (ties up), sh >= 0; |I| < 2^62.
__device__ __forceinline__ long long shift_round(long long I, int sh) {
    if (sh == 0) return I;
    if (sh > 62) return 0;
    return (I + (1ll << (sh - 1))) >> sh;
}

// Add one window's eight group sums of this thread's row (TMEM address taddr: set + lane quarter) and
// columns col0 .. col0 + NC - 1 of the 32-column tile to int64 accumulators in units of 2^-53 (U49: 2^-49)
// of the window's scale, shifted down by sh bits (a window sliced against a row bound 2^sh below the
// tile's).
template <int NC, bool U49 = false>
__device__ __forceinline__ void drain_set32(uint32_t taddr, int col0, int sh, long long (&acc)[NC]) {
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += 8) {
        float mg[kGroups][8];
#pragma unroll
        for (int g = 0; g < kGroups; ++g) tmem_ld8(taddr + g * kDbN + col0 + c0, mg[g]);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float grp[kGroups];
#pragma unroll
            for (int g = 0; g < kGroups; ++g) grp[g] = mg[g][j];
            acc[c0 + j] += shift_round(U49 ? combine_units49(grp) : combine_units53(grp), sh);
        }
    }
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, %0;\n" ::"r"(kDbEpi) : "memory"); }
// Barrier 2 over the drain warps with an OR of v: a wait that gave up in any drain warp ends all of them
// at the same point (none is left at a barrier the others no longer reach).
__device__ __forceinline__ bool epi_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 2, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "r"(kDbEpi)
        : "memory");
    return r != 0;
}

template <bool SUB>
__global__ void __launch_bounds__(kDbThreads, 1)
k_ozaki_gemm_db(const uint8_t* __restrict__ aimg, const int32_t* __restrict__ xexp, int K,
                const uint8_t* __restrict__ yblocks, const int32_t* __restrict__ yexp, int N, const double* B,
                int64_t ldb, double* C, int64_t ldc, int64_t m, int32_t* info, long spin, int tri, int img_nkw,
                const int32_t* __restrict__ bexp, int64_t ld_bexp) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t load_bar[2], empty_bar[2], acc_full[2], acc_empty[2], done_bar;
    __shared__ uint32_t tslot;
    __shared__ int abort_s;
    if (load_status(info) != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* stA[2] = {sm, sm + kDbStage};
    uint8_t* stB[2] = {sm + kAStage, sm + kDbStage + kAStage};
    double* W = reinterpret_cast<double*>(sm + 2 * kDbStage);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tslot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&load_bar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty_bar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&acc_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&acc_empty[i])), "r"(kDbEpiWarps));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        abort_s = 0;
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tslot;

    const int nkw = (K + kKW - 1) / kKW;
    const int ntn = (N + kDbN - 1) / kDbN;
    const int64_t ntm = (m + kTileM - 1) / kTileM;
    const int64_t ntiles = ntm * ntn;
    const bool tr = tri != 0;
    // exactness windows of 4 stages (K = 128), against one row bound xexp, or (bexp) each against its own
    // row bound bexp[w * ld_bexp + row] (the image's column groups: window w = columns 128 w .. 128 w + 127)
    const int wlen = 4;

    if (warp == kDbEpiWarps) {
        // stage copies, running ahead of the MMAs by the two stage buffers
        if (lane == 0) {
            int64_t g = 0, issued[2] = {0, 0};
            bool ok = true;
            // L2 prefetch cursor, kPrefetchAhead stages ahead of the copies (the same walk over tiles/stages)
            int64_t pt = blockIdx.x;
            int pkw = 0, pnk = pt < ntiles ? db_tile_stages(tile_col(pt, ntn, tr), nkw, tr) : 0;
            auto prefetch_next = [&]() {
                if (pt >= ntiles) return;
                bulk_prefetch_l2(aimg + static_cast<size_t>((pt / ntn) * img_nkw + pkw) * kAStage, kAStage);
                if (++pkw == pnk) {
                    pkw = 0;
                    pt += gridDim.x;
                    if (pt < ntiles) pnk = db_tile_stages(tile_col(pt, ntn, tr), nkw, tr);
                }
            };
            for (int i = 0; i < kPrefetchAhead; ++i) prefetch_next();
            // B rows of a tile are read at its end, after all its stages: bring them into L2 when its first
            // stage is issued (whole 16-byte granules of each row inside the row; only for 16-byte aligned rows)
            const bool b_pf = SUB && (reinterpret_cast<uintptr_t>(B) & 15) == 0 && (ldb & 1) == 0;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int64_t tm = t / ntn;
                const int tn = tile_col(t, ntn, tr);
                const int nk = db_tile_stages(tn, nkw, tr);
                if (b_pf) {
                    const int nb = ((N - tn * kDbN < kDbN ? N - tn * kDbN : kDbN) * 8) & ~15;
                    const int64_t rend = (tm + 1) * kTileM < m ? (tm + 1) * kTileM : m;
                    if (nb > 0)
                        for (int64_t r = tm * kTileM; r < rend; ++r)
                            bulk_prefetch_l2(B + r * ldb + tn * kDbN, static_cast<uint32_t>(nb));
                }
                for (int kw = 0; kw < nk; ++kw, ++g) {
                    const int s = static_cast<int>(g & 1);
                    if (g >= 2 && !mbar_wait_ab(&empty_bar[s], static_cast<uint32_t>(((g >> 1) - 1) & 1), &abort_s, spin)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&load_bar[s], kDbStage);
                    bulk_g2s(stA[s], aimg + static_cast<size_t>(tm * img_nkw + kw) * kAStage, kAStage, &load_bar[s]);
                    // slices of Y's 64-column block tn / 2, rows 32 (tn & 1).. of each: the 32-column tile
                    const uint8_t* bsrc = yblocks + static_cast<size_t>(((tn >> 1) * nkw + kw) * kSlices) * kBSlice +
                                          (tn & 1) * kDbBSlice;
#pragma unroll
                    for (int b = 0; b < kSlices; ++b)
                        bulk_g2s(stB[s] + b * kDbBSlice, bsrc + static_cast<size_t>(b) * kBSlice, kDbBSlice, &load_bar[s]);
                    ++issued[s];
                    prefetch_next();
                }
            }
            if (!bulk_drain(load_bar, issued)) ok = false;
            if (!ok) abort_s = 1;
        }
        __syncwarp();
    } else if (warp == kDbEpiWarps + 1) {
        // MMAs: window by window into alternating accumulator sets
        if (lane == 0) {
            int64_t g = 0, wc = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int nk = db_tile_stages(tile_col(t, ntn, tr), nkw, tr);
                for (int kw = 0; kw < nk; ++kw, ++g) {
                    const bool first = kw % wlen == 0;
                    const int set = static_cast<int>(wc & 1);
                    if (first && wc >= 2 &&
                        !mbar_wait_ab(&acc_empty[set], static_cast<uint32_t>(((wc >> 1) - 1) & 1), &abort_s, spin)) {
                        ok = false;
                        break;
                    }
                    const int s = static_cast<int>(g & 1);
                    if (!mbar_wait_ab(&load_bar[s], static_cast<uint32_t>((g >> 1) & 1), &abort_s, spin)) {
                        ok = false;
                        break;
                    }
                    tc_after_sync();
                    issue_stage_n32(tmem + static_cast<uint32_t>(set) * (kGroups * kDbN), smem_u32(stA[s]),
                                    smem_u32(stB[s]), first);
                    mma_commit(&empty_bar[s]);
                    if (kw % wlen == wlen - 1 || kw == nk - 1) {
                        mma_commit(&acc_full[set]);
                        ++wc;
                    }
                }
            }
            // every MMA issued here is complete before the tensor memory is released
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0u)) ok = false;
            if (!ok) abort_s = 1;
        }
        __syncwarp();
    } else {
        // drain: thread (row lr, column half h); the tile's result is staged in W and written in whole rows
        const int lr = tid & (kTileM - 1), h = tid >> 7;
        const uint32_t lane_off = static_cast<uint32_t>((warp & 3) * 32) << 16;
        int64_t wc = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int64_t tm = t / ntn;
            const int tn = tile_col(t, ntn, tr);
            const int nk = db_tile_stages(tn, nkw, tr);
            const int64_t row = tm * kTileM + lr;
            const int nwin = (nk + wlen - 1) / wlen;
            int E = kNoExp;
            if (row < m) {
                if (bexp) {
                    for (int w = 0; w < nwin; ++w) E = bexp[w * ld_bexp + row] > E ? bexp[w * ld_bexp + row] : E;
                } else {
                    E = xexp[row];
                }
            }
            long long acc[kDbCols];
#pragma unroll
            for (int j = 0; j < kDbCols; ++j) acc[j] = 0;
            for (int w = 0; w < nwin; ++w, ++wc) {
                const int set = static_cast<int>(wc & 1);
                const bool got = mbar_wait_ab(&acc_full[set], static_cast<uint32_t>((wc >> 1) & 1), &abort_s, spin);
                if (epi_sync_or(!got)) {
                    ok = false;
                    break;
                }
                tc_after_sync();
                int sh = 0;
                if (bexp && row < m) {
                    const int ew = bexp[w * ld_bexp + row];
                    sh = ew > kNoExp ? E - ew : 63;
                }
                drain_set32<kDbCols>(tmem + lane_off + static_cast<uint32_t>(set) * (kGroups * kDbN), kDbCols * h, sh,
                                     acc);
                tc_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[set]);
            }
            if (!ok) break;   // (uniform over the drain warps)
            const int col0 = tn * kDbN;
            const int ncols = N - col0 < kDbN ? N - col0 : kDbN;
            // this thread's B values of the store loop below, all in flight while the tile is scaled
            constexpr int kStoreIt = kTileM * kDbN / kDbEpi;
            double bv[SUB ? kStoreIt : 1];
            if constexpr (SUB) {
#pragma unroll
                for (int i = 0; i < kStoreIt; ++i) {
                    const int e = tid + i * kDbEpi;
                    const int r = e >> 5, c = e & 31;
                    const int64_t grow = tm * kTileM + r;
                    bv[i] = (grow < m && c < ncols) ? B[grow * ldb + col0 + c] : 0.0;
                }
            }
#pragma unroll
            for (int j = 0; j < kDbCols; ++j) {
                const int col = col0 + kDbCols * h + j;
                const int ey = col < N ? yexp[col] : kNoExp;
                W[lr * kDbEpiLd + kDbCols * h + j] =
                    (E > kNoExp && ey > kNoExp) ? scale_pow2(acc[j], E + ey - 53) : 0.0;
            }
            epi_sync();
#pragma unroll
            for (int i = 0; i < kStoreIt; ++i) {
                const int e = tid + i * kDbEpi;
                const int r = e >> 5, c = e & 31;
                const int64_t grow = tm * kTileM + r;
                if (grow < m && c < ncols) {
                    if constexpr (SUB) C[grow * ldc + col0 + c] = bv[i] - W[r * kDbEpiLd + c];
                    else C[grow * ldc + col0 + c] = W[r * kDbEpiLd + c];
                }
            }
            epi_sync();
        }
        if (!ok) abort_s = 1;
    }

    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0 && abort_s) set_status(info, RPCHOLQR_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// ---- C = B - X Y for K <= 32 (the right-looking updates of the split first pass) -------------------------
// Tiles of 128 rows x 32 output columns, so that one tile's eight group accumulators take 256 TMEM
// columns and two tiles are in flight: the tensor core fills one buffer while the other is drained.
// The X slices of a 128-row block (one K stage) are produced once and used by all N/32 column tiles of
// the block; the Y slices (at most 128 columns) stay in shared memory for the whole launch.  The X rows
// of the producers' next block arrive by cp.async in a raw buffer (whole rows across consecutive lanes)
// while the current block is sliced, so the slicing reads shared memory.  Warp roles:
// warps 0-3 produce (thread = row of the block), warps 4-19 drain (warp w reads TMEM lanes 32 (w % 4)..,
// columns 8 ((w - 4) / 4)..: four warps per lane quarter keep enough independent FP64 conversions and
// subtractions in flight), warp 20 issues the MMAs.  Barriers: stage_full/stage_empty per X stage
// buffer, acc_full/acc_empty per TMEM buffer.  Same exactness window, combination and rounding as
// k_ozaki_gemm_ws<false, true>: the results are identical.
constexpr int kUpdTileN = 32;
constexpr int kUpdMaxN = 128;
constexpr int kUpdProducers = 4, kUpdDrainers = 16;
constexpr int kUpdThreads = 32 * (kUpdProducers + kUpdDrainers + 1);
constexpr int kUpdRawLd = kKW + 1;                                       // raw X row stride (doubles)
constexpr int kUpdRawOff = 2 * kAStage + (kUpdMaxN / kTileN) * kBStage;  // after the stages and Y slices
constexpr int kUpdSmem = kUpdRawOff + kTileM * kUpdRawLd * 8;            // 225 KB
static_assert(kUpdSmem + 1024 <= 232448, "k_ozaki_update exceeds the 227 KB shared-memory limit");
constexpr int kUpdBSlice = kUpdTileN * kKW * 2;                          // 2 KB: one slice of a 32-column tile
constexpr int kUpdBTile = kSlices * kUpdBSlice;                          // 16 KB: its eight slices
// The 36 slice pairs of one 32-column tile for nkk K steps of 16 (group d into columns (d - 2) * 32 of
// the tile's TMEM buffer), 8 MMAs per step: the tile's eight B slices lie back to back (2 KB apart, one
// 256-row operand), so slice a of X meets slices b = 1 .. 9 - a in one MMA with N = 32 (9 - a) whose
// accumulators d = a + 1 .. 9 are adjacent.  The first MMA (a = 1, all eight groups) clears them.
__device__ __forceinline__ void issue_tile_n32(uint32_t tmem, uint32_t a_base, uint32_t b_base, int nkk) {
    const uint64_t a0 = sdesc(a_base), b0 = sdesc(b_base);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        if (kk >= nkk) break;
#pragma unroll
        for (int a = 1; a <= 8; ++a) {
            const uint64_t ad = a0 + static_cast<uint32_t>(((a - 1) * kASlice + kk * 256) >> 4);
            mma_bf16_n(tmem + (a - 1) * kUpdTileN, ad, b0 + static_cast<uint32_t>(kk * 16),
                       idesc_bf16(kUpdTileN * (9 - a)), (kk == 0 && a == 1) ? 0u : 1u);
        }
    }
}

__global__ void __launch_bounds__(kUpdThreads, 1)
k_ozaki_update(const double* X, int64_t ldx, const int32_t* __restrict__ xexp, int K,
               const uint8_t* __restrict__ yblocks, const int32_t* __restrict__ yexp, int N, const double* B,
               int64_t ldb, double* C, int64_t ldc, int64_t m, int32_t* info, long spin) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t stage_full[2], stage_empty[2], acc_full[2], acc_empty[2], done_bar;
    __shared__ uint32_t tslot;
    __shared__ int abort_s;
    if (load_status(info) != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* stA[2] = {sm, sm + kAStage};
    uint8_t* yres = sm + 2 * kAStage;                 // Y slices: 32-column tile j at j * kUpdBTile
    double* raw = reinterpret_cast<double*>(sm + kUpdRawOff);   // X rows of the producers' next block
    const int nsub = (N + kUpdTileN - 1) / kUpdTileN;
    const int nkk = (K + 15) / 16;
    const int64_t ntm = (m + kTileM - 1) / kTileM;
    const int64_t my_tiles =
        static_cast<int64_t>(blockIdx.x) < ntm ? (ntm - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tslot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&stage_full[i])),
                         "r"(kUpdProducers));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&stage_empty[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&acc_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&acc_empty[i])),
                         "r"(kUpdDrainers));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        abort_s = 0;
    }
    // the Y slices of every column block (K <= 32: one K stage each), resident for the launch, regrouped
    // per 32-column tile u: its slice b (rows 32 (u & 1).. of slice b of 64-column block u / 2, 2 KB) at
    // u * kUpdBTile + b * 2 KB
    {
        const int bytes = ((N + kTileN - 1) / kTileN) * kBStage;
        for (int e = tid; e < bytes / 16; e += kUpdThreads) {
            const int u = e / (kUpdBTile / 16), r = e - u * (kUpdBTile / 16);
            const int b = r / (kUpdBSlice / 16), o = r - b * (kUpdBSlice / 16);
            const unsigned dst = smem_u32(yres + 16 * e);
            const uint8_t* src = yblocks + static_cast<size_t>(u >> 1) * kBStage + b * kBSlice + (u & 1) * kUpdBSlice + 16 * o;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
        }
        cp_async_commit();
        cp_async_wait_all();
        fence_async_smem();
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tslot;

    if (warp < kUpdProducers) {
        // producers: the 128 threads copy a block's X rows into raw (whole rows, one value per lane) one
        // block ahead; thread lr slices row lr of the current block from raw into its stage
        const int lr = tid;
        auto copy_raw = [&](int64_t tt) {
            const int64_t rbase = (blockIdx.x + tt * gridDim.x) * kTileM;
            for (int e = tid; e < kTileM * K; e += 32 * kUpdProducers) {
                const int r = e / K, c = e - r * K;
                const bool in = rbase + r < m;
                cp_async8(raw + r * kUpdRawLd + c, in ? X + (rbase + r) * ldx + c : X, in);
            }
            cp_async_commit();
        };
        if (my_tiles > 0) copy_raw(0);
        uint32_t ph[2] = {0u, 0u};
        for (int64_t t = 0; t < my_tiles; ++t) {
            const int s = static_cast<int>(t & 1);
            bool ok = true;
            if (t >= 2) {
                ok = mbar_wait_ab(&stage_empty[s], ph[s], &abort_s, spin);
                ph[s] ^= 1u;
            }
            cp_async_wait_all();
            if (prod_sync_or(!ok, 32 * kUpdProducers)) {   // raw rows landed; a wait that gave up ends all
                abort_s = 1;
                break;
            }
            const int64_t row = (blockIdx.x + t * gridDim.x) * kTileM + lr;
            const int E = row < m ? xexp[row] : kNoExp;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c >= 2 * nkk) break;          // chunks the MMAs read; values k >= K are zero
                double x[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k = 8 * c + i;
                    x[i] = k < K ? raw[lr * kUpdRawLd + k] : 0.0;
                }
                slice_store8(x, E, stA[s] + core_off(lr, 16 * c), kASlice);
            }
            fence_async_smem();
            prod_sync(32 * kUpdProducers);        // every row sliced, raw free
            if (lane == 0) mbar_arrive(&stage_full[s]);
            if (t + 1 < my_tiles) copy_raw(t + 1);
        }
        cp_async_wait_all();
    } else if (warp < kUpdProducers + kUpdDrainers) {
        // drainers: warp w reads TMEM lanes 32 (w % 4).. and columns 8 h.. of every tile
        const int q = warp & 3, h = (warp - kUpdProducers) >> 2;
        const int lr = 32 * q + lane;
        // B and C rows 16-byte aligned (column tiles start at multiples of 8 values): pairs as one access
        const bool vec = ((reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15) == 0 &&
                         ((ldb | ldc) & 1) == 0;
        int64_t u = 0;   // tiles drained so far (TMEM buffer u & 1)
        for (int64_t t = 0; t < my_tiles && !*reinterpret_cast<volatile int*>(&abort_s); ++t) {
            const int64_t row = (blockIdx.x + t * gridDim.x) * kTileM + lr;
            const int E = row < m ? xexp[row] : kNoExp;
            for (int j = 0; j < nsub; ++j, ++u) {
                const int b = static_cast<int>(u & 1);
                const int cbase = j * kUpdTileN + 8 * h;
                // this thread's 8 values of B, read while the tile's MMAs run (16-byte pairs where aligned)
                double bv[8];
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const int col = cbase + i;
                    if (vec && row < m && col + 1 < N) {
                        const double2 v2 = *reinterpret_cast<const double2*>(B + row * ldb + col);
                        bv[i] = v2.x;
                        bv[i + 1] = v2.y;
                    } else {
                        bv[i] = (row < m && col < N) ? B[row * ldb + col] : 0.0;
                        bv[i + 1] = (row < m && col + 1 < N) ? B[row * ldb + col + 1] : 0.0;
                    }
                }
                if (!mbar_wait_ab(&acc_full[b], static_cast<uint32_t>((u >> 1) & 1), &abort_s, spin)) {
                    abort_s = 1;
                    break;
                }
                tc_after_sync();
                const uint32_t tb = tmem + (static_cast<uint32_t>(32 * q) << 16) + 256u * b + 8u * h;
#pragma unroll
                for (int c0 = 0; c0 < 8; c0 += 4) {
                    float mg[kGroups][4];
#pragma unroll
                    for (int g = 0; g < kGroups; ++g) tmem_ld4(tb + g * kUpdTileN + c0, mg[g]);
                    tmem_wait_ld();
                    if (row < m) {
                        double cv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int col = cbase + c0 + i;
                            float grp[kGroups];
#pragma unroll
                            for (int g = 0; g < kGroups; ++g) grp[g] = mg[g][i];
                            const long long I = combine_units53_k32(grp);
                            const int ey = col < N ? yexp[col] : kNoExp;
                            const double v = (E > kNoExp && ey > kNoExp) ? scale_pow2(I, E + ey - 53) : 0.0;
                            cv[i] = bv[c0 + i] - v;
                        }
#pragma unroll
                        for (int i = 0; i < 4; i += 2) {
                            const int col = cbase + c0 + i;
                            if (vec && col + 1 < N) {
                                *reinterpret_cast<double2*>(C + row * ldc + col) = make_double2(cv[i], cv[i + 1]);
                            } else {
                                if (col < N) C[row * ldc + col] = cv[i];
                                if (col + 1 < N) C[row * ldc + col + 1] = cv[i + 1];
                            }
                        }
                    }
                }
                tc_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[b]);
            }
        }
    } else {
        // MMA warp: one lane issues the column tiles of every block into alternating TMEM buffers
        if (lane == 0) {
            uint32_t phs[2] = {0u, 0u};
            int64_t u = 0;
            for (int64_t t = 0; t < my_tiles; ++t) {
                const int s = static_cast<int>(t & 1);
                if (!mbar_wait_ab(&stage_full[s], phs[s], &abort_s, spin)) { abort_s = 1; break; }
                phs[s] ^= 1u;
                tc_after_sync();
                bool ok = true;
                for (int j = 0; j < nsub; ++j, ++u) {
                    const int b = static_cast<int>(u & 1);
                    if (u >= 2 && !mbar_wait_ab(&acc_empty[b], static_cast<uint32_t>(((u >> 1) + 1) & 1), &abort_s, spin)) {
                        ok = false;
                        break;
                    }
                    tc_after_sync();
                    const uint32_t bbase = smem_u32(yres) + j * kUpdBTile;
                    issue_tile_n32(tmem + 256u * b, smem_u32(stA[s]), bbase, nkk);
                    mma_commit(&acc_full[b]);
                }
                if (!ok) { abort_s = 1; break; }
                mma_commit(&stage_empty[s]);
            }
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0u)) abort_s = 1;
        }
        __syncwarp();
    }

    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0 && abort_s) set_status(info, RPCHOLQR_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// ---- Gram partials from column stage images, with the accumulators double-buffered ------------------------
// Output tiles (P, Qb) of rows p in [128P, 128P+128) (TMEM lanes) x columns q in [32Qb, 32Qb+32), all
// tiles with Qb >= 4P (every q >= p is covered); grid = ntiles x nranges, CTA (tile, rr) sums the rows
// [rr*rows_per, ...) of the launch.  A = P's 128-column stage image (64 KB), B = rows 32 (Qb % 4).. of
// each slice of block Qb / 4's image (eight 2 KB copies); windows of 128 rows alternate between the two
// TMEM sets as in k_ozaki_gemm_db, each drained into int64 in units of 2^-49 and, every 64 windows and
// at the end, added into the CTA's FP64 partial (accum: the launch adds into partials of earlier row
// chunks).  The same slices, sums and flush points as k_ozaki_gram's 64-column tiles: the same bits.
__device__ __forceinline__ void gram_tile_coords32(int nqb, int tt, int& P, int& Qb) {
    P = 0;
    while (tt >= nqb - 4 * P) { tt -= nqb - 4 * P; ++P; }
    Qb = 4 * P + tt;
}

__global__ void __launch_bounds__(kDbThreads, 1)
k_ozaki_gram_db(int64_t m, int n, int np, const int32_t* __restrict__ colexp, int64_t rows_per, int ntiles,
                double* __restrict__ gpart, int32_t* info, long spin, const uint8_t* __restrict__ gimg, int accum) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t load_bar[2], empty_bar[2], acc_full[2], acc_empty[2], done_bar;
    __shared__ uint32_t tslot;
    __shared__ int abort_s;
    if (load_status(info) != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* stA[2] = {sm, sm + kDbStage};
    uint8_t* stB[2] = {sm + kAStage, sm + kDbStage + kAStage};
    const int nqb = (np + kDbN - 1) / kDbN;
    int P, Qb;
    gram_tile_coords32(nqb, blockIdx.x % ntiles, P, Qb);
    const int64_t rr = blockIdx.x / ntiles;
    const int64_t r0 = rr * rows_per;
    const int64_t r1 = (r0 + rows_per < m) ? r0 + rows_per : m;
    const int64_t nstages = r1 > r0 ? (r1 - r0 + kKW - 1) / kKW : 0;
    const int64_t nsg = (m + kKW - 1) / kKW;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tslot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&load_bar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty_bar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&acc_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&acc_empty[i])), "r"(kDbEpiWarps));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        abort_s = 0;
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tslot;

    if (warp == kDbEpiWarps) {
        if (lane == 0) {
            int64_t issued[2] = {0, 0};
            bool ok = true;
            const uint8_t* abase = gimg + static_cast<size_t>(P) * nsg * kAStage;
            const uint8_t* bbase = gimg + static_cast<size_t>(Qb >> 2) * nsg * kAStage + (Qb & 3) * kDbBSlice;
            // L2 prefetch of the stage kPrefetchAhead ahead (A stage and B's eight slices)
            auto prefetch = [&](int64_t pst) {
                if (pst >= nstages) return;
                const size_t sg = static_cast<size_t>(r0 / kKW + pst);
                bulk_prefetch_l2(abase + sg * kAStage, kAStage);
                if ((Qb >> 2) != P)
#pragma unroll
                    for (int b = 0; b < kSlices; ++b)
                        bulk_prefetch_l2(bbase + sg * kAStage + static_cast<size_t>(b) * kASlice, kDbBSlice);
            };
            for (int i = 0; i < kPrefetchAhead; ++i) prefetch(i);
            for (int64_t st = 0; st < nstages; ++st) {
                const int s = static_cast<int>(st & 1);
                if (st >= 2 && !mbar_wait_ab(&empty_bar[s], static_cast<uint32_t>(((st >> 1) - 1) & 1), &abort_s, spin)) {
                    ok = false;
                    break;
                }
                const size_t sg = static_cast<size_t>(r0 / kKW + st);
                mbar_expect_tx(&load_bar[s], kDbStage);
                bulk_g2s(stA[s], abase + sg * kAStage, kAStage, &load_bar[s]);
#pragma unroll
                for (int b = 0; b < kSlices; ++b)
                    bulk_g2s(stB[s] + b * kDbBSlice, bbase + sg * kAStage + static_cast<size_t>(b) * kASlice, kDbBSlice,
                             &load_bar[s]);
                ++issued[s];
                prefetch(st + kPrefetchAhead);
            }
            if (!bulk_drain(load_bar, issued)) ok = false;
            if (!ok) abort_s = 1;
        }
        __syncwarp();
    } else if (warp == kDbEpiWarps + 1) {
        if (lane == 0) {
            int64_t wc = 0;
            bool ok = true;
            for (int64_t st = 0; st < nstages; ++st) {
                const bool first = (st & 3) == 0;
                const int set = static_cast<int>(wc & 1);
                if (first && wc >= 2 &&
                    !mbar_wait_ab(&acc_empty[set], static_cast<uint32_t>(((wc >> 1) - 1) & 1), &abort_s, spin)) {
                    ok = false;
                    break;
                }
                const int s = static_cast<int>(st & 1);
                if (!mbar_wait_ab(&load_bar[s], static_cast<uint32_t>((st >> 1) & 1), &abort_s, spin)) {
                    ok = false;
                    break;
                }
                tc_after_sync();
                issue_stage_n32(tmem + static_cast<uint32_t>(set) * (kGroups * kDbN), smem_u32(stA[s]), smem_u32(stB[s]),
                                first);
                mma_commit(&empty_bar[s]);
                if ((st & 3) == 3 || st == nstages - 1) {
                    mma_commit(&acc_full[set]);
                    ++wc;
                }
            }
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0u)) ok = false;
            if (!ok) abort_s = 1;
        }
        __syncwarp();
    } else {
        const int lr = tid & (kTileM - 1), h = tid >> 7;
        const uint32_t lane_off = static_cast<uint32_t>((warp & 3) * 32) << 16;
        const int p = 128 * P + lr;
        const int Ep = p < n ? colexp[p] : kNoExp;
        double* out = gpart + static_cast<size_t>(rr) * np * np + static_cast<size_t>(p) * np;
        long long acc[kDbCols];
#pragma unroll
        for (int j = 0; j < kDbCols; ++j) acc[j] = 0;
        bool flushed = accum != 0, ok = true;
        // acc into the FP64 partial (the first flush of a launch that does not accumulate initialises it)
        auto flush = [&]() {
            if (p < np) {
#pragma unroll
                for (int j = 0; j < kDbCols; ++j) {
                    const int q = kDbN * Qb + kDbCols * h + j;
                    if (q < np) {
                        const int Eq = q < n ? colexp[q] : kNoExp;
                        const double v = (Ep > kNoExp && Eq > kNoExp) ? scale_pow2(acc[j], Ep + Eq - 49) : 0.0;
                        out[q] = (flushed ? out[q] : 0.0) + v;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kDbCols; ++j) acc[j] = 0;
            flushed = true;
        };
        const int64_t nwin = (nstages + 3) / 4;
        for (int64_t w = 0; w < nwin; ++w) {
            const int set = static_cast<int>(w & 1);
            const bool got = mbar_wait_ab(&acc_full[set], static_cast<uint32_t>((w >> 1) & 1), &abort_s, spin);
            if (epi_sync_or(!got)) {
                ok = false;
                break;
            }
            tc_after_sync();
            drain_set32<kDbCols, true>(tmem + lane_off + static_cast<uint32_t>(set) * (kGroups * kDbN), kDbCols * h, 0,
                                       acc);
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[set]);
            if ((w & 63) == 63 || w == nwin - 1) flush();   // every 64 windows and at the end
        }
        if (!ok) {
            abort_s = 1;
        } else if (nstages == 0 && !accum && p < np) {
            for (int j = 0; j < kDbCols; ++j) {
                const int q = kDbN * Qb + kDbCols * h + j;
                if (q < np) out[q] = 0.0;
            }
        }
    }

    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0 && abort_s) set_status(info, RPCHOLQR_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// ---- Gram partials G_rr = X_rr^T X_rr -------------------------------------------------------------------
// X: m x n FP64 (ldx), column exponent bounds colexp[n] over all m rows.  Output tiles (P, Qb): rows
// p in [128P, 128P+128) (TMEM lanes) x columns q in [64Qb, 64Qb+64), all tiles with Qb >= 2P (every
// q >= p is covered).  Grid = ntiles x nranges CTAs; CTA (tile, rr) accumulates the rows
// [rr*rows_per, ...) and writes gpart[rr][p][q] (np x np) for its tile.  The B operand reuses the A
// slices when its 64 columns lie inside the P block, else it is sliced into its own stage.  Exactness
// windows of 128 rows are drained into int64 accumulators in units of 2^-49 of the scale 2^(Ep+Eq)
// (one output row per thread, 32 columns); every 64 windows (8192 rows, |sum| < 2^63 even for maximal
// slices) they are added into the CTA's own FP64 partial and cleared.
__device__ __forceinline__ void gram_tile_coords(int nqb, int tt, int& P, int& Qb) {
    P = 0;
    while (tt >= nqb - 2 * P) { tt -= nqb - 2 * P; ++P; }
    Qb = 2 * P + tt;
}

// Warp roles: kGramNT producer threads slice and drain; the last warp issues the MMAs (full[s]: stage s
// sliced, one arrival per producer warp; empty[s]: its MMAs done).  A window's drain waits for the
// MMAs of the stage before and arrives on full of the next stage only after reading TMEM.
constexpr int kGramNT = kThreads;
// PRE: the column slices of every (128-column block, 32-row stage) of this launch's rows were made
// beforehand by k_slice_col_images (gimg): A is one 64 KB copy per stage, B (when it is not part of A)
// the matching half of another block's image.  accum: add into the partials instead of starting them
// (the launch is one of several row chunks summed in order).
template <bool PRE>
__global__ void __launch_bounds__(kGramNT + 32, 1)
k_ozaki_gram(const double* __restrict__ X, int64_t ldx, int64_t m, int n, int np,
             const int32_t* __restrict__ colexp, int64_t rows_per, int ntiles, double* __restrict__ gpart,
             int32_t* info, long spin, const uint8_t* __restrict__ gimg, int accum) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t empty_bar[2], full_bar[2], load_bar[2], done_bar;
    __shared__ uint32_t tslot;
    __shared__ int abort_s;
    if (load_status(info) != 0) return;
    constexpr int NT = kGramNT;
    constexpr int kCols = Share<NT>::kDrainCols, NCH = Share<NT>::kChunks;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nqb = (np + kTileN - 1) / kTileN;
    int P, Qb;
    gram_tile_coords(nqb, blockIdx.x % ntiles, P, Qb);
    const int64_t rr = blockIdx.x / ntiles;
    const int64_t r0 = rr * rows_per;
    const int64_t r1 = (r0 + rows_per < m) ? r0 + rows_per : m;
    uint8_t* stA[2] = {sm, sm + kAStage};
    uint8_t* stB[2] = {sm + 2 * kAStage, sm + 2 * kAStage + kBStage};
    const bool b_inside = 64 * Qb >= 128 * P && 64 * Qb + 64 <= 128 * P + 128;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tslot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty_bar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&full_bar[i])), "r"(NT / 32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&load_bar[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        abort_s = 0;
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tslot;
    const int64_t nstages = r1 > r0 ? (r1 - r0 + kKW - 1) / kKW : 0;

    if (warp == NT / 32) {
        if (lane == 0) {
            uint32_t fphase[2] = {0u, 0u}, lphase[2] = {0u, 0u};
            const uint32_t boff = b_inside ? static_cast<uint32_t>(((64 * Qb - 128 * P) / 8) * kSBO) : 0u;
            for (int64_t st = 0; st < nstages; ++st) {
                const int s = static_cast<int>(st & 1);
                if (!mbar_wait_ab(&full_bar[s], fphase[s], &abort_s, spin) ||
                    (PRE && !mbar_wait_ab(&load_bar[s], lphase[s], &abort_s, spin))) {
                    abort_s = 1;
                    break;
                }
                fphase[s] ^= 1u;
                lphase[s] ^= 1u;
                tc_after_sync();
                if (!PRE && b_inside)
                    issue_stage_pairs(tmem, smem_u32(stA[s]), smem_u32(stA[s]) + boff, kASlice, (st & 3) == 0);
                else
                    issue_stage(tmem, smem_u32(stA[s]), smem_u32(stB[s]), (st & 3) == 0);
                mma_commit(&empty_bar[s]);
            }
            mma_commit(&done_bar);
            if (!mbar_wait(&done_bar, 0u)) abort_s = 1;
        }
        __syncwarp();
    } else {
        const int lr = tid & 127;               // TMEM lane: output row p = 128P + lr; producer column of A
        const int rq = tid >> 7;                // producer row chunk(s) NCH*rq..; drain columns kCols*rq..
        const int p = 128 * P + lr;
        const int Ep = p < n ? colexp[p] : kNoExp;
        long long acc[kCols];
#pragma unroll
        for (int j = 0; j < kCols; ++j) acc[j] = 0;
        uint32_t phase[2] = {0u, 0u};
        bool pending[2] = {false, false};
        bool timed_out = false;
        int64_t issued[2] = {0, 0};         // bulk copies issued into each stage buffer (PRE, thread 0)

        // Drain the window just finished (its MMAs complete) into acc; every 64 windows, and at the end,
        // add acc into the CTA's FP64 partial (the first flush initialises it) and clear it.
        bool flushed = accum != 0;
        auto drain_window = [&](bool flush) {
            tc_after_sync();
            drain_acc<false, kCols, 4>(tmem, warp, kCols * rq, acc);
            if (flush && p < np) {
                double* out = gpart + static_cast<size_t>(rr) * np * np + static_cast<size_t>(p) * np;
#pragma unroll
                for (int j = 0; j < kCols; ++j) {
                    const int q = 64 * Qb + kCols * rq + j;
                    if (q < np) {
                        const int Eq = q < n ? colexp[q] : kNoExp;
                        const double v = (Ep > kNoExp && Eq > kNoExp) ? scale_pow2(acc[j], Ep + Eq - 49) : 0.0;
                        out[q] = (flushed ? out[q] : 0.0) + v;
                    }
                    acc[j] = 0;
                }
            }
            if (flush) flushed = true;
        };

        // Stage st is sliced into buffer st & 1 while the MMAs of stage st - 1 run; a stage that opens a
        // window first drains the previous window (after being produced, before it is handed over).
        for (int64_t st = 0; st < nstages; ++st) {
            const int s = static_cast<int>(st & 1);
            if (pending[s]) {
                const bool ok = mbar_wait_ab(&empty_bar[s], phase[s], &abort_s, spin);
                if (prod_sync_or(!ok, NT)) { timed_out = true; break; }
                phase[s] ^= 1u;
                pending[s] = false;
            }
            const int64_t k0 = r0 + st * kKW;
            if constexpr (PRE) {
                // A: the P block's 64 KB stage image; B (columns 64 Qb .. 64 Qb + 63): half (Qb & 1) of every
                // slice of block Qb / 2's image (P's own when they lie inside the P block), eight 4 KB pieces
                // placed back to back for the stacked MMAs.  Bulk copies on the stage's load barrier.
                if (tid == 0) {
                    const int64_t sg = k0 / kKW, nsg = (m + kKW - 1) / kKW;
                    const uint8_t* asrc = gimg + static_cast<size_t>(P * nsg + sg) * kAStage;
                    const uint8_t* bsrc = gimg + static_cast<size_t>((Qb >> 1) * nsg + sg) * kAStage +
                                          (Qb & 1) * kBSlice;
                    mbar_expect_tx(&load_bar[s], kAStage + kBStage);
                    bulk_g2s(stA[s], asrc, kAStage, &load_bar[s]);
#pragma unroll
                    for (int a = 0; a < kSlices; ++a)
                        bulk_g2s(stB[s] + a * kBSlice, bsrc + static_cast<size_t>(a) * kASlice, kBSlice, &load_bar[s]);
                    ++issued[s];
                }
            }
            if constexpr (!PRE) {
#pragma unroll
            for (int cc = 0; cc < NCH; ++cc) {
                const int c = NCH * rq + cc;
                double x[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int64_t row = k0 + 8 * c + i;
                    x[i] = (row < r1 && p < n) ? X[row * ldx + p] : 0.0;
                }
                slice_store8(x, Ep, stA[s] + core_off(lr, 16 * c), kASlice);
            }
            }
            if (!PRE && !b_inside) {
                for (int e = tid; e < 4 * 64; e += NT) {
                    const int c = e >> 6, col = 64 * Qb + (e & 63);   // 64 columns x 4 chunks of 8 rows
                    const int Ec = col < n ? colexp[col] : kNoExp;
                    double x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int64_t row = k0 + 8 * c + i;
                        x[i] = (row < r1 && col < n) ? X[row * ldx + col] : 0.0;
                    }
                    slice_store8(x, Ec, stB[s] + core_off(e & 63, 16 * c), kBSlice);
                }
            }
            fence_async_smem();
            if (st > 0 && (st & 3) == 0) {
                const int sp = s ^ 1;
                if (pending[sp]) {
                    const bool ok = mbar_wait_ab(&empty_bar[sp], phase[sp], &abort_s, spin);
                    if (prod_sync_or(!ok, NT)) { timed_out = true; break; }
                    phase[sp] ^= 1u;
                    pending[sp] = false;
                }
                drain_window((st & 255) == 0);   // the window ending at stage st - 1; every 64 windows flush
            }
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[s]);
            pending[s] = true;
        }
        if (!timed_out && nstages > 0) {
            for (int q = 0; q < 2 && !timed_out; ++q)
                if (pending[q]) {
                    const bool ok = mbar_wait_ab(&empty_bar[q], phase[q], &abort_s, spin);
                    if (prod_sync_or(!ok, NT)) { timed_out = true; break; }
                    phase[q] ^= 1u;
                    pending[q] = false;
                }
            if (!timed_out) drain_window(true);
        }
        if (PRE && tid == 0 && !bulk_drain(load_bar, issued)) timed_out = true;
        if (timed_out) {
            abort_s = 1;
        } else if (nstages == 0 && p < np && !accum) {
            double* out = gpart + static_cast<size_t>(rr) * np * np + static_cast<size_t>(p) * np;
            for (int j = 0; j < kCols; ++j) {
                const int q = 64 * Qb + kCols * rq + j;
                if (q < np) out[q] = 0.0;
            }
        }
    }

    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0 && abort_s) set_status(info, RPCHOLQR_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// rowexp[i] = exponent bound of row i of X (m x K, ldx); kNoExp for an all-zero row.
__global__ void k_row_exp(const double* __restrict__ X, int64_t ldx, int64_t m, int K, int32_t* __restrict__ rowexp) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int E = kNoExp;
    for (int k = 0; k < K; ++k) {
        const int e = exp_bound(X[i * ldx + k]);
        E = e > E ? e : E;
    }
    rowexp[i] = E;
}

// colexp[c] = max over rows of the exponent bounds (atomicMax; colexp must start at kNoExp).
__global__ void k_col_exp(const double* __restrict__ X, int64_t ldx, int64_t m, int n, int32_t* colexp) {
    const int c = threadIdx.x;
    if (c >= n) return;
    int E = kNoExp;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const int e = exp_bound(X[i * ldx + c]);
        E = e > E ? e : E;
    }
    if (E > kNoExp) atomicMax(&colexp[c], E);
}

__global__ void k_fill_i32(int32_t* p, int n, int32_t v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace oz

// ---- host launchers ----------------------------------------------------------------------------------
size_t ozaki_yblocks_bytes(int K, int N) {
    const int nkw = (K + oz::kKW - 1) / oz::kKW, ntn = (N + oz::kTileN - 1) / oz::kTileN;
    return static_cast<size_t>(nkw) * ntn * oz::kSlices * oz::kBSlice;
}

void launch_ozaki_slice_cols(const double* Y, int64_t ldy, int K, int N, uint8_t* blocks, int32_t* yexp,
                             const int32_t* info, cudaStream_t st) {
    dim3 grid((N + oz::kTileN - 1) / oz::kTileN, (K + oz::kKW - 1) / oz::kKW);
    oz::k_ozaki_slice_cols<<<grid, 256, 0, st>>>(Y, ldy, K, N, blocks, yexp, info);
}

cudaError_t launch_ozaki_gemm(bool sub, const double* X, int64_t ldx, const int32_t* xexp, int K,
                              const uint8_t* yblocks, const int32_t* yexp, int N, const double* B,
                              int64_t ldb, double* C, int64_t ldc, int64_t m, int32_t* info, int grid,
                              cudaStream_t st, long spin, bool y_upper, const uint8_t* aimg, int img_nkw,
                              const int32_t* bexp, int64_t ld_bexp) {
    if (K > 64 * oz::kKW) return cudaErrorInvalidValue;   // int64 accumulators hold K <= 2048 (see drain_acc)
    const bool win = K > 4 * oz::kKW;
    const int nt = win ? oz::kThreadsWin : oz::kThreads;
    cudaError_t err;
    if (sub && K <= oz::kKW && N <= oz::kUpdMaxN) {
        const int64_t ntm = (m + oz::kTileM - 1) / oz::kTileM;
        const int g = static_cast<int>(grid < ntm ? grid : ntm);
        err = cudaFuncSetAttribute(oz::k_ozaki_update, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::kUpdSmem);
        if (err != cudaSuccess) return err;
        oz::k_ozaki_update<<<g, oz::kUpdThreads, oz::kUpdSmem, st>>>(X, ldx, xexp, K, yblocks, yexp, N, B, ldb, C,
                                                                    ldc, m, info, spin);
        return cudaGetLastError();
    }
    if (aimg) {
        // pre-sliced X: the double-buffered kernel over 128 x 32 tiles
        auto kdb = sub ? oz::k_ozaki_gemm_db<true> : oz::k_ozaki_gemm_db<false>;
        err = cudaFuncSetAttribute(kdb, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::kDbSmem);
        if (err != cudaSuccess) return err;
        const int64_t tiles = ((m + oz::kTileM - 1) / oz::kTileM) * ((N + oz::kDbN - 1) / oz::kDbN);
        const int g = static_cast<int>(grid < tiles ? grid : tiles);
        const int nkw = (K + oz::kKW - 1) / oz::kKW;
        if (img_nkw < nkw) return cudaErrorInvalidValue;
        kdb<<<g, oz::kDbThreads, oz::kDbSmem, st>>>(aimg, xexp, K, yblocks, yexp, N, B, ldb, C, ldc, m, info, spin,
                                                    y_upper ? 1 : 0, img_nkw, bexp, ld_bexp);
        return cudaGetLastError();
    }
    auto kern = win ? (sub ? oz::k_ozaki_gemm_ws<true, true> : oz::k_ozaki_gemm_ws<true, false>)
                    : (sub ? oz::k_ozaki_gemm_ws<false, true> : oz::k_ozaki_gemm_ws<false, false>);
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::kGemmSmem);
    if (err != cudaSuccess) return err;
    kern<<<grid, nt + 32, oz::kGemmSmem, st>>>(X, ldx, xexp, K, yblocks, yexp, N, B, ldb, C, ldc, m, info, spin,
                                                y_upper ? 1 : 0);
    return cudaGetLastError();
}

// Stage images of the row slices of X (m x K, ldx; row bounds xexp) for k_ozaki_gemm_ws with aimg:
// ceil(m / 128) x ceil(K / 32) images of 64 KB (ozaki_image_bytes).
size_t ozaki_image_bytes(int64_t m, int K) {
    return static_cast<size_t>((m + oz::kTileM - 1) / oz::kTileM) * ((K + oz::kKW - 1) / oz::kKW) * oz::kAStage;
}
void launch_slice_images(const double* X, int64_t ldx, int64_t m, int K, const int32_t* xexp, uint8_t* img,
                         const int32_t* info, cudaStream_t st) {
    dim3 grid(static_cast<unsigned>((m + oz::kTileM - 1) / oz::kTileM), (K + oz::kKW - 1) / oz::kKW);
    oz::k_slice_images<<<grid, 512, 0, st>>>(X, ldx, m, K, xexp, img, info);
}

int32_t ozaki_no_exp() { return kNoExp; }

void launch_row_exp(const double* X, int64_t ldx, int64_t m, int K, int32_t* rowexp, cudaStream_t st) {
    oz::k_row_exp<<<static_cast<unsigned>((m + 255) / 256), 256, 0, st>>>(X, ldx, m, K, rowexp);
}

void launch_col_exp(const double* X, int64_t ldx, int64_t m, int n, int32_t* colexp, cudaStream_t st) {
    oz::k_fill_i32<<<(n + 127) / 128, 128, 0, st>>>(colexp, n, kNoExp);
    const int64_t blocks = m < 1024 ? m : 1024;
    oz::k_col_exp<<<static_cast<unsigned>(blocks), (n + 31) / 32 * 32, 0, st>>>(X, ldx, m, n, colexp);
}

// Output tiles of the split Gram kernel for padded width np.
int ozaki_gram_halves(int np) {
    const int nqb = (np + oz::kTileN - 1) / oz::kTileN;
    int c = 0;
    for (int P = 0; 2 * P < nqb; ++P) c += nqb - 2 * P;
    return c;
}
// Output tiles of the split Gram: 128 x 64 (k_ozaki_gram), or 128 x 32 from stage images (k_ozaki_gram_db).
int ozaki_gram_tiles(int np, bool images) {
    if (!images) return ozaki_gram_halves(np);
    const int nqb = (np + oz::kDbN - 1) / oz::kDbN;
    int c = 0;
    for (int P = 0; 4 * P < nqb; ++P) c += nqb - 4 * P;
    return c;
}

void launch_fill_noexp(int32_t* p, int n, cudaStream_t st) {
    oz::k_fill_i32<<<(n + 127) / 128, 128, 0, st>>>(p, n, kNoExp);
}

// gimg (nullable): column stage images of these m rows from launch_slice_col_images; accum: add into gpart.
cudaError_t launch_ozaki_gram(const double* X, int64_t ldx, int64_t m, int n, int np, const int32_t* colexp,
                              int nranges, double* gpart, int32_t* info, cudaStream_t st, long spin,
                              const uint8_t* gimg, bool accum) {
    if (gimg) {
        cudaError_t err = cudaFuncSetAttribute(oz::k_ozaki_gram_db, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               oz::kDbSmem);
        if (err != cudaSuccess) return err;
        const int nt = ozaki_gram_tiles(np, true);
        int64_t rows_per = (m + nranges - 1) / nranges;
        rows_per = (rows_per + oz::kKW - 1) / oz::kKW * oz::kKW;
        oz::k_ozaki_gram_db<<<nt * nranges, oz::kDbThreads, oz::kDbSmem, st>>>(m, n, np, colexp, rows_per, nt, gpart,
                                                                              info, spin, gimg, accum ? 1 : 0);
        return cudaGetLastError();
    }
    const int smem = 2 * (oz::kAStage + oz::kBStage);
    auto kern = oz::k_ozaki_gram<false>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    const int nt = ozaki_gram_halves(np);
    int64_t rows_per = (m + nranges - 1) / nranges;
    rows_per = (rows_per + oz::kKW - 1) / oz::kKW * oz::kKW;
    kern<<<nt * nranges, oz::kGramNT + 32, smem, st>>>(X, ldx, m, n, np, colexp, rows_per, nt, gpart, info, spin,
                                                       gimg, accum ? 1 : 0);
    return cudaGetLastError();
}

void launch_slice_block_images(const double* X, int64_t ldx, int64_t m, int nc, uint8_t* img, int img_nkw, int kw0,
                               int32_t* bexp, const int32_t* info, cudaStream_t st) {
    if (cudaFuncSetAttribute(oz::k_slice_block_images, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::kSbSmem) !=
        cudaSuccess)
        return;   // the launch error surfaces at the caller's check
    // both halves of every 128-row tile (rows past m are written as zero slices, as the products read them)
    oz::k_slice_block_images<<<static_cast<unsigned>((m + oz::kTileM - 1) / oz::kTileM * 2), 256, oz::kSbSmem, st>>>(
        X, ldx, m, nc, img, img_nkw, kw0, bexp, info);
}
void launch_slice_col_images(const double* X, int64_t ldx, int64_t m, int n, int np, const int32_t* colexp,
                             uint8_t* img, const int32_t* info, cudaStream_t st) {
    dim3 grid(static_cast<unsigned>((m + oz::kKW - 1) / oz::kKW), (np + 127) / 128);
    oz::k_slice_col_images<<<grid, 512, 0, st>>>(X, ldx, m, n, colexp, img, info);
}

}  // namespace rpq
