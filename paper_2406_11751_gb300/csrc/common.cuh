// Device-side building blocks shared by the rpCholesky-QR kernels (sm_103a).
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rpcholqr.h"

namespace rpq {

// Every matrix dimension is padded to a multiple of this (the k extent of mma m16n8k16).
constexpr int kPad = 16;
constexpr int kMaxNP = 128;             // widest panel the row-pass kernels keep in shared memory

__host__ __device__ constexpr int pad16(int n) { return (n + kPad - 1) / kPad * kPad; }
// Padded width of the n x n factors: a multiple of 16 up to 128 columns, of 64 above (64-column blocks).
__host__ __device__ constexpr int pad_np(int n) { return n <= kMaxNP ? pad16(n) : (n + 63) / 64 * 64; }

// ---- launch shape of the FP64 row passes (rowpass.cu) ----------------------------------------------
// Warps per CTA: 8 when the 256-row panel fits shared memory (NP <= 64), else 4 (128-row panel).
__host__ __device__ constexpr int rowpass_warps(int np) { return np <= 64 ? 8 : 4; }
// Rows of one panel (32 per warp).
__host__ __device__ constexpr int rowpass_rows(int np) { return 32 * rowpass_warps(np); }
// The plain solve up to 48 columns runs two CTAs per SM (128 registers a thread, two panels fit the
// shared memory): one CTA's panel load overlaps the other's FP64 work and each scheduler has four
// warps' dependent chains to interleave.  The fused Gram keeps one CTA per SM: the caller sizes its
// per-CTA partials for the grid it passes, which the launcher then uses unchanged.
__host__ __device__ constexpr int rowpass_ctas_per_sm(int np, bool syrk) { return !syrk && np <= 48 ? 2 : 1; }
static_assert(rowpass_ctas_per_sm(16, true) == 1 && rowpass_ctas_per_sm(64, true) == 1 &&
                  rowpass_ctas_per_sm(128, true) == 1,
              "the fused Gram pass writes one partial per CTA of the grid its caller passes");

// ---- power-of-two bounds used by the split-precision products ------------------------------------
// exp_bound(v): |v| < 2^e for a normal v (e = unbiased exponent + 1); kNoExp for 0 or subnormal.
constexpr int kNoExp = INT_MIN / 2;
__device__ __forceinline__ int exp_bound(double v) {
    const int ex = static_cast<int>((__double_as_longlong(v) >> 52) & 0x7FF);
    return ex == 0 ? kNoExp : ex - 1022;
}

// ---- status word: info[0] = status, info[1] = pivot ---------------------------------------------
__device__ __forceinline__ int load_status(const int32_t* info) {
    return *reinterpret_cast<const volatile int32_t*>(info);
}
// First error wins.
__device__ __forceinline__ void set_status(int32_t* info, int status, int pivot = -1) {
    if (atomicCAS(info, 0, status) == 0 && pivot >= 0) info[1] = pivot;
}

// ---- FP64 tensor-core mma: D(16x8) += A(16x16) * B(16x8), all FP64 ------------------------------
// Fragment layouts (g = lane/4, t = lane%4):
//   A: a[i] = A[g + 8*(i&1)][t + 4*(i>>1)]      i = 0..7
//   B: b[i] = B[t + 4*i][g]                     i = 0..3
//   C: c[i] = C[g + 8*(i>>1)][2*t + (i&1)]      i = 0..3
__device__ __forceinline__ void mma_f64_16816(double (&d)[4], const double (&a)[8],
                                              const double (&b)[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
          "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// D(16x8) += A(16x8) * B(8x8), FP64: the same fragment layouts restricted to k < 8
// (a[i] = A[g + 8*(i&1)][t + 4*(i>>1)], i = 0..3;  b[i] = B[t + 4*i][g], i = 0..1).
__device__ __forceinline__ void mma_f64_1688(double (&d)[4], const double (&a)[4], const double (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}

// ---- cp.async (Ampere+ LDGSTS), 8-byte granules with zero fill ----------------------------------
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src, bool valid) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    int src_size = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem_src),
                 "r"(src_size));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace rpq
