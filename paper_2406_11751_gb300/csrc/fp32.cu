// FP32 mode: the two passes of Algorithm alg_2 in single precision, for single-precision Krylov /
// LOBPCG users (A, Q, R stored as float).  The sample, the Householder R_s and the Cholesky factor R1
// stay in FP64 (they are small, and their stability needs it: Section 4 keeps R_s^{-1} applied to the
// ill-conditioned A); the m-row work runs on the FP32 FMA pipe (~70 TFLOP/s on GB300, against ~1 for
// FP64):
//
//   k_prep_f32       T32 = float(T) padded with the identity, rinv32 = 1 / diag(T32);
//   k_rowsolve_f32   Y = X T^{-1} row by row (Section 2.1: each row of A_1 is a triangular solve with
//                    R_s), one row per thread, left-looking over 32-column blocks: the off-diagonal
//                    part of a block is a length-32J dot product per column against the block of T
//                    staged in shared memory (broadcast reads), the 32 x 32 diagonal block is forward
//                    substitution in registers;
//   k_syrk_f32       per-range partials of G = A_1^T A_1 over 64 x 64 upper tiles, FP32 products summed
//                    in FP32 over 256-row chunks, the chunks added into FP64 totals.
#include "common.cuh"

namespace rpq {

constexpr int kF32Blk = 32;      // column block of the row solves
constexpr int kF32Rows = 256;    // rows per CTA, one per thread
constexpr int kSyrkChunkRows = 256;

__host__ __device__ constexpr int pad32(int n) { return (n + 31) / 32 * 32; }

// T32 (np32 x np32 row-major): float(T) on and above the diagonal of the leading n x n block, 0 below,
// identity in the padding.  A diagonal that is not a normal FP32 number sets `fail_status`.
__global__ void k_prep_f32(const double* __restrict__ T, int64_t ldt, int n, int np32, float* __restrict__ T32,
                           float* __restrict__ rinv32, int fail_status, int32_t* info) {
    if (load_status(info) != 0) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np32 * np32) return;
    const int r = e / np32, c = e - r * np32;
    float v;
    if (r < n && c < n) v = r <= c ? static_cast<float>(T[static_cast<int64_t>(r) * ldt + c]) : 0.0f;
    else v = r == c ? 1.0f : 0.0f;
    T32[e] = v;
    if (r == c) {
        if (!(fabsf(v) >= 1.17549435e-38f) || !isfinite(v)) set_status(info, fail_status, r);
        rinv32[r] = 1.0f / v;
    }
}

// Y = X T^{-1} for upper-triangular T (T32, rinv32 from k_prep_f32).  Y may equal X (ldy == ldx).
__global__ void __launch_bounds__(kF32Rows)
k_rowsolve_f32(const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t m, int n,
               const float* __restrict__ T32, int np32, const float* __restrict__ rinv32, int32_t* info,
               bool check_finite, bool vec) {
    extern __shared__ float4 ts4[];   // rows 0 .. 32J+31 of the 32 columns of block J (8 float4 per row)
    if (load_status(info) != 0) return;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * kF32Rows + threadIdx.x;
    const bool live = r < m;
    const float* xr = X + (live ? r : 0) * ldx;
    float* yr = Y + (live ? r : 0) * ldy;
    bool bad = false;
    for (int c0 = 0; c0 < n; c0 += kF32Blk) {
        __syncthreads();   // the previous block's reads of ts4 are done
        for (int e = threadIdx.x; e < (c0 + kF32Blk) * 8; e += blockDim.x) {
            const int k = e >> 3, q = e & 7;
            ts4[e] = reinterpret_cast<const float4*>(T32 + static_cast<size_t>(k) * np32 + c0)[q];
        }
        __syncthreads();
        if (!live) continue;
        float acc[kF32Blk];
#pragma unroll
        for (int c = 0; c < kF32Blk; ++c) {
            acc[c] = c0 + c < n ? xr[c0 + c] : 0.0f;
            bad |= !isfinite(acc[c]);
        }
        // acc -= Y[r, 0:c0] T[0:c0, c0:c0+32]; with 16-byte aligned rows, 8 solved values per two
        // vector loads, two such groups in flight
        if (vec) {
#pragma unroll 2
            for (int k = 0; k < c0; k += 8) {
                const float4 ya = *reinterpret_cast<const float4*>(yr + k);
                const float4 yb = *reinterpret_cast<const float4*>(yr + k + 4);
                const float yv[8] = {-ya.x, -ya.y, -ya.z, -ya.w, -yb.x, -yb.y, -yb.z, -yb.w};
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const float4* tk = ts4 + (k + kk) * 8;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 t = tk[q];
                        acc[4 * q + 0] = fmaf(yv[kk], t.x, acc[4 * q + 0]);
                        acc[4 * q + 1] = fmaf(yv[kk], t.y, acc[4 * q + 1]);
                        acc[4 * q + 2] = fmaf(yv[kk], t.z, acc[4 * q + 2]);
                        acc[4 * q + 3] = fmaf(yv[kk], t.w, acc[4 * q + 3]);
                    }
                }
            }
        } else {
            for (int k = 0; k < c0; ++k) {
                const float yk = -yr[k];
                const float4* tk = ts4 + k * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 t = tk[q];
                    acc[4 * q + 0] = fmaf(yk, t.x, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(yk, t.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(yk, t.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(yk, t.w, acc[4 * q + 3]);
                }
            }
        }
        // diagonal block: forward substitution, row j of the block's T read as float4s
#pragma unroll
        for (int j = 0; j < kF32Blk; ++j) {
            acc[j] *= rinv32[c0 + j];
            const float xj = -acc[j];
            const float4* trow = ts4 + (c0 + j) * 8;
#pragma unroll
            for (int q = (j + 1) / 4; q < 8; ++q) {
                const float4 t = trow[q];
                if (4 * q + 0 > j) acc[4 * q + 0] = fmaf(xj, t.x, acc[4 * q + 0]);
                if (4 * q + 1 > j) acc[4 * q + 1] = fmaf(xj, t.y, acc[4 * q + 1]);
                if (4 * q + 2 > j) acc[4 * q + 2] = fmaf(xj, t.z, acc[4 * q + 2]);
                if (4 * q + 3 > j) acc[4 * q + 3] = fmaf(xj, t.w, acc[4 * q + 3]);
            }
        }
#pragma unroll
        for (int c = 0; c < kF32Blk; ++c)
            if (c0 + c < n) yr[c0 + c] = acc[c];
    }
    if (__syncthreads_or(check_finite && bad) && threadIdx.x == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
}

// Partials of G = X^T X: CTA (tile, range) accumulates the 64 x 64 tile (I, J), I <= J, over the rows
// [range*rows_per, ...) and writes gpart[range][p][q] (ld np64, FP64) for its tile.  Thread (ty, tx)
// owns the 4 x 4 outputs p = 64I + 4ty + i, q = 64J + 4tx + j.
__global__ void __launch_bounds__(256)
k_syrk_f32(const float* __restrict__ X, int64_t ldx, int64_t m, int n, int np64, int64_t rows_per,
           double* __restrict__ gpart, const int32_t* info) {
    __shared__ __align__(16) float xs[2][32][2 * 64 + 4];   // double-buffered 32-row chunks
    if (load_status(info) != 0) return;
    const int nb = np64 / 64;
    int tt = blockIdx.x, I = 0;
    while (tt >= nb - I) { tt -= nb - I; ++I; }
    const int J = I + tt;
    const int64_t rb = static_cast<int64_t>(blockIdx.y) * rows_per;
    const int64_t re = (rb + rows_per < m) ? rb + rows_per : m;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    float acc[4][4];
    double tot[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j] = 0.0f; tot[i][j] = 0.0; }
    // rows k0 .. k0+31 of the two 64-column blocks into xs[b] (4-byte cp.async, zero-filled outside X)
    auto stage = [&](int64_t k0, int b) {
        for (int e = tid; e < 32 * 128; e += 256) {
            const int rr = e >> 7, cc = e & 127;
            const int col = cc < 64 ? 64 * I + cc : 64 * J + (cc - 64);
            const bool ok = k0 + rr < re && col < n;
            const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(&xs[b][rr][cc]));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst),
                         "l"(ok ? X + (k0 + rr) * ldx + col : X), "r"(ok ? 4 : 0));
        }
    };
    if (rb < re) stage(rb, 0);
    asm volatile("cp.async.commit_group;\n");
    int64_t chunk_end = rb + kSyrkChunkRows;
    int b = 0;
    for (int64_t k0 = rb; k0 < re; k0 += 32, b ^= 1) {
        if (k0 + 32 < re) stage(k0 + 32, b ^ 1);   // xs[b ^ 1] was last read before the barrier below
        asm volatile("cp.async.commit_group;\n");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(&xs[b][kk][4 * ty]);
            const float4 bb = *reinterpret_cast<const float4*>(&xs[b][kk][64 + 4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (k0 + 32 >= chunk_end) {
            chunk_end += kSyrkChunkRows;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) { tot[i][j] += acc[i][j]; acc[i][j] = 0.0f; }
        }
        __syncthreads();   // every thread is done with xs[b] before it is refilled
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    double* out = gpart + static_cast<size_t>(blockIdx.y) * np64 * np64;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = 64 * I + 4 * ty + i, q = 64 * J + 4 * tx + j;
            out[static_cast<size_t>(p) * np64 + q] = tot[i][j] + acc[i][j];
        }
}

// dst (n x n float, ld ldd) = float(src) (n x n, ld lds)
__global__ void k_f64_to_f32(const double* __restrict__ src, int64_t lds, int n, float* __restrict__ dst,
                             int64_t ldd) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int r = e / n, c = e - r * n;
    dst[static_cast<int64_t>(r) * ldd + c] = static_cast<float>(src[static_cast<int64_t>(r) * lds + c]);
}

// ---- host launchers --------------------------------------------------------------------------------
int f32_pad(int n) { return pad32(n); }

void launch_prep_f32(const double* T, int64_t ldt, int n, float* T32, float* rinv32, int fail_status,
                     int32_t* info, cudaStream_t st) {
    const int np32 = pad32(n);
    k_prep_f32<<<(np32 * np32 + 255) / 256, 256, 0, st>>>(T, ldt, n, np32, T32, rinv32, fail_status, info);
}

cudaError_t launch_rowsolve_f32(const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t m, int n,
                                const float* T32, const float* rinv32, int32_t* info, bool check_finite,
                                cudaStream_t st) {
    const int np32 = pad32(n);
    const int smem = np32 * kF32Blk * static_cast<int>(sizeof(float));
    cudaError_t err = cudaFuncSetAttribute(k_rowsolve_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    const int64_t grid = (m + kF32Rows - 1) / kF32Rows;
    // vector loads of solved values need 16-byte aligned rows
    const bool vec = (reinterpret_cast<uintptr_t>(Y) % 16 == 0) && (ldy % 4 == 0);
    k_rowsolve_f32<<<static_cast<unsigned>(grid), kF32Rows, smem, st>>>(X, ldx, Y, ldy, m, n, T32, np32, rinv32,
                                                                         info, check_finite, vec);
    return cudaGetLastError();
}

// ranges x np64 x np64 doubles in gpart; returns the number of ranges used.
int launch_syrk_f32(const float* X, int64_t ldx, int64_t m, int n, int max_ranges, double* gpart,
                    const int32_t* info, cudaStream_t st) {
    const int np64 = (n + 63) / 64 * 64;
    const int nb = np64 / 64;
    const int tiles = nb * (nb + 1) / 2;
    int ranges = (3 * max_ranges) / tiles;   // about three CTAs per SM
    if (ranges > max_ranges) ranges = max_ranges;
    if (ranges < 1) ranges = 1;
    const int64_t most = (m + 31) / 32;
    if (ranges > most) ranges = static_cast<int>(most);
    int64_t rows_per = (m + ranges - 1) / ranges;
    rows_per = (rows_per + 31) / 32 * 32;
    k_syrk_f32<<<dim3(tiles, ranges), 256, 0, st>>>(X, ldx, m, n, np64, rows_per, gpart, info);
    return ranges;
}

void launch_f64_to_f32(const double* src, int64_t lds, int n, float* dst, int64_t ldd, cudaStream_t st) {
    k_f64_to_f32<<<(n * n + 255) / 256, 256, 0, st>>>(src, lds, n, dst, ldd);
}

}  // namespace rpq
