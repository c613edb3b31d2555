// FP64 building blocks for n > 128 (the row pass keeps at most a 128-column panel in shared memory):
//
//   k_gemm_sub_fp64:  C = B - X Y      X: m x K (ldx), Y: K x N (ldy, small), B, C: m x N
//                     the off-diagonal block update A[:, J] - A_1[:, <J] T[<J, J] of a left-looking
//                     blocked row solve (the diagonal blocks are solved by the row pass);
//   k_syrk_fp64:      per-range partials of G = X^T X over 64 x 64 upper tiles (the Gram step of
//                     Algorithm alg_2 for wide A_1), summed afterwards in a fixed order.
//
// Both run FP64 mma.sync m16n8k16 (the FP64 pipe is the bound: ~1.05 TFLOP/s on GB300) with eight
// independent accumulator tiles per warp.  Memory traffic is far below the HBM roofline, so operands are
// read with plain loads; the small right-hand factor is staged in shared memory 64 rows at a time.
#include "common.cuh"

namespace rpq {

constexpr int kGemmRows = 128;     // rows per CTA tile (8 warps x 16)
constexpr int kGemmCols = 64;      // columns per CTA tile (8 n8 tiles per warp)
constexpr int kGemmKChunk = 64;    // rows of Y staged per smem refill

// C = B - X Y on a persistent grid of 128 x 64 tiles.  Y chunk in shared memory as B fragments.
__global__ void __launch_bounds__(256, 1)
k_gemm_sub_fp64(const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y, int64_t ldy,
                const double* B, int64_t ldb, double* C, int64_t ldc, int64_t m, int K, int N,
                const int32_t* info) {
    __shared__ double ys[kGemmKChunk][kGemmCols + 1];
    if (info && load_status(info) != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ntn = (N + kGemmCols - 1) / kGemmCols;
    const int64_t ntm = (m + kGemmRows - 1) / kGemmRows;
    for (int64_t tile = blockIdx.x; tile < ntm * ntn; tile += gridDim.x) {
        const int64_t tm = tile / ntn;
        const int tn = static_cast<int>(tile - tm * ntn);
        const int64_t r0 = tm * kGemmRows + warp * 16;
        const int c0 = tn * kGemmCols;
        double acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0;
        for (int k0 = 0; k0 < K; k0 += kGemmKChunk) {
            __syncthreads();
            for (int e = threadIdx.x; e < kGemmKChunk * kGemmCols; e += blockDim.x) {
                const int kk = e / kGemmCols, cc = e - kk * kGemmCols;
                ys[kk][cc] = (k0 + kk < K && c0 + cc < N) ? Y[static_cast<int64_t>(k0 + kk) * ldy + c0 + cc] : 0.0;
            }
            __syncthreads();
            const int kmax = (K - k0) < kGemmKChunk ? (K - k0) : kGemmKChunk;
            for (int kc = 0; kc < kmax; kc += 16) {
                double a[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int64_t r = r0 + g + 8 * (i & 1);
                    const int k = k0 + kc + t + 4 * (i >> 1);
                    a[i] = (r < m && k < K) ? X[r * ldx + k] : 0.0;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    double b[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) b[i] = ys[kc + t + 4 * i][8 * j + g];
                    mma_f64_16816(acc[j], a, b);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t r = r0 + g + 8 * (i >> 1);
                const int c = c0 + 8 * j + 2 * t + (i & 1);
                if (r < m && c < N) C[r * ldc + c] = B[r * ldb + c] - acc[j][i];
            }
    }
}

// Partials of G = X^T X: block (tile, range) accumulates the 64 x 64 tile (I, J), I <= J, of the rows
// [range*rows_per, ...) and writes gpart[range][p][q] (ld np) for its tile.  Rows staged 32 at a time.
// Two-level sums: the mma accumulators take 8192 rows, then are added into a running total and
// cleared, so a range of R rows accumulates rounding over ~8192 + R/8192 terms instead of R.
__global__ void __launch_bounds__(256, 2)
k_syrk_fp64(const double* __restrict__ X, int64_t ldx, int64_t m, int n, int np, int64_t rows_per,
            double* __restrict__ gpart, const int32_t* info) {
    __shared__ double xs[32][2 * 64 + 1];   // 32 rows x (64 columns of I | 64 columns of J)
    if (info && load_status(info) != 0) return;
    const int nb = np / 64;
    // tile index -> (I, J) with I <= J
    int tt = blockIdx.x, I = 0;
    while (tt >= nb - I) { tt -= nb - I; ++I; }
    const int J = I + tt;
    const int64_t range = blockIdx.y;
    const int64_t rb = range * rows_per;
    const int64_t re = (rb + rows_per < m) ? rb + rows_per : m;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // warp w: output rows 16*(w&3) .. (within the 64 of I), output column tiles 4*(w>>2) .. +3 (n8 each)
    const int mi = warp & 3, nj0 = 4 * (warp >> 2);
    double acc[4][4], tot[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = tot[j][i] = 0.0;
    int chunk = 0;
    for (int64_t k0 = rb; k0 < re; k0 += 32) {
        if (++chunk == 256) {
            chunk = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    tot[j][i] += acc[j][i];
                    acc[j][i] = 0.0;
                }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 128; e += blockDim.x) {
            const int rr = e >> 7, cc = e & 127;
            const int col = cc < 64 ? 64 * I + cc : 64 * J + (cc - 64);
            xs[rr][cc] = (k0 + rr < re && col < n) ? X[(k0 + rr) * ldx + col] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kc = 0; kc < 32; kc += 16) {
            double a[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = xs[kc + t + 4 * (i >> 1)][16 * mi + g + 8 * (i & 1)];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                double b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) b[i] = xs[kc + t + 4 * i][64 + 8 * (nj0 + j) + g];
                mma_f64_16816(acc[j], a, b);
            }
        }
    }
    double* out = gpart + static_cast<size_t>(range) * np * np;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = 64 * I + 16 * mi + g + 8 * (i >> 1);
            const int q = 64 * J + 8 * (nj0 + j) + 2 * t + (i & 1);
            out[static_cast<size_t>(p) * np + q] = tot[j][i] + acc[j][i];
        }
}

cudaError_t launch_gemm_sub_fp64(const double* X, int64_t ldx, const double* Y, int64_t ldy, const double* B,
                                 int64_t ldb, double* C, int64_t ldc, int64_t m, int K, int N,
                                 const int32_t* info, int grid, cudaStream_t st) {
    const int64_t tiles = ((m + kGemmRows - 1) / kGemmRows) * ((N + kGemmCols - 1) / kGemmCols);
    const int g = static_cast<int>(tiles < grid ? tiles : grid);
    k_gemm_sub_fp64<<<g, 256, 0, st>>>(X, ldx, Y, ldy, B, ldb, C, ldc, m, K, N, info);
    return cudaGetLastError();
}

// ranges: row splits; gpart must hold ranges x np x np doubles (only upper 64 x 64 tiles written).
cudaError_t launch_syrk_fp64(const double* X, int64_t ldx, int64_t m, int n, int np, int ranges, double* gpart,
                             const int32_t* info, cudaStream_t st) {
    const int nb = np / 64;
    int64_t rows_per = (m + ranges - 1) / ranges;
    rows_per = (rows_per + 31) / 32 * 32;
    dim3 grid(nb * (nb + 1) / 2, ranges);
    k_syrk_fp64<<<grid, 256, 0, st>>>(X, ldx, m, n, np, rows_per, gpart, info);
    return cudaGetLastError();
}

}  // namespace rpq
