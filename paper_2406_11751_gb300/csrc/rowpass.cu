// Streaming passes of Algorithm alg_2 (Section 4) over the rows of a tall-skinny matrix:
//
//   pass 1 ('precondition' + 'Gram'):  A1 = A R_s^{-1}  and  G1 += A1_panel^T A1_panel
//   pass 2 ('solve'):                  Q  = A1 R_1^{-1}  (in place over A1)
//
// Both are m independent row solves x_i^T = T^{-T} b_i^T (the row-wise view of Section 2.1).
//
// GB300 design.  FP64 on this part runs at about 1.05 TFLOP/s whether it is issued as DFMA or as the
// FP64 tensor-core mma.sync m16n8k16 (measured); HBM is ~100x faster than this FP64 work needs, so the
// kernels are organised to keep the FP64 pipe busy, not for bandwidth.  mma.sync m16n8k16 carries 2048
// FMAs per instruction, so the issue slots stay free for address math and shared-memory traffic:
//   * a CTA (4 warps, or 8 when NP <= 64) owns a 32-rows-per-warp panel staged in shared memory with
//     cp.async; the row stride
//     NP+4 doubles keeps every fragment load at the minimum two wavefronts;
//   * the solve is blocked by 8 columns, left-looking: block J of a 16-row tile is
//       acc = X[:, J] - A1[:, <J] T[<J, J]          (mma m16n8k16, FP64, B = -T chunks)
//       A1[:, J] = acc T[J, J]^{-1}                 (8-column forward substitution, DFMA,
//                                                    one lane per row, reciprocal diagonal)
//     each warp runs two 16-row tiles with two split-k accumulators (4 chains per warp);
//   * the Gram matrix keeps only the upper 16x8 tiles (72 tiles at n = 128), 18 per warp,
//     accumulated in registers across every panel the CTA visits; each CTA writes one partial
//     and a second kernel sums the partials in a fixed order (deterministic, no atomics).
#include "common.cuh"

namespace rpq {

// Number of 16x8 tiles of an NP x NP matrix that touch the upper triangle.
__host__ __device__ constexpr int upper_tiles(int np) {
    int c = 0;
    for (int I = 0; I < np / 16; ++I) c += np / 8 - 2 * I;
    return c;
}

__device__ __forceinline__ void tile_coords(int np, int tt, int& I, int& J) {
    const int nb = np / 8;
    I = 0;
    while (tt >= nb - 2 * I) { tt -= nb - 2 * I; ++I; }
    J = 2 * I + tt;
}

// ---- triangular-factor tables for the row solve --------------------------------------------------
// T: n x n upper triangular (ld ldt), padded to np with the identity.
//   frag[((kc*NB + J)*32 + lane)*4 + i] = -T[16kc + t + 4i][8J + g]  if 16kc + t + 4i < 8J, else 0
//     (the B fragment of mma m16n8k16 for k-chunk kc and column block J),
//   diag[J*64 + r*8 + c] = T[8J+r][8J+c] for r < c, 1/T[8J+c][8J+c] for r == c, 0 for r > c.
__global__ void k_prep_tri(const double* __restrict__ T, int64_t ldt, int n, int np,
                           double* __restrict__ frag, double* __restrict__ diag,
                           const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int nb = np / 8;
    const int nfrag = np * np;  // (np/16) * nb * 128
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    auto tval = [&](int r, int c) -> double {
        if (r < n && c < n) return T[static_cast<int64_t>(r) * ldt + c];
        return r == c ? 1.0 : 0.0;
    };
    if (e < nfrag) {
        const int i = e & 3, lane = (e >> 2) & 31, blk = e >> 7;
        const int kc = blk / nb, J = blk - kc * nb;
        const int g = lane >> 2, t = lane & 3;
        const int r = 16 * kc + t + 4 * i, c = 8 * J + g;
        frag[e] = (r < 8 * J) ? -tval(r, c) : 0.0;
    } else if (e < nfrag + nb * 64) {
        const int d = e - nfrag;
        const int J = d >> 6, r = (d >> 3) & 7, c = d & 7;
        double v = 0.0;
        if (r < c) v = tval(8 * J + r, 8 * J + c);
        else if (r == c) v = 1.0 / tval(8 * J + c, 8 * J + c);
        diag[d] = v;
    }
}

// Warps per CTA: 8 when the 256-row panel fits shared memory (NP <= 64), else 4 (128-row panel).
__host__ __device__ constexpr int rowpass_warps(int np) { return np <= 64 ? 8 : 4; }
// The plain solve up to 48 columns runs two CTAs per SM (128 registers a thread, two panels fit the
// shared memory): one CTA's panel load overlaps the other's FP64 work and each scheduler has four
// warps' dependent chains to interleave.  The fused Gram keeps one CTA per SM (its partials are sized
// for one CTA per SM).
__host__ __device__ constexpr int rowpass_ctas_per_sm(int np, bool syrk) { return !syrk && np <= 48 ? 2 : 1; }

template <int NP, bool SYRK>
__global__ void __launch_bounds__(rowpass_warps(NP) * 32, rowpass_ctas_per_sm(NP, SYRK))
k_rowpass(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m, int n,
          const double* __restrict__ frag, const double* __restrict__ diag,
          double* __restrict__ gpart, int32_t* info, bool check_finite, int32_t* rowexp, int rowexp_mode,
          int32_t* colexp) {
    constexpr int S = NP + 4;    // shared-memory row stride in doubles
    constexpr int WARPS = rowpass_warps(NP);
    constexpr int ROWS = 32 * WARPS;   // panel rows: 32 per warp
    constexpr int NB = NP / 8;         // 8-column blocks
    constexpr int NT = upper_tiles(NP);
    constexpr int TPW = (NT + WARPS - 1) / WARPS;
    extern __shared__ double panel[];

    if (load_status(info) != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t npanels = (m + ROWS - 1) / ROWS;

    double gacc[SYRK ? TPW : 1][4];
    int tI[SYRK ? TPW : 1], tJ[SYRK ? TPW : 1];
    if constexpr (SYRK) {
#pragma unroll
        for (int q = 0; q < TPW; ++q) {
            gacc[q][0] = gacc[q][1] = gacc[q][2] = gacc[q][3] = 0.0;
            const int tt = warp + WARPS * q;
            if (tt < NT) tile_coords(NP, tt, tI[q], tJ[q]);
            else { tI[q] = 0; tJ[q] = 0; }
        }
    }
    bool bad = false;
    int col_e = kNoExp;   // column threadIdx.x: exponent bound over the rows this CTA solved

    for (int64_t p = blockIdx.x; p < npanels; p += gridDim.x) {
        const int64_t row0 = p * ROWS;
        for (int e = threadIdx.x; e < ROWS * NP; e += blockDim.x) {
            const int r = e / NP, c = e - r * NP;
            const int64_t gr = row0 + r;
            const bool ok = gr < m && c < n;
            cp_async8(&panel[r * S + c], ok ? X + gr * ldx + c : X, ok);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();

        // ---- blocked forward substitution of this warp's 32 rows ----
        const int wr0 = warp * 32;
        for (int J = 0; J < NB; ++J) {
            double acc[2][4], acc2[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = wr0 + mt * 16 + g + 8 * (i >> 1);
                    const int c = 8 * J + 2 * t + (i & 1);
                    acc[mt][i] = panel[r * S + c];
                    acc2[mt][i] = 0.0;
                    if (check_finite) bad |= !isfinite(acc[mt][i]);
                }
            // the 8J solved columns: full 16-wide chunks as m16n8k16, an 8-wide remainder (odd J) as
            // m16n8k8 with the first half of the chunk's fragments (its upper half is zero padding)
            const int nk = (8 * J) / 16;
            for (int kc = 0; kc < nk; ++kc) {
                const double2* fb = reinterpret_cast<const double2*>(
                    frag + ((static_cast<size_t>(kc) * NB + J) * 32 + lane) * 4);
                const double2 b01 = __ldg(fb), b23 = __ldg(fb + 1);
                const double b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    double a[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        a[i] = panel[(wr0 + mt * 16 + g + 8 * (i & 1)) * S + kc * 16 + t + 4 * (i >> 1)];
                    if (kc & 1) mma_f64_16816(acc2[mt], a, b);
                    else mma_f64_16816(acc[mt], a, b);
                }
            }
            if (J & 1) {
                const double2 b01 = __ldg(reinterpret_cast<const double2*>(
                    frag + ((static_cast<size_t>(nk) * NB + J) * 32 + lane) * 4));
                const double b[2] = {b01.x, b01.y};
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    double a[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        a[i] = panel[(wr0 + mt * 16 + g + 8 * (i & 1)) * S + nk * 16 + t + 4 * (i >> 1)];
                    if (nk & 1) mma_f64_1688(acc2[mt], a, b);
                    else mma_f64_1688(acc[mt], a, b);
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = wr0 + mt * 16 + g + 8 * (i >> 1);
                    const int c = 8 * J + 2 * t + (i & 1);
                    panel[r * S + c] = acc[mt][i] + acc2[mt][i];
                }
            __syncwarp();
            {
                double* xr = &panel[(wr0 + lane) * S + 8 * J];
                const double* d = diag + J * 64;
                double x[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) x[c] = xr[c];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    double v = x[c];
#pragma unroll
                    for (int k = 0; k < c; ++k) v -= x[k] * __ldg(d + k * 8 + c);
                    x[c] = v * __ldg(d + c * 9);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) xr[c] = x[c];
            }
            __syncwarp();
        }
        __syncthreads();

        for (int e = threadIdx.x; e < ROWS * NP; e += blockDim.x) {
            const int r = e / NP, c = e - r * NP;
            const int64_t gr = row0 + r;
            if (gr < m && c < n) Y[gr * ldy + c] = panel[r * S + c];
        }
        // power-of-two bounds of the solved rows (one thread per row) and columns, for the
        // split-precision products that read A1 next
        if (rowexp) {
            const int r = threadIdx.x;          // ROWS == blockDim.x
            const int64_t gr = row0 + r;
            if (gr < m) {
                int e = kNoExp;
                for (int c = 0; c < n; ++c) {
                    const int ec = exp_bound(panel[r * S + c]);
                    e = ec > e ? ec : e;
                }
                if (rowexp_mode == 2 && rowexp[gr] > e) e = rowexp[gr];
                rowexp[gr] = e;
            }
        }
        if (colexp && threadIdx.x < n) {
            const int c = threadIdx.x;
            const int64_t rows = (m - row0) < ROWS ? (m - row0) : ROWS;
            for (int r = 0; r < rows; ++r) {
                const int ec = exp_bound(panel[r * S + c]);
                col_e = ec > col_e ? ec : col_e;
            }
        }

        if constexpr (SYRK) {
#pragma unroll
            for (int q = 0; q < TPW; ++q) {
                if (warp + WARPS * q < NT) {
                    const int I = tI[q], Jt = tJ[q];
#pragma unroll 2
                    for (int kc = 0; kc < ROWS / 16; ++kc) {
                        double a[8], b[4];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            a[i] = panel[(kc * 16 + t + 4 * (i >> 1)) * S + 16 * I + g + 8 * (i & 1)];
#pragma unroll
                        for (int i = 0; i < 4; ++i) b[i] = panel[(kc * 16 + t + 4 * i) * S + 8 * Jt + g];
                        mma_f64_16816(gacc[q], a, b);
                    }
                }
            }
        }
        __syncthreads();
    }

    if constexpr (SYRK) {
        double* out = gpart + static_cast<size_t>(blockIdx.x) * NP * NP;
#pragma unroll
        for (int q = 0; q < TPW; ++q) {
            if (warp + WARPS * q < NT) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int pr = 16 * tI[q] + g + 8 * (i >> 1);
                    const int pc = 8 * tJ[q] + 2 * t + (i & 1);
                    out[pr * NP + pc] = gacc[q][i];
                }
            }
        }
    }
    if (colexp && threadIdx.x < n && col_e > kNoExp) atomicMax(&colexp[threadIdx.x], col_e);
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
}

// G[p][q] = G[q][p] = sum over CTAs b = 0..nparts-1 (in this order) of part_b[p][q], q >= p.
__global__ void k_gram_reduce(const double* __restrict__ gpart, int nparts, int np, int n,
                              double* __restrict__ G, int64_t ldg, const int32_t* info) {
    if (load_status(info) != 0) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int p = e / n, q = e - p * n;
    if (q < p) return;
    double sum = 0.0;
    for (int b = 0; b < nparts; ++b) sum += gpart[static_cast<size_t>(b) * np * np + p * np + q];
    G[static_cast<int64_t>(p) * ldg + q] = sum;
    G[static_cast<int64_t>(q) * ldg + p] = sum;
}

// ---- host launchers ------------------------------------------------------------------------------
void launch_prep_tri(const double* T, int64_t ldt, int n, int np, double* frag, double* diag,
                     const int32_t* info, cudaStream_t st) {
    const int total = np * np + (np / 8) * 64;
    k_prep_tri<<<(total + 255) / 256, 256, 0, st>>>(T, ldt, n, np, frag, diag, info);
}

size_t rowpass_smem_bytes(int np) {
    return static_cast<size_t>(32 * rowpass_warps(np)) * (np + 4) * sizeof(double);
}

template <int NP, bool SYRK>
static cudaError_t launch_rowpass_t(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                                    int n, const double* frag, const double* diag, double* gpart,
                                    int32_t* info, int grid, cudaStream_t st, bool check, int32_t* rowexp,
                                    int rowexp_mode, int32_t* colexp) {
    const size_t smem = rowpass_smem_bytes(NP);
    cudaError_t err = cudaFuncSetAttribute(k_rowpass<NP, SYRK>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    if (rowpass_ctas_per_sm(NP, SYRK) > 1) {
        const int64_t npanels = (m + 32 * rowpass_warps(NP) - 1) / (32 * rowpass_warps(NP));
        const int64_t g = static_cast<int64_t>(grid) * rowpass_ctas_per_sm(NP, SYRK);
        grid = static_cast<int>(g < npanels ? g : npanels);
    }
    k_rowpass<NP, SYRK><<<grid, 32 * rowpass_warps(NP), smem, st>>>(X, ldx, Y, ldy, m, n, frag, diag, gpart, info,
                                                                    check, rowexp, rowexp_mode, colexp);
    return cudaGetLastError();
}

template <bool SYRK>
static cudaError_t launch_rowpass_np(int np, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                     int64_t m, int n, const double* frag, const double* diag,
                                     double* gpart, int32_t* info, int grid, cudaStream_t st, bool check,
                                     int32_t* rowexp, int rowexp_mode, int32_t* colexp) {
    switch (np) {
#define RPQ_CASE(V)                                                                                     \
    case V:                                                                                             \
        return launch_rowpass_t<V, SYRK>(X, ldx, Y, ldy, m, n, frag, diag, gpart, info, grid, st, check, \
                                         rowexp, rowexp_mode, colexp);
        RPQ_CASE(16) RPQ_CASE(32) RPQ_CASE(48) RPQ_CASE(64) RPQ_CASE(80) RPQ_CASE(96) RPQ_CASE(112)
        RPQ_CASE(128)
#undef RPQ_CASE
        default: return cudaErrorInvalidValue;
    }
}

// check_finite: set NONFINITE when an input entry is NaN/Inf.  rowexp (optional): exponent bound of
// every solved row over its n columns, stored (rowexp_mode 1) or max-merged (2); colexp (optional,
// pre-filled with kNoExp): exponent bound of every column over all rows (atomicMax).
cudaError_t launch_rowpass_ex(bool syrk, int np, const double* X, int64_t ldx, double* Y, int64_t ldy,
                              int64_t m, int n, const double* frag, const double* diag, double* gpart,
                              int32_t* info, int grid, cudaStream_t st, bool check_finite, int32_t* rowexp,
                              int rowexp_mode, int32_t* colexp) {
    return syrk ? launch_rowpass_np<true>(np, X, ldx, Y, ldy, m, n, frag, diag, gpart, info, grid, st,
                                          check_finite, rowexp, rowexp_mode, colexp)
                : launch_rowpass_np<false>(np, X, ldx, Y, ldy, m, n, frag, diag, gpart, info, grid, st,
                                           check_finite, rowexp, rowexp_mode, colexp);
}

// The fused Gram pass checks its input for NaN/Inf, the plain solve does not.
cudaError_t launch_rowpass(bool syrk, int np, const double* X, int64_t ldx, double* Y, int64_t ldy,
                           int64_t m, int n, const double* frag, const double* diag, double* gpart,
                           int32_t* info, int grid, cudaStream_t st) {
    return launch_rowpass_ex(syrk, np, X, ldx, Y, ldy, m, n, frag, diag, gpart, info, grid, st, syrk, nullptr, 0,
                             nullptr);
}

void launch_gram_reduce(const double* gpart, int nparts, int np, int n, double* G, int64_t ldg,
                        const int32_t* info, cudaStream_t st) {
    const int total = n * n;
    k_gram_reduce<<<(total + 255) / 256, 256, 0, st>>>(gpart, nparts, np, n, G, ldg, info);
}

}  // namespace rpq
