// Device-side pieces of the FP64 row passes (the row-wise solves of Algorithm alg_2, Section 4),
// shared by the row-pass kernels (rowpass.cu) and the persistent batched kernel (persist.cu).
#pragma once
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
// Entry e (0 <= e < np * np + (np / 8) * 64) of the tables above.
__device__ __forceinline__ void prep_tri_entry(const double* __restrict__ T, int64_t ldt, int n, int np,
                                               double* __restrict__ frag, double* __restrict__ diag, int e) {
    const int nb = np / 8;
    const int nfrag = np * np;  // (np/16) * nb * 128
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

// The row pass over the panels p_first, p_first + p_stride, ... of X (ROWS = rowpass_rows(NP) rows
// each) by the calling CTA: the first rowpass_warps(NP) warps solve and accumulate, every thread of the
// CTA (any number of warps >= rowpass_warps(NP)) takes part in the panel copies and barriers.  panel:
// the CTA's shared memory, rowpass_smem_bytes(NP).  With SYRK the CTA's Gram partial over its panels,
// upper 16x8 tiles, is handed over at the end: every thread calls before_emit() (a point where the
// caller may wait), then emit(pr, pc, v) for each entry it holds.  Returns this thread's non-finite
// flag (check_finite); the caller reduces it over the CTA.  FULL: the CTA has exactly
// rowpass_warps(NP) warps (every warp solves).  LDG: frag and diag are read through the read-only
// (non-coherent) cache -- only when no CTA of the same launch writes them.
template <int NP, bool SYRK, bool FULL, bool LDG, class BeforeEmit, class Emit>
__device__ __forceinline__ bool rowpass_panels(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                                               int n, const double* __restrict__ frag,
                                               const double* __restrict__ diag, bool check_finite,
                                               int32_t* rowexp, int rowexp_mode, int32_t* colexp,
                                               int64_t p_first, int64_t p_stride, double* panel,
                                               BeforeEmit before_emit, Emit emit) {
    constexpr int S = NP + 4;    // shared-memory row stride in doubles
    constexpr int WARPS = rowpass_warps(NP);
    constexpr int ROWS = 32 * WARPS;   // panel rows: 32 per warp
    constexpr int NB = NP / 8;         // 8-column blocks
    constexpr int NT = upper_tiles(NP);
    constexpr int TPW = (NT + WARPS - 1) / WARPS;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const bool solver = FULL || warp < WARPS;
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

    for (int64_t p = p_first; p < npanels; p += p_stride) {
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
        for (int J = 0; J < NB && solver; ++J) {
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
                const double2 b01 = LDG ? __ldg(fb) : fb[0], b23 = LDG ? __ldg(fb + 1) : fb[1];
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
                const double2* fb = reinterpret_cast<const double2*>(
                    frag + ((static_cast<size_t>(nk) * NB + J) * 32 + lane) * 4);
                const double2 b01 = LDG ? __ldg(fb) : fb[0];
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
                    for (int k = 0; k < c; ++k) v -= x[k] * (LDG ? __ldg(d + k * 8 + c) : d[k * 8 + c]);
                    x[c] = v * (LDG ? __ldg(d + c * 9) : d[c * 9]);
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
        if (rowexp && threadIdx.x < ROWS) {
            const int r = threadIdx.x;          // one thread per panel row
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
                if (solver && warp + WARPS * q < NT) {
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
        before_emit();
#pragma unroll
        for (int q = 0; q < TPW; ++q) {
            if (solver && warp + WARPS * q < NT) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int pr = 16 * tI[q] + g + 8 * (i >> 1);
                    const int pc = 8 * tJ[q] + 2 * t + (i & 1);
                    emit(pr, pc, gacc[q][i]);
                }
            }
        }
    }
    if (colexp && threadIdx.x < n && col_e > kNoExp) atomicMax(&colexp[threadIdx.x], col_e);
    return bad;
}

// Shared memory of one row-pass CTA: the panel, ROWS rows of NP + 4 doubles.
__host__ __device__ constexpr size_t rowpass_smem_bytes(int np) {
    return static_cast<size_t>(rowpass_rows(np)) * (np + 4) * sizeof(double);
}

}  // namespace rpq
