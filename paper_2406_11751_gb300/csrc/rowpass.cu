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
#include "rowpass.cuh"

namespace rpq {

__global__ void k_prep_tri(const double* __restrict__ T, int64_t ldt, int n, int np,
                           double* __restrict__ frag, double* __restrict__ diag,
                           const int32_t* info) {
    if (info && load_status(info) != 0) return;
    prep_tri_entry(T, ldt, n, np, frag, diag, blockIdx.x * blockDim.x + threadIdx.x);
}

template <int NP, bool SYRK>
__global__ void __launch_bounds__(rowpass_warps(NP) * 32, rowpass_ctas_per_sm(NP, SYRK))
k_rowpass(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m, int n,
          const double* __restrict__ frag, const double* __restrict__ diag,
          double* __restrict__ gpart, int32_t* info, bool check_finite, int32_t* rowexp, int rowexp_mode,
          int32_t* colexp) {
    extern __shared__ double panel[];
    if (load_status(info) != 0) return;
    double* out = SYRK ? gpart + static_cast<size_t>(blockIdx.x) * NP * NP : nullptr;
    const bool bad = rowpass_panels<NP, SYRK, true, true>(
        X, ldx, Y, ldy, m, n, frag, diag, check_finite, rowexp, rowexp_mode, colexp, blockIdx.x, gridDim.x, panel,
        [] {}, [out](int pr, int pc, double v) { out[pr * NP + pc] = v; });
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
