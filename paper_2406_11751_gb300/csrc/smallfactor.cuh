// Device-side pieces of the small dense steps of Algorithm alg_2 (Section 4) -- the Householder QR of
// the sample and the n x n Cholesky factorisation -- shared by their kernels (smallfactor.cu) and the
// persistent batched kernel (persist.cu).
#pragma once
#include <cfloat>

#include "common.cuh"

namespace rpq {

// Householder QR of the sample on one thread-block cluster.  FP64 on GB300 retires one warp-wide
// DFMA per 64 cycles per SM sub-partition, so a single CTA would run this O(s n^2) step at 1/152 of
// the GPU; instead kClusterQr CTAs (one per SM) share the columns round-robin and advance one
// column per hardware cluster barrier:
//   every CTA: read column j (rows j..s-1), form the reflector (beta = -sign(alpha)||x||,
//              v = x / (alpha - beta) with v_j = 1, tau = (beta - alpha) / beta; no reflection when
//              nothing is below the diagonal) -- identical in every CTA;
//   every CTA: apply it to its own columns k > j;
//   cluster barrier (release/acquire orders the global-memory column updates).
// The diagonal betas are kept in shared memory (column j is still being read by the other CTAs
// while it is reflected) and CTA 0 assembles R_s at the end: each row negated where its diagonal is
// negative, padded with the identity; a diagonal that is 0, subnormal or not finite sets
// SINGULAR_SKETCH.  W: s x n column-major (ld lds), overwritten.
constexpr int kClusterQr = 16;
constexpr int kClusterQrThreads = 256;

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
    return r;
}

// The factorisation itself, by the calling CTA as CTA `rank` of `csize` (CLUSTER: the CTAs of a thread-block
// cluster, joined by the hardware cluster barrier; otherwise csize = 1 and a CTA barrier).  The arithmetic
// of every column step depends on the CTA size (kClusterQrThreads threads) but not on csize, so one CTA
// alone gives the cluster's bits.  qsm: (s + n + 34) doubles of shared memory.
template <bool CLUSTER>
__device__ __forceinline__ void hh_factor(double* __restrict__ W, int64_t lds, int s, int n, int np,
                                          double* __restrict__ Rs, double* __restrict__ Rs_user, int32_t* info,
                                          unsigned rank, unsigned csize, double* qsm) {
    double* v = qsm;                 // s
    double* betas = qsm + s;         // n
    double* red = betas + n;         // 32 warp partials, then tau and 1 / (alpha - beta)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;

    for (int j = 0; j < n; ++j) {
        const double* colj = W + static_cast<int64_t>(j) * lds;
        double part = 0.0;
        for (int i = j + 1 + tid; i < s; i += blockDim.x) part += colj[i] * colj[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        // the reflector's scalars in one thread (FP64 square root and divisions are long sequences on
        // the FP64 units; formed once instead of by every thread), then shared
        if (tid == 0) {
            double sigma = 0.0;
            for (int w = 0; w < nwarps; ++w) sigma += red[w];
            const double alpha = colj[j];
            double beta, tau, inv;
            if (sigma == 0.0) {
                beta = alpha; tau = 0.0; inv = 0.0;
            } else {
                const double nrm = sqrt(alpha * alpha + sigma);
                beta = alpha >= 0.0 ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                inv = 1.0 / (alpha - beta);
            }
            betas[j] = beta;
            red[32] = tau;
            red[33] = inv;
        }
        __syncthreads();
        const double tau = red[32], inv = red[33];
        for (int i = j + tid; i < s; i += blockDim.x) v[i] = (i == j) ? 1.0 : colj[i] * inv;
        __syncthreads();
        if (tau != 0.0) {
            // this CTA's columns k > j: k = rank (mod csize); one warp per column
            const int k0 = j + 1 + static_cast<int>((rank + csize - static_cast<unsigned>((j + 1) % csize)) % csize);
            for (int k = k0 + warp * static_cast<int>(csize); k < n; k += nwarps * static_cast<int>(csize)) {
                double* colk = W + static_cast<int64_t>(k) * lds;
                // four independent partial sums keep four column loads in flight per lane
                double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
                int i = j + lane;
                for (; i + 96 < s; i += 128) {
                    w0 += v[i] * colk[i];
                    w1 += v[i + 32] * colk[i + 32];
                    w2 += v[i + 64] * colk[i + 64];
                    w3 += v[i + 96] * colk[i + 96];
                }
                for (; i < s; i += 32) w0 += v[i] * colk[i];
                double w = (w0 + w1) + (w2 + w3);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                const double tw = tau * w;
#pragma unroll 4
                for (int i2 = j + lane; i2 < s; i2 += 32) colk[i2] -= v[i2] * tw;
            }
        }
        __syncthreads();
        if constexpr (CLUSTER) cluster_sync_all();
    }

    if (rank != 0) return;
    bool singular = false;
    for (int e = tid; e < np * np; e += blockDim.x) {
        const int r = e / np, c = e - r * np;
        double val;
        if (r < n && c < n) {
            const double d = betas[r];
            const double sg = d < 0.0 ? -1.0 : 1.0;
            val = c > r ? sg * W[static_cast<int64_t>(c) * lds + r] : (c == r ? fabs(d) : 0.0);
            if (c == r && (!isfinite(d) || fabs(d) < DBL_MIN)) singular = true;
            if (Rs_user) Rs_user[r * n + c] = val;
        } else {
            val = (r == c) ? 1.0 : 0.0;
        }
        Rs[e] = val;
    }
    if (__syncthreads_or(singular) && tid == 0) set_status(info, RPCHOLQR_ERR_SINGULAR_SKETCH);
}

// Upper Cholesky G = R^T R, row by row:
//   t_l = G[j][l] - sum_{k<j} R[k][j] R[k][l]  (l >= j),  R[j][j] = sqrt(t_j),  R[j][l] = t_l / R[j][j].
// G: n x n (ld ldg), n <= 128.  R: np x np row-major (ld np), padded with the identity; R_user
// (optional, n x n, ld n).  A pivot t_j that is not > 0 sets NOT_SPD with pivot j.
// Thread (part, l) = (tid / 128, tid % 128): each dot product is split over kCholParts threads
// (k = part, part + kCholParts, ...), so that all four schedulers' FP64 units work on it; the partial
// sums are subtracted in part order.  The upper triangle of G is copied into the working matrix first,
// so a step touches shared memory only; the square root is taken once per step.
constexpr int kCholParts = 8;
constexpr int kCholThreads = 128 * kCholParts;
// The factorisation by a CTA of NT threads (NT divides kCholThreads): thread tid plays the virtual
// threads tid, tid + NT, ... of the kCholThreads-thread layout above, so every sum is formed in the same
// order whatever NT.  csm: (np * np + kCholParts * np) doubles of shared memory.  Returns false on
// NOT_SPD (status set) or when info already holds a status.
template <int NT>
__device__ __forceinline__ bool cholesky_small(const double* __restrict__ G, int64_t ldg, int n, int np,
                                               double* __restrict__ R, double* __restrict__ R_user, int32_t* info,
                                               double* csm) {
    static_assert(kCholThreads % NT == 0, "the virtual-thread layout must tile the CTA");
    double* psum = csm + np * np;
    __shared__ double diag_s;
    __shared__ int fail_s;
    const int tid = threadIdx.x;
    for (int e = tid; e < np * np; e += NT) {
        const int r = e / np, c = e - r * np;
        csm[e] = (r <= c && c < n) ? G[static_cast<int64_t>(r) * ldg + c] : 0.0;
    }
    if (tid == 0) fail_s = -1;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
#pragma unroll
        for (int vt = tid; vt < kCholThreads; vt += NT) {
            const int part = vt >> 7, l = vt & 127;
            if (l >= j && l < n) {
                double acc = 0.0;
                for (int k = part; k < j; k += kCholParts) acc += csm[k * np + j] * csm[k * np + l];
                psum[part * np + l] = acc;
            }
        }
        __syncthreads();
#pragma unroll
        for (int vt = tid; vt < kCholThreads; vt += NT) {
            const int part = vt >> 7, l = vt & 127;
            if (part == 0 && l > j && l < n) {
                double tl = csm[j * np + l];
#pragma unroll
                for (int q = 0; q < kCholParts; ++q) tl -= psum[q * np + l];
                csm[j * np + l] = tl;
            } else if (vt == 0) {
                double tj = csm[j * np + j];
#pragma unroll
                for (int q = 0; q < kCholParts; ++q) tj -= psum[q * np + j];
                if (!(tj > 0.0)) {
                    fail_s = j;
                } else {
                    diag_s = sqrt(tj);
                    csm[j * np + j] = diag_s;
                }
            }
        }
        __syncthreads();
        if (fail_s >= 0) break;
#pragma unroll
        for (int vt = tid; vt < kCholThreads; vt += NT) {
            const int part = vt >> 7, l = vt & 127;
            if (part == 0 && l > j && l < n) csm[j * np + l] /= diag_s;
        }
        __syncthreads();
    }
    if (fail_s >= 0) {
        if (tid == 0) set_status(info, RPCHOLQR_ERR_NOT_SPD, fail_s);
        return false;
    }
    for (int e = tid; e < np * np; e += NT) {
        const int r = e / np, c = e - r * np;
        double val = (r < n && c < n) ? csm[e] : (r == c ? 1.0 : 0.0);
        R[e] = val;
        if (R_user && r < n && c < n) R_user[r * n + c] = val;
    }
    return true;
}

// Entry (i, j) of R = R1 Rs for upper-triangular R1 (ld ld1) and Rs (ld lds): sum_{k=i..j} R1[i][k] Rs[k][j]
// in order of k, 0 below the diagonal.
__device__ __forceinline__ double triu_mul_entry(const double* __restrict__ R1, int64_t ld1,
                                                 const double* __restrict__ Rs, int64_t lds, int i, int j) {
    double acc = 0.0;
    for (int k = i; k <= j; ++k) acc += R1[i * ld1 + k] * Rs[k * lds + j];
    return acc;
}

}  // namespace rpq
