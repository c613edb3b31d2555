// The small dense steps of Algorithm alg_2 (Section 4):
//   'factor'   A_s = Q_s R_s   -- Householder QR of the s x n sample on a 16-CTA cluster;
//   'Cholesky' G_1 = R_1^T R_1 -- n x n upper Cholesky, one CTA;
//   'recover'  R = R_1 R_s     -- product of upper-triangular factors, one CTA per row.
#include <cfloat>

#include "smallfactor.cuh"

namespace rpq {

// Block-wide sum of one double per thread (every thread gets the result).
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kClusterQrThreads)
k_hh_cluster(double* __restrict__ W, int64_t lds, int s, int n, int np, double* __restrict__ Rs,
             double* __restrict__ Rs_user, const int32_t* info_in, int32_t* info) {
    extern __shared__ double qsm[];
    // every CTA of the cluster sees the same status, so all take the same number of barriers
    if (load_status(info_in) != 0) return;
    hh_factor<true>(W, lds, s, n, np, Rs, Rs_user, info, cluster_rank(), cluster_size(), qsm);
}

__global__ void __launch_bounds__(kCholThreads)
k_cholesky(const double* __restrict__ G, int64_t ldg, int n, int np, double* __restrict__ R,
           double* __restrict__ R_user, int32_t* info) {
    extern __shared__ double csm[];  // np x np working copy of R (row-major), then kCholParts x np partials
    if (load_status(info) != 0) return;
    cholesky_small<kCholThreads>(G, ldg, n, np, R, R_user, info, csm);
}

// The same factorisation for np > 128, working in global memory: R (np x np) is the work array, held
// column-major while factoring (column l of R contiguous, so the lanes of a warp read both operands of
// a dot product coalesced) and transposed to row-major at the end.  Left-looking: step j forms row j,
// R[j][l] = G[j][l] - sum_{k<j} R[k][j] R[k][l], one warp per column l splitting the sum over its lanes.
__global__ void __launch_bounds__(1024)
k_cholesky_wide(const double* __restrict__ G, int64_t ldg, int n, int np, double* __restrict__ R,
                double* __restrict__ R_user, int32_t* info) {
    __shared__ double diag_s;
    __shared__ int fail_s;
    if (load_status(info) != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
    for (int e = tid; e < np * np; e += blockDim.x) R[e] = 0.0;
    if (tid == 0) fail_s = -1;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const double* cj = R + static_cast<size_t>(j) * np;   // column j (rows < j are final)
        for (int l = j + warp; l < n; l += nwarps) {
            const double* cl = R + static_cast<size_t>(l) * np;
            double part = 0.0;
            for (int k = lane; k < j; k += 32) part = fma(cj[k], cl[k], part);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) R[static_cast<size_t>(l) * np + j] = G[static_cast<int64_t>(j) * ldg + l] - part;
        }
        __syncthreads();
        if (tid == 0) {
            const double d = R[static_cast<size_t>(j) * np + j];
            if (!(d > 0.0)) fail_s = j;
            else { diag_s = sqrt(d); R[static_cast<size_t>(j) * np + j] = diag_s; }
        }
        __syncthreads();
        if (fail_s >= 0) break;
        const double inv = 1.0 / diag_s;
        for (int l = j + 1 + tid; l < n; l += blockDim.x) R[static_cast<size_t>(l) * np + j] *= inv;
        __syncthreads();
    }
    if (fail_s >= 0) {
        if (tid == 0) set_status(info, RPCHOLQR_ERR_NOT_SPD, fail_s);
        return;
    }
    // column-major -> row-major
    for (int e = tid; e < np * np; e += blockDim.x) {
        const int r = e / np, c = e - r * np;
        if (r < c) {
            const double t = R[e];
            R[e] = R[static_cast<size_t>(c) * np + r];
            R[static_cast<size_t>(c) * np + r] = t;
        }
    }
    __syncthreads();
    for (int e = tid; e < np * np; e += blockDim.x) {
        const int r = e / np, c = e - r * np;
        if (r >= n || c >= n) R[e] = (r == c) ? 1.0 : 0.0;
        else if (R_user) R_user[r * n + c] = R[e];
    }
}

// R[i][j] = sum_{k=i..j} R1[i][k] Rs[k][j] for j >= i, 0 below; block i = row i.
__global__ void k_triu_mul(const double* __restrict__ R1, int64_t ld1, const double* __restrict__ Rs,
                           int64_t lds, int n, double* __restrict__ R, int64_t ldr,
                           const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        R[static_cast<int64_t>(i) * ldr + j] = triu_mul_entry(R1, ld1, Rs, lds, i, j);
}

// W = T^{-1} for upper-triangular T (n x n, ld ldt, n <= 512): back substitution, one warp per column.
//   W[j][j] = 1/T[j][j],  W[i][j] = -(sum_{k=i+1..j} T[i][k] W[k][j]) / T[i][i]  (i < j).
// Column j lives in the registers of its warp (lane l holds rows l, l+32, ...); the dot product
// of each step is split over the lanes and summed with shuffles; reciprocal diagonals are formed once.
// W: np x np row-major (ld np), padded with the identity.  kQ = rows per lane (n <= 32 kQ).
template <int kQ>
__global__ void __launch_bounds__(256) k_triu_inv(const double* __restrict__ T, int64_t ldt, int n, int np,
                                                  double* __restrict__ W, const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps_total = (gridDim.x * blockDim.x) >> 5;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < np * np; e += gridDim.x * blockDim.x) {
        const int r = e / np, c = e - r * np;
        if (r >= n || c >= n || r > c) W[e] = (r == c) ? 1.0 : 0.0;
    }
    double rinv[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const int i = lane + 32 * q;
        rinv[q] = i < n ? 1.0 / T[static_cast<int64_t>(i) * ldt + i] : 0.0;
    }
    for (int j = gw; j < n; j += nwarps_total) {
        double w[kQ];                         // W[lane + 32q][j]
#pragma unroll
        for (int q = 0; q < kQ; ++q) w[q] = 0.0;
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            if ((j & 31) == lane && (j >> 5) == q) w[q] = rinv[q];
        for (int i = j - 1; i >= 0; --i) {
            const double* Ti = T + static_cast<int64_t>(i) * ldt;
            double part = 0.0;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const int k = lane + 32 * q;
                if (k > i && k <= j) part = fma(Ti[k], w[q], part);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            double rq = 0.0;
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                if ((i >> 5) == q) rq = rinv[q];
            const double ri = __shfl_sync(0xffffffffu, rq, i & 31);
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                if ((i & 31) == lane && (i >> 5) == q) w[q] = -part * ri;
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int k = lane + 32 * q;
            if (k <= j) W[k * np + j] = w[q];
        }
    }
}

// ---- host launchers ------------------------------------------------------------------------------
size_t householder_smem_bytes(int s, int n) { return (static_cast<size_t>(s) + n + 40) * sizeof(double); }

// W: s x n column-major (ld lds).  One cluster of kClusterQr CTAs (16 needs the non-portable cluster
// size; 8 is used where the device refuses 16).
cudaError_t launch_householder(double* W, int64_t lds, int s, int n, int np, double* Rs,
                               double* Rs_user, int32_t* info, cudaStream_t st) {
    const size_t smem = householder_smem_bytes(s, n);
    cudaError_t err = cudaFuncSetAttribute(k_hh_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_hh_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
    for (int csize : {kClusterQr, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(csize, 1, 1);
        cfg.blockDim = dim3(kClusterQrThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_hh_cluster, &cfg) != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            continue;
        }
        err = cudaLaunchKernelEx(&cfg, k_hh_cluster, W, lds, s, n, np, Rs, Rs_user,
                                 static_cast<const int32_t*>(info), info);
        return err == cudaSuccess ? cudaGetLastError() : err;
    }
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_cholesky(const double* G, int64_t ldg, int n, int np, double* R, double* R_user,
                            int32_t* info, cudaStream_t st) {
    if (np > kMaxNP) {
        k_cholesky_wide<<<1, 1024, 0, st>>>(G, ldg, n, np, R, R_user, info);
        return cudaGetLastError();
    }
    const size_t smem = static_cast<size_t>(np + kCholParts) * np * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    k_cholesky<<<1, kCholThreads, smem, st>>>(G, ldg, n, np, R, R_user, info);
    return cudaGetLastError();
}

void launch_triu_mul(const double* R1, int64_t ld1, const double* Rs, int64_t lds, int n, double* R,
                     int64_t ldr, const int32_t* info, cudaStream_t st) {
    const int threads = n < 32 ? 32 : (n > 256 ? 256 : (n + 31) / 32 * 32);
    k_triu_mul<<<n, threads, 0, st>>>(R1, ld1, Rs, lds, n, R, ldr, info);
}

}  // namespace rpq

namespace rpq {
__global__ void k_fill_identity(double* __restrict__ W, int np, const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < static_cast<int64_t>(np) * np) W[e] = (e / np == e % np) ? 1.0 : 0.0;
}

// W (np x np) = I.
void launch_fill_identity(double* W, int np, const int32_t* info, cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(np) * np;
    k_fill_identity<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(W, np, info);
}

void launch_triu_inv(const double* T, int64_t ldt, int n, int np, double* W, const int32_t* info,
                     cudaStream_t st) {
    if (n <= 128) k_triu_inv<4><<<(n + 7) / 8, 256, 0, st>>>(T, ldt, n, np, W, info);
    else k_triu_inv<16><<<(n + 7) / 8, 256, 0, st>>>(T, ldt, n, np, W, info);
}
}  // namespace rpq

// ---- choice of the split mode's second pass -------------------------------------------------------
// Q = A1 R1^{-1} as a split tensor-core product with the explicit inverse W = R1^{-1} is accurate to
// ~u times the product of the row bounds of A1 and the column bounds of W; its residual ||A - QR||
// grows with kappa(A1), while an FP64 row-wise substitution stays backward stable.  est =
// ||R1||_F ||W||_F / n lies between kappa(A1)/n and kappa(A1) (about 1.2 for well-sampled incoherent
// A).  The kernel writes two gate status words: the branch not taken gets kGateSkip (its kernels
// return at once), the taken one 0, and both carry an earlier error of info.
namespace rpq {

constexpr int kGateSkip = 1000;

__global__ void __launch_bounds__(1024)
k_pass2_gate(const double* __restrict__ R1, const double* __restrict__ W, int n, int np, double tau,
             const int32_t* info, int32_t* gate_split, int32_t* gate_fp64, int32_t* used_fp64) {
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        const double x = R1[r * np + c], y = W[r * np + c];
        a = fma(x, x, a);
        b = fma(y, y, b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = a; red[1][warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa += red[0][w]; sb += red[1][w]; }
        const int st = load_status(info);
        const double est = sqrt(sa) * sqrt(sb) / n;
        const bool fp = !(est <= tau);
        gate_split[0] = st ? st : (fp ? kGateSkip : 0);
        gate_fp64[0] = st ? st : (fp ? 0 : kGateSkip);
        gate_split[1] = gate_fp64[1] = -1;
        *used_fp64 = fp ? 1 : 0;
    }
}

// The first real error of the taken branch into info.
__global__ void k_gate_merge(int32_t* info, const int32_t* gate_split, const int32_t* gate_fp64) {
    if (threadIdx.x != 0 || load_status(info) != 0) return;
    const int32_t* g[2] = {gate_split, gate_fp64};
    for (int k = 0; k < 2; ++k)
        if (g[k][0] != 0 && g[k][0] != kGateSkip) {
            info[1] = g[k][1];
            info[0] = g[k][0];
            return;
        }
}

void launch_pass2_gate(const double* R1, const double* W, int n, int np, double tau, const int32_t* info,
                       int32_t* gates, cudaStream_t st) {
    k_pass2_gate<<<1, 1024, 0, st>>>(R1, W, n, np, tau, info, gates, gates + 2, gates + 4);
}
void launch_gate_merge(int32_t* info, const int32_t* gates, cudaStream_t st) {
    k_gate_merge<<<1, 32, 0, st>>>(info, gates, gates + 2);
}
}  // namespace rpq

namespace rpq {
// Shifted Cholesky-QR3's first stage (Fukaya et al. 2020, cited in Section 1): G += sigma I with
// sigma = 11 (m n + n (n + 1)) u trace(G), the trace summed in index order by one thread.
__global__ void k_scholqr3_shift(double* G, int64_t ldg, int n, int64_t m, const int32_t* info) {
    __shared__ double sigma;
    if (load_status(info) != 0) return;
    if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int i = 0; i < n; ++i) tr += G[static_cast<int64_t>(i) * ldg + i];
        sigma = 11.0 * (static_cast<double>(m) * static_cast<double>(n) +
                        static_cast<double>(n) * static_cast<double>(n + 1)) * 0x1p-53 * tr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) G[static_cast<int64_t>(i) * ldg + i] += sigma;
}

void launch_scholqr3_shift(double* G, int64_t ldg, int n, int64_t m, const int32_t* info, cudaStream_t st) {
    k_scholqr3_shift<<<1, 256, 0, st>>>(G, ldg, n, m, info);
}
}  // namespace rpq
