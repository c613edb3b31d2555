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

// ---- blocked Cholesky for np > 128 (right-looking over 32 x 32 blocks, on many SMs) ---------------------
// The n x n Cholesky G = R^T R takes n^3/3 FP64 flops, 45 MFLOP at n = 512: about 5.5 ms on the FP64
// units of one SM, so the wide factorisation spreads every step over the SMs.  R (np x np row-major) is
// the work array: k_chol_init copies G's upper triangle (zero below, identity padding); step k of
// nb = ceil(n / 32) is
//   k_chol_panel (nb - k CTAs): every CTA factors the updated diagonal block W_kk = R_kk^T R_kk itself
//     (32 column steps in shared memory); CTA 0 stores R_kk and reports a non-positive pivot; CTA c > 0
//     solves R_{k,k+c} = R_kk^{-T} W_{k,k+c} (forward substitution, one thread per column);
//   k_chol_trail (one CTA per block pair k < i <= j): W_ij -= R_ki^T R_kj.
// Every sum runs in a fixed order, so the factor does not depend on the launch shape.
constexpr int kCb = 32;

__global__ void k_chol_init(const double* __restrict__ G, int64_t ldg, int n, int np, double* __restrict__ R,
                            const int32_t* info) {
    if (load_status(info) != 0) return;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= static_cast<int64_t>(np) * np) return;
    const int r = static_cast<int>(e / np), c = static_cast<int>(e % np);
    double v;
    if (r >= n || c >= n) v = r == c ? 1.0 : 0.0;
    else v = r <= c ? G[static_cast<int64_t>(r) * ldg + c] : 0.0;
    R[e] = v;
}

// The updated diagonal block (rows/columns k0 .. k0 + nk - 1) factored in shared memory: d[i][j] (i <= j)
// becomes R_kk; returns (in *bad) the first non-positive pivot's local index, or -1.  256 threads.
__device__ __forceinline__ void chol_block32(double (*d)[kCb + 1], int nk, int* bad) {
    const int tid = threadIdx.x;
    for (int i = 0; i < nk; ++i) {
        __syncthreads();
        if (tid == 0) {
            const double piv = d[i][i];
            if (!(piv > 0.0) && *bad < 0) *bad = i;
            d[i][i] = piv > 0.0 ? sqrt(piv) : 1.0;
        }
        __syncthreads();
        const double inv = 1.0 / d[i][i];
        for (int j = i + 1 + tid; j < nk; j += blockDim.x) d[i][j] *= inv;
        __syncthreads();
        // trailing part of the block: d[j][l] -= d[i][j] d[i][l], i < j <= l
        for (int e = tid; e < (nk - i - 1) * (nk - i - 1); e += blockDim.x) {
            const int j = i + 1 + e / (nk - i - 1), l = i + 1 + e % (nk - i - 1);
            if (j <= l) d[j][l] -= d[i][j] * d[i][l];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_chol_panel(double* __restrict__ R, int n, int np, int k, int32_t* info) {
    __shared__ double d[kCb][kCb + 1];
    __shared__ int bad;
    if (load_status(info) != 0) return;
    const int tid = threadIdx.x;
    const int k0 = k * kCb, nk = n - k0 < kCb ? n - k0 : kCb;
    for (int e = tid; e < kCb * kCb; e += blockDim.x) {
        const int i = e / kCb, j = e % kCb;
        d[i][j] = (i < nk && j < nk && i <= j) ? R[static_cast<int64_t>(k0 + i) * np + k0 + j] : 0.0;
    }
    if (tid == 0) bad = -1;
    chol_block32(d, nk, &bad);
    const int c = blockIdx.x;
    if (c == 0) {
        for (int e = tid; e < nk * nk; e += blockDim.x) {
            const int i = e / nk, j = e % nk;
            if (i <= j) R[static_cast<int64_t>(k0 + i) * np + k0 + j] = d[i][j];
        }
        if (tid == 0 && bad >= 0) set_status(info, RPCHOLQR_ERR_NOT_SPD, k0 + bad);
        return;
    }
    if (bad >= 0) return;
    // R_{k,j} = R_kk^{-T} W_{k,j} for column block j = k + c: thread = column, rows i in order
    const int j0 = (k + c) * kCb, nj = n - j0 < kCb ? n - j0 : kCb;
    if (tid < nj) {
        double x[kCb];
        const int64_t col = j0 + tid;
#pragma unroll
        for (int i = 0; i < kCb; ++i) {
            if (i < nk) {
                double v = R[static_cast<int64_t>(k0 + i) * np + col];
                for (int p = 0; p < i; ++p) v -= d[p][i] * x[p];
                x[i] = v / d[i][i];
                R[static_cast<int64_t>(k0 + i) * np + col] = x[i];
            }
        }
    }
}

// W_ij -= R_ki^T R_kj for the block pair of this CTA (i <= j, both > k); 256 threads, 4 outputs each.
__global__ void __launch_bounds__(256) k_chol_trail(double* __restrict__ R, int n, int np, int k, const int32_t* info) {
    __shared__ double a[kCb][kCb + 1], b[kCb][kCb + 1];
    if (load_status(info) != 0) return;
    const int nb = (n + kCb - 1) / kCb, m = nb - k - 1;
    // pair index -> (i, j), k < i <= j < nb: row-major over the upper triangle of the m x m trailing blocks
    int t = blockIdx.x, ii = 0;
    while (t >= m - ii) { t -= m - ii; ++ii; }
    const int bi = k + 1 + ii, bj = bi + t;
    const int k0 = k * kCb, nk = n - k0 < kCb ? n - k0 : kCb;
    const int i0 = bi * kCb, j0 = bj * kCb;
    const int tid = threadIdx.x;
    for (int e = tid; e < kCb * kCb; e += blockDim.x) {
        const int p = e / kCb, q = e % kCb;
        a[p][q] = (p < nk && i0 + q < n) ? R[static_cast<int64_t>(k0 + p) * np + i0 + q] : 0.0;
        b[p][q] = (p < nk && j0 + q < n) ? R[static_cast<int64_t>(k0 + p) * np + j0 + q] : 0.0;
    }
    __syncthreads();
    const int q = tid & 31, r0 = tid >> 5;   // column q of the tile, rows r0, r0 + 8, r0 + 16, r0 + 24
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
        const int r = r0 + 8 * rr;
        const int gi = i0 + r, gj = j0 + q;
        if (gi < n && gj < n && gi <= gj) {
            double sum = 0.0;
            for (int p = 0; p < nk; ++p) sum = fma(a[p][r], b[p][q], sum);
            R[static_cast<int64_t>(gi) * np + gj] -= sum;
        }
    }
}

__global__ void k_chol_out(const double* __restrict__ R, int n, int np, double* __restrict__ R_user,
                           const int32_t* info) {
    if (load_status(info) != 0) return;
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= static_cast<int64_t>(n) * n) return;
    const int r = static_cast<int>(e / n), c = static_cast<int>(e % n);
    R_user[e] = R[static_cast<int64_t>(r) * np + c];
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
        const int64_t tot = static_cast<int64_t>(np) * np;
        k_chol_init<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(G, ldg, n, np, R, info);
        const int nb = (n + kCb - 1) / kCb;
        for (int k = 0; k < nb; ++k) {
            k_chol_panel<<<nb - k, 256, 0, st>>>(R, n, np, k, info);
            const int m = nb - k - 1;
            if (m > 0) k_chol_trail<<<m * (m + 1) / 2, 256, 0, st>>>(R, n, np, k, info);
        }
        if (R_user)
            k_chol_out<<<static_cast<unsigned>((static_cast<int64_t>(n) * n + 255) / 256), 256, 0, st>>>(R, n, np,
                                                                                                     R_user, info);
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
