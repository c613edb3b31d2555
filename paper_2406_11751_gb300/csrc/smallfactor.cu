// The small dense steps of Algorithm alg_2 (Section 4):
//   'factor'   A_s = Q_s R_s   -- Householder QR of the s x n sample, one CTA;
//   'Cholesky' G_1 = R_1^T R_1 -- n x n upper Cholesky, one CTA;
//   'recover'  R = R_1 R_s     -- product of upper-triangular factors, one CTA per row.
#include <cfloat>

#include "common.cuh"

namespace rpq {

constexpr int kQrThreads = 1024;

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

// Householder QR of W (s x n, column-major, ld lds; overwritten).  Reflector for column j:
// beta = -sign(alpha) ||x||, v = x / (alpha - beta) with v_j = 1, tau = (beta - alpha) / beta;
// a column with nothing below the diagonal is left as is (tau = 0).  On exit Rs (np x np,
// row-major, ld np) holds R_s with each row negated where its diagonal was negative, padded with
// the identity; Rs_user (optional, n x n, ld n) receives the same n x n block.  A diagonal that is
// 0, subnormal or not finite sets SINGULAR_SKETCH.
__global__ void __launch_bounds__(kQrThreads)
k_householder(double* __restrict__ W, int64_t lds, int s, int n, int np, double* __restrict__ Rs,
              double* __restrict__ Rs_user, int32_t* info) {
    extern __shared__ double qsm[];
    double* v = qsm;            // s
    double* red = qsm + s;      // 32
    if (load_status(info) != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;

    for (int j = 0; j < n; ++j) {
        double* colj = W + static_cast<int64_t>(j) * lds;
        double part = 0.0;
        for (int i = j + 1 + tid; i < s; i += blockDim.x) part += colj[i] * colj[i];
        const double sigma = block_sum(part, red);
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
        for (int i = j + tid; i < s; i += blockDim.x) v[i] = (i == j) ? 1.0 : colj[i] * inv;
        __syncthreads();
        if (tid == 0) colj[j] = beta;
        if (tau != 0.0) {
            for (int k = j + 1 + warp; k < n; k += nwarps) {
                double* colk = W + static_cast<int64_t>(k) * lds;
                double w = 0.0;
                for (int i = j + lane; i < s; i += 32) w += v[i] * colk[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                const double tw = tau * w;
                for (int i = j + lane; i < s; i += 32) colk[i] -= v[i] * tw;
            }
        }
        __syncthreads();
    }

    bool singular = false;
    for (int e = tid; e < np * np; e += blockDim.x) {
        const int r = e / np, c = e - r * np;
        double val;
        if (r < n && c < n) {
            const double d = W[static_cast<int64_t>(r) * lds + r];
            const double sg = d < 0.0 ? -1.0 : 1.0;
            val = (c >= r) ? sg * W[static_cast<int64_t>(c) * lds + r] : 0.0;
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
// G: n x n (ld ldg).  R: np x np row-major (ld np), padded with the identity; R_user (optional,
// n x n, ld n).  A pivot t_j that is not > 0 sets NOT_SPD with pivot j.
__global__ void __launch_bounds__(256)
k_cholesky(const double* __restrict__ G, int64_t ldg, int n, int np, double* __restrict__ R,
           double* __restrict__ R_user, int32_t* info) {
    extern __shared__ double csm[];  // np x np working copy of R (row-major)
    __shared__ double diag_s;
    __shared__ int fail_s;
    if (load_status(info) != 0) return;
    const int tid = threadIdx.x;
    for (int e = tid; e < np * np; e += blockDim.x) csm[e] = 0.0;
    if (tid == 0) fail_s = -1;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        for (int l = j + tid; l < n; l += blockDim.x) {
            double tl = G[static_cast<int64_t>(j) * ldg + l];
            for (int k = 0; k < j; ++k) tl -= csm[k * np + j] * csm[k * np + l];
            csm[j * np + l] = tl;
        }
        __syncthreads();
        if (tid == 0) {
            const double d = csm[j * np + j];
            if (!(d > 0.0)) fail_s = j;
            else diag_s = sqrt(d);
            if (fail_s < 0) csm[j * np + j] = diag_s;
        }
        __syncthreads();
        if (fail_s >= 0) break;
        const double rjj = diag_s;
        for (int l = j + 1 + tid; l < n; l += blockDim.x) csm[j * np + l] /= rjj;
        __syncthreads();
    }
    if (fail_s >= 0) {
        if (tid == 0) set_status(info, RPCHOLQR_ERR_NOT_SPD, fail_s);
        return;
    }
    for (int e = tid; e < np * np; e += blockDim.x) {
        const int r = e / np, c = e - r * np;
        double val = (r < n && c < n) ? csm[e] : (r == c ? 1.0 : 0.0);
        R[e] = val;
        if (R_user && r < n && c < n) R_user[r * n + c] = val;
    }
}

// R[i][j] = sum_{k=i..j} R1[i][k] Rs[k][j] for j >= i, 0 below; block i = row i.
__global__ void k_triu_mul(const double* __restrict__ R1, int64_t ld1, const double* __restrict__ Rs,
                           int64_t lds, int n, double* __restrict__ R, int64_t ldr,
                           const int32_t* info) {
    if (info && load_status(info) != 0) return;
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double acc = 0.0;
        for (int k = i; k <= j; ++k) acc += R1[i * ld1 + k] * Rs[k * lds + j];
        R[static_cast<int64_t>(i) * ldr + j] = acc;
    }
}

// W = T^{-1} for upper-triangular T (n x n, ld ldt), by back substitution, one column per thread:
//   W[j][j] = 1/T[j][j],  W[i][j] = -(sum_{k=i+1..j} T[i][k] W[k][j]) / T[i][i]  (i < j).
// W: np x np row-major (ld np), padded with the identity.
__global__ void __launch_bounds__(256) k_triu_inv(const double* __restrict__ T, int64_t ldt, int n, int np,
                                                  double* __restrict__ W, const int32_t* info) {
    if (info && load_status(info) != 0) return;
    for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
        const int r = e / np, c = e - r * np;
        if (r >= n || c >= n || r > c) W[e] = (r == c) ? 1.0 : 0.0;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        W[j * np + j] = 1.0 / T[static_cast<int64_t>(j) * ldt + j];
        for (int i = j - 1; i >= 0; --i) {
            double acc = 0.0;
            for (int k = i + 1; k <= j; ++k) acc += T[static_cast<int64_t>(i) * ldt + k] * W[k * np + j];
            W[i * np + j] = -acc / T[static_cast<int64_t>(i) * ldt + i];
        }
    }
}

// ---- host launchers ------------------------------------------------------------------------------
size_t householder_smem_bytes(int s) { return (static_cast<size_t>(s) + 40) * sizeof(double); }

cudaError_t launch_householder(double* W, int64_t lds, int s, int n, int np, double* Rs,
                               double* Rs_user, int32_t* info, cudaStream_t st) {
    const size_t smem = householder_smem_bytes(s);
    cudaError_t err = cudaFuncSetAttribute(k_householder, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    k_householder<<<1, kQrThreads, smem, st>>>(W, lds, s, n, np, Rs, Rs_user, info);
    return cudaGetLastError();
}

cudaError_t launch_cholesky(const double* G, int64_t ldg, int n, int np, double* R, double* R_user,
                            int32_t* info, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(np) * np * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    k_cholesky<<<1, 256, smem, st>>>(G, ldg, n, np, R, R_user, info);
    return cudaGetLastError();
}

void launch_triu_mul(const double* R1, int64_t ld1, const double* Rs, int64_t lds, int n, double* R,
                     int64_t ldr, const int32_t* info, cudaStream_t st) {
    const int threads = n < 32 ? 32 : (n > 256 ? 256 : (n + 31) / 32 * 32);
    k_triu_mul<<<n, threads, 0, st>>>(R1, ld1, Rs, lds, n, R, ldr, info);
}

}  // namespace rpq

namespace rpq {
void launch_triu_inv(const double* T, int64_t ldt, int n, int np, double* W, const int32_t* info,
                     cudaStream_t st) {
    k_triu_inv<<<1, 128, 0, st>>>(T, ldt, n, np, W, info);
}
}  // namespace rpq
