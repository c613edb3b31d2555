// Smoothing F = F_T D before sampling (Algorithm alg_2 samples rows of F A; the Blendenpik remark of
// Section 4: F_T a Walsh-Hadamard, cosine or Hartley transform, D a Rademacher diagonal).  F_T is
// the orthogonal Walsh-Hadamard transform of order m' = 2^p >= m in natural order, acting on A padded
// with zero rows; D_i = -1 when bit 63 of Philox word (i mod 4) of block i/4 under key (seed, 1) is
// set; the c sampled rows are drawn from [0, m') and scaled by sqrt(m'/c).
//
// The fast transform runs in two passes over HBM (its p butterfly stages split by row-index bits):
//   k_wht_low          tiles of L = 2^l1 consecutive rows x 8 columns in shared memory: the signs
//                      D_i, then the l1 stages of the low index bits; stored to T in 8-column
//                      blocks (T[cb][r][0..7], each tile one contiguous 128 KB region);
//   k_wht_high_sample  for CS columns and G consecutive low indices, the 2^l2 rows that differ only
//                      in the high bits (stride L) in shared memory: the remaining l2 stages; then
//                      only the sampled rows leave the SM, scaled, into the column-major sample.
// Butterflies map (a, b) to (a + b, a - b); 1/sqrt(m') and sqrt(m'/c) are applied to the sampled
// values only.  Traffic: A read once, T written and read once.
#include "common.cuh"
#include "philox.cuh"

namespace rpq {

constexpr int kWhtCols = 8;            // columns per column block of T
constexpr int kWhtLowBits = 11;        // L = 2048 rows per pass-1 tile
constexpr int kWhtLowThreads = 512;
constexpr int kWhtMaxBits = 25;        // m' <= 2^25
constexpr int kWhtHighSmem = 128 * 1024;

__device__ __forceinline__ double rademacher_sign(uint64_t seed, int64_t i) {
    uint64_t x[4] = {static_cast<uint64_t>(i >> 2), 0ull, 0ull, 0ull};
    philox4x64_10_dev(x, seed, 1ull);
    const int q = static_cast<int>(i & 3);
    const uint64_t w = q == 0 ? x[0] : q == 1 ? x[1] : q == 2 ? x[2] : x[3];
    return (w >> 63) ? -1.0 : 1.0;
}

// Pass 1.  Grid (m' / L, ceil(n / 8)).  smem: L x 9 doubles (row stride 9 avoids bank conflicts) + L signs.
template <typename TA>
__global__ void __launch_bounds__(kWhtLowThreads)
k_wht_low(const TA* __restrict__ A, int64_t m, int n, int64_t lda, int l1, uint64_t seed, double* __restrict__ T,
          int64_t mp, int32_t* info) {
    extern __shared__ double ws[];
    constexpr int CS = kWhtCols + 1;
    const int L = 1 << l1;
    double* sgn = ws + static_cast<size_t>(L) * CS;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * L;
    const int cb = blockIdx.y, c0 = cb * kWhtCols;
    const int tid = threadIdx.x;
    for (int r = tid; r < L; r += blockDim.x) sgn[r] = rademacher_sign(seed, r0 + r);
    __syncthreads();
    bool bad = false;
    for (int e = tid; e < L * kWhtCols; e += blockDim.x) {
        const int r = e / kWhtCols, c = e - r * kWhtCols;
        const int64_t row = r0 + r;
        double v = 0.0;
        if (row < m && c0 + c < n) {
            v = static_cast<double>(A[row * lda + c0 + c]);
            bad |= !isfinite(v);
        }
        ws[r * CS + c] = sgn[r] * v;
    }
    __syncthreads();
    for (int h = 1; h < L; h <<= 1) {
        for (int e = tid; e < (L / 2) * kWhtCols; e += blockDim.x) {
            const int q = e / kWhtCols, c = e - q * kWhtCols;
            const int i0 = ((q & ~(h - 1)) << 1) | (q & (h - 1));
            const double a = ws[i0 * CS + c], b = ws[(i0 + h) * CS + c];
            ws[i0 * CS + c] = a + b;
            ws[(i0 + h) * CS + c] = a - b;
        }
        __syncthreads();
    }
    double* dst = T + (static_cast<size_t>(cb) * mp + r0) * kWhtCols;
    for (int e = tid; e < L * kWhtCols; e += blockDim.x) {
        const int r = e / kWhtCols, c = e - r * kWhtCols;
        dst[e] = ws[r * CS + c];
    }
    if (__syncthreads_or(bad) && tid == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
}

// Pass 2.  Grid (L / G, ceil(n / 8) * (8 / CSUB)); CTA (g, y): column block cb = y / (8 / CSUB), columns
// cb*8 + cs0 .. + CSUB - 1, low indices g*G .. g*G + G - 1.  smem H2 x G x CSUB doubles.
__global__ void __launch_bounds__(256)
k_wht_high_sample(const double* __restrict__ T, int64_t mp, int n, int l1, int l2, int lg, int csub,
                  const int64_t* __restrict__ idx, int s, double inv_sqrt_mp, double scale,
                  double* __restrict__ As, int64_t lds, const int32_t* info) {
    extern __shared__ double hs[];
    if (load_status(info) != 0) return;
    const int L = 1 << l1, H2 = 1 << l2, G = 1 << lg;
    const int per_block = kWhtCols / csub;
    const int cb = blockIdx.y / per_block, cs0 = (blockIdx.y - cb * per_block) * csub;
    const int lo0 = blockIdx.x * G;
    const int U = G * csub;                       // units (lo, cs) per hi
    const int tid = threadIdx.x;
    const double* src = T + static_cast<size_t>(cb) * mp * kWhtCols;
    for (int e = tid; e < H2 * U; e += blockDim.x) {
        const int hi = e / U, u = e - hi * U;
        const int lo = u / csub, cs = u - lo * csub;
        hs[e] = src[(static_cast<int64_t>(hi) * L + lo0 + lo) * kWhtCols + cs0 + cs];
    }
    __syncthreads();
    for (int h = 1; h < H2; h <<= 1) {
        for (int e = tid; e < (H2 / 2) * U; e += blockDim.x) {
            const int q = e / U, u = e - q * U;
            const int i0 = ((q & ~(h - 1)) << 1) | (q & (h - 1));
            const double a = hs[i0 * U + u], b = hs[(i0 + h) * U + u];
            hs[i0 * U + u] = a + b;
            hs[(i0 + h) * U + u] = a - b;
        }
        __syncthreads();
    }
    for (int e = tid; e < s * csub; e += blockDim.x) {
        const int j = e / csub, cs = e - j * csub;
        const int64_t r = idx[j];
        const int lo = static_cast<int>(r & (L - 1));
        if ((lo >> lg) != static_cast<int>(blockIdx.x)) continue;
        const int c = cb * kWhtCols + cs0 + cs;
        if (c >= n) continue;
        const int hi = static_cast<int>(r >> l1);
        As[static_cast<int64_t>(c) * lds + j] = (hs[hi * U + (lo - lo0) * csub + cs] * inv_sqrt_mp) * scale;
    }
}

// dst (row-major s x n, ld ldd) = src (column-major, ld lds)
__global__ void k_colmajor_to_rows(const double* __restrict__ src, int64_t lds, int s, int n, double* __restrict__ dst,
                                   int64_t ldd) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= static_cast<int64_t>(s) * n) return;
    const int j = static_cast<int>(e / n), c = static_cast<int>(e - static_cast<int64_t>(j) * n);
    dst[static_cast<int64_t>(j) * ldd + c] = src[static_cast<int64_t>(c) * lds + j];
}

// ---- host side ------------------------------------------------------------------------------------
int smooth_bits(int64_t m) {
    int p = 0;
    while ((int64_t{1} << p) < m) ++p;
    return p;
}

bool smooth_supported(int64_t m) { return smooth_bits(m) <= kWhtMaxBits; }

// Bytes of the transform buffer T for up to max_m rows and max_n columns.
size_t smooth_buffer_bytes(int64_t max_m, int max_n) {
    const int64_t mp = int64_t{1} << smooth_bits(max_m);
    const int64_t cbs = (max_n + kWhtCols - 1) / kWhtCols;
    return static_cast<size_t>(cbs) * mp * kWhtCols * sizeof(double);
}

void launch_sample_indices(uint64_t seed, uint64_t stream_id, int64_t m, int32_t s, int64_t* idx, cudaStream_t st);

// Smoothed sample into As (column-major, ld lds, np columns; columns n..np-1 zeroed).  idx: device
// int64[s] scratch (receives the sample rows of F A).  A: device m x n (lda), double or float.
template <typename TA>
static cudaError_t smoothed_sample_t(const TA* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, double* T,
                                     int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                                     cudaStream_t st) {
    const int p = smooth_bits(m);
    if (p > kWhtMaxBits) return cudaErrorInvalidValue;
    const int64_t mp = int64_t{1} << p;
    const int l1 = p < kWhtLowBits ? p : kWhtLowBits, l2 = p - l1;
    const int L = 1 << l1, H2 = 1 << l2;
    const int cbs = (n + kWhtCols - 1) / kWhtCols;
    launch_sample_indices(seed, 0, mp, s, idx, st);
    const size_t smem1 = (static_cast<size_t>(L) * (kWhtCols + 1) + L) * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_wht_low<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem1));
    if (err != cudaSuccess) return err;
    k_wht_low<TA><<<dim3(static_cast<unsigned>(mp / L), cbs), kWhtLowThreads, smem1, st>>>(A, m, n, lda, l1, seed, T,
                                                                                           mp, info);
    // pass 2 shape: the most units (G low indices x CSUB columns) that fit 128 KB, columns first
    const int units = kWhtHighSmem / (H2 * static_cast<int>(sizeof(double)));
    int csub = kWhtCols;
    while (csub > 1 && csub > units) csub >>= 1;
    int lg = 0;
    while ((2 << lg) * csub <= units && (2 << lg) <= L) ++lg;
    const size_t smem2 = static_cast<size_t>(H2) * (1 << lg) * csub * sizeof(double);
    err = cudaFuncSetAttribute(k_wht_high_sample, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem2));
    if (err != cudaSuccess) return err;
    if (np > n) {
        err = cudaMemsetAsync(As + static_cast<int64_t>(n) * lds, 0,
                              sizeof(double) * static_cast<size_t>(np - n) * static_cast<size_t>(lds), st);
        if (err != cudaSuccess) return err;
    }
    const double inv_sqrt_mp = 1.0 / std::sqrt(static_cast<double>(mp));
    const double scale = std::sqrt(static_cast<double>(mp) / static_cast<double>(s));
    k_wht_high_sample<<<dim3(static_cast<unsigned>(L >> lg), cbs * (kWhtCols / csub)), 256, smem2, st>>>(
        T, mp, n, l1, l2, lg, csub, idx, s, inv_sqrt_mp, scale, As, lds, info);
    return cudaGetLastError();
}

cudaError_t launch_smoothed_sample(const double* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, double* T,
                                   int64_t* idx, double* As, int64_t lds, int np, int32_t* info, cudaStream_t st) {
    return smoothed_sample_t<double>(A, m, n, lda, s, seed, T, idx, As, lds, np, info, st);
}

cudaError_t launch_smoothed_sample_f32(const float* A, int64_t m, int n, int64_t lda, int s, uint64_t seed,
                                       double* T, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                                       cudaStream_t st) {
    return smoothed_sample_t<float>(A, m, n, lda, s, seed, T, idx, As, lds, np, info, st);
}

void launch_colmajor_to_rows(const double* src, int64_t lds, int s, int n, double* dst, int64_t ldd,
                             cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(s) * n;
    k_colmajor_to_rows<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(src, lds, s, n, dst, ldd);
}

}  // namespace rpq
