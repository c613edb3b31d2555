// Smoothing F = F_T D before sampling (Algorithm alg_2 samples rows of F A; the Blendenpik remark of
// Section 4: F_T a Walsh-Hadamard, cosine or Hartley transform, D a Rademacher diagonal).  F_T is
// the orthogonal Walsh-Hadamard transform of order m' = 2^p >= m in natural order, acting on A padded
// with zero rows; D_i = -1 when bit 63 of Philox word (i mod 4) of block i/4 under key (seed, 1) is
// set; the c sampled rows are drawn from [0, m') and scaled by sqrt(m'/c) (unless the plan turned the
// sample scale off).
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
#include <algorithm>

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
    __shared__ int needed;
    if (load_status(info) != 0) return;
    const int L = 1 << l1, H2 = 1 << l2, G = 1 << lg;
    // only low-index groups that hold a sampled row are transformed
    if (threadIdx.x == 0) needed = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < s; j += blockDim.x)
        if ((static_cast<int>(idx[j] & (L - 1)) >> lg) == static_cast<int>(blockIdx.x)) needed = 1;
    __syncthreads();
    if (!needed) return;
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
                                     cudaStream_t st, bool scale_sample) {
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
    const double scale = scale_sample ? std::sqrt(static_cast<double>(mp) / static_cast<double>(s)) : 1.0;
    k_wht_high_sample<<<dim3(static_cast<unsigned>(L >> lg), cbs * (kWhtCols / csub)), 256, smem2, st>>>(
        T, mp, n, l1, l2, lg, csub, idx, s, inv_sqrt_mp, scale, As, lds, info);
    return cudaGetLastError();
}

cudaError_t launch_smoothed_sample(const double* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, double* T,
                                   int64_t* idx, double* As, int64_t lds, int np, int32_t* info, cudaStream_t st,
                                   bool scale_sample) {
    return smoothed_sample_t<double>(A, m, n, lda, s, seed, T, idx, As, lds, np, info, st, scale_sample);
}

cudaError_t launch_smoothed_sample_f32(const float* A, int64_t m, int n, int64_t lda, int s, uint64_t seed,
                                       double* T, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                                       cudaStream_t st, bool scale_sample) {
    return smoothed_sample_t<float>(A, m, n, lda, s, seed, T, idx, As, lds, np, info, st, scale_sample);
}

void launch_colmajor_to_rows(const double* src, int64_t lds, int s, int n, double* dst, int64_t ldd,
                             cudaStream_t st) {
    const int64_t total = static_cast<int64_t>(s) * n;
    k_colmajor_to_rows<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(src, lds, s, n, dst, ldd);
}


// ---- the cosine transform (Remark r_exp: MATLAB's dct) --------------------------------------------------
// F_T = orthonormal DCT-II of order N = m' = 2^p on D [A; 0]:  y_k = w_k sum_i x_i cos(pi (2i+1) k / 2N).
// Makhoul's reordering turns it into one complex DFT of length N:  v_i = x_(2i) for i < N/2,
// v_(N-1-i) = x_(2i+1);  V = DFT(v);  y_k = w_k Re(exp(-i pi k / 2N) V_k).  The DFT runs as a four-step
// FFT with N = L H (i = lo + L hi, k = kH + H kL):
//   pass A (k_dct_pass_a): for each lo, the length-H DFT over hi (stride L, in shared memory), times
//                          the twiddle exp(-2 pi i lo kH / N); stored to T at row kH L + lo;
//   pass B (k_dct_pass_b): for each kH, the length-L DFT over lo (contiguous); only CTAs whose kH
//                          some sample needs run, and only sampled rows are written, scaled.
// T: complex, 8-column blocks of N rows (T[cb][r][c8]).  Radix-2 decimation-in-time in shared memory
// on bit-reversed input, twiddles from a per-CTA table (sincospi).
struct Cplx { double re, im; };
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// exp(-2 pi i t / len)
__device__ __forceinline__ Cplx unit_root(int64_t t, int64_t len) {
    double sn, cs;
    sincospi(2.0 * static_cast<double>(t) / static_cast<double>(len), &sn, &cs);
    return {cs, -sn};
}

__global__ void k_rademacher_signs(uint64_t seed, int64_t m, int8_t* __restrict__ sgn) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b * 4 >= m) return;
    uint64_t x[4] = {static_cast<uint64_t>(b), 0ull, 0ull, 0ull};
    philox4x64_10_dev(x, seed, 1ull);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (b * 4 + q < m) sgn[b * 4 + q] = (x[q] >> 63) ? -1 : 1;
}

// In-place radix-2 DIT over `len` points of U interleaved lanes (element (q, u) at buf[q * U + u]),
// bit-reversed input, natural output; tw[t] = exp(-2 pi i t / len), t < len / 2.
__device__ __forceinline__ void fft_stages(Cplx* buf, int len, int U, const Cplx* tw) {
    for (int h = 1; h < len; h <<= 1) {
        const int stride = len / (2 * h);
        for (int e = threadIdx.x; e < (len / 2) * U; e += blockDim.x) {
            const int q = e / U, u = e - q * U;
            const int j = q & (h - 1);
            const int i0 = ((q & ~(h - 1)) << 1) | j;
            const Cplx a = buf[i0 * U + u];
            const Cplx b = cmul(buf[(i0 + h) * U + u], tw[j * stride]);
            buf[i0 * U + u] = {a.re + b.re, a.im + b.im};
            buf[(i0 + h) * U + u] = {a.re - b.re, a.im - b.im};
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bit_reverse(int q, int bits) {
    return bits ? static_cast<int>(__brev(static_cast<unsigned>(q)) >> (32 - bits)) : 0;
}

// Pass A.  Grid (L / G, ceil(n / CS)).  smem: H x G x CS complex + H/2 twiddles.
template <typename TA>
__global__ void __launch_bounds__(256)
k_dct_pass_a(const TA* __restrict__ A, int64_t m, int n, int64_t lda, int p, int l1, int lg, int cs,
             const int8_t* __restrict__ sgn, Cplx* __restrict__ T, int32_t* info) {
    extern __shared__ Cplx cs_buf[];
    if (load_status(info) != 0) return;
    const int64_t N = int64_t{1} << p;
    const int L = 1 << l1, l2 = p - l1, H = 1 << l2, G = 1 << lg;
    const int U = G * cs;
    Cplx* buf = cs_buf;
    Cplx* tw = cs_buf + static_cast<size_t>(H) * U;
    const int lo0 = blockIdx.x * G, c0 = blockIdx.y * cs;
    for (int t = threadIdx.x; t < H / 2; t += blockDim.x) tw[t] = unit_root(t, H);
    bool bad = false;
    for (int e = threadIdx.x; e < H * U; e += blockDim.x) {
        const int hi = e / U, u = e - hi * U;
        const int g = u / cs, c = u - g * cs;
        const int64_t i = lo0 + g + static_cast<int64_t>(L) * hi;
        const int64_t row = i < (N + 1) / 2 ? 2 * i : 2 * (N - 1 - i) + 1;
        double v = 0.0;
        if (row < m && c0 + c < n) {
            v = static_cast<double>(A[row * lda + c0 + c]);
            bad |= !isfinite(v);
            v *= static_cast<double>(sgn[row]);
        }
        buf[bit_reverse(hi, l2) * U + u] = {v, 0.0};
    }
    __syncthreads();
    fft_stages(buf, H, U, tw);
    for (int e = threadIdx.x; e < H * U; e += blockDim.x) {
        const int kH = e / U, u = e - kH * U;
        const int g = u / cs, c = u - g * cs;
        const int col = c0 + c;
        if (col >= n) continue;
        const int64_t lo = lo0 + g;
        const Cplx y = cmul(buf[e], unit_root((lo * kH) & (N - 1), N));
        T[(static_cast<int64_t>(col >> 3) * N + static_cast<int64_t>(kH) * L + lo) * 8 + (col & 7)] = y;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
}

// Pass B.  Grid (H / GB, ceil(n / CS)).  smem: L x GB x CS complex + L/2 twiddles.
__global__ void __launch_bounds__(256)
k_dct_pass_b(const Cplx* __restrict__ T, int p, int l1, int n, int lgb, int cs, const int64_t* __restrict__ idx,
             int s, double w0, double w1, double scale, double* __restrict__ As, int64_t lds, const int32_t* info) {
    extern __shared__ Cplx cs_buf[];
    __shared__ int needed;
    if (load_status(info) != 0) return;
    const int64_t N = int64_t{1} << p;
    const int L = 1 << l1, l2 = p - l1, GB = 1 << lgb;
    const int U = GB * cs;
    const int kh0 = blockIdx.x * GB, c0 = blockIdx.y * cs;
    if (threadIdx.x == 0) needed = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < s; j += blockDim.x)
        if (((static_cast<int>(idx[j] & ((int64_t{1} << l2) - 1))) >> lgb) == static_cast<int>(blockIdx.x))
            needed = 1;
    __syncthreads();
    if (!needed) return;
    Cplx* buf = cs_buf;
    Cplx* tw = cs_buf + static_cast<size_t>(L) * U;
    for (int t = threadIdx.x; t < L / 2; t += blockDim.x) tw[t] = unit_root(t, L);
    for (int e = threadIdx.x; e < L * U; e += blockDim.x) {
        const int lo = e / U, u = e - lo * U;
        const int g = u / cs, c = u - g * cs;
        const int col = c0 + c;
        Cplx v = {0.0, 0.0};
        if (col < n) v = T[(static_cast<int64_t>(col >> 3) * N + static_cast<int64_t>(kh0 + g) * L + lo) * 8 + (col & 7)];
        buf[bit_reverse(lo, l1) * U + u] = v;
    }
    __syncthreads();
    fft_stages(buf, L, U, tw);
    for (int e = threadIdx.x; e < s * cs; e += blockDim.x) {
        const int j = e / cs, c = e - j * cs;
        const int64_t k = idx[j];
        const int kH = static_cast<int>(k & ((int64_t{1} << l2) - 1));
        if ((kH >> lgb) != static_cast<int>(blockIdx.x)) continue;
        const int col = c0 + c;
        if (col >= n) continue;
        const int kL = static_cast<int>(k >> l2);
        const Cplx V = buf[(static_cast<size_t>(kL) * GB + (kH - kh0)) * cs + c];
        double sn, cn;
        sincospi(static_cast<double>(k) / static_cast<double>(2 * N), &sn, &cn);
        const double y = V.re * cn + V.im * sn;
        As[static_cast<int64_t>(col) * lds + j] = (y * (k == 0 ? w0 : w1)) * scale;
    }
}

constexpr int kDctSmem = 64 * 1024;   // per CTA: three CTAs per SM

size_t smooth_dct_buffer_bytes(int64_t max_m, int max_n) {
    const int64_t mp = int64_t{1} << smooth_bits(max_m);
    const int64_t cbs = (max_n + 7) / 8;
    return static_cast<size_t>(cbs) * mp * 8 * sizeof(Cplx);
}

template <typename TA>
static cudaError_t dct_sample_t(const TA* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, void* Tbuf,
                                int8_t* sgn, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                                cudaStream_t st, bool scale_sample) {
    const int p = smooth_bits(m);
    if (p > kWhtMaxBits) return cudaErrorInvalidValue;
    const int64_t N = int64_t{1} << p;
    const int l1 = p <= 10 ? p : (p - 13 > 10 ? p - 13 : 10), l2 = p - l1;
    const int L = 1 << l1, H = 1 << l2;
    Cplx* T = static_cast<Cplx*>(Tbuf);
    launch_sample_indices(seed, 0, N, s, idx, st);
    k_rademacher_signs<<<static_cast<unsigned>((m + 1023) / 1024), 256, 0, st>>>(seed, m, sgn);
    // pass A shape: units G x CS with H x units complex + H/2 twiddles within the budget (64 KB, or what
    // one column of the longest transforms needs: at most 196 KB for H = 8192)
    const int budget_a = std::max(kDctSmem / static_cast<int>(sizeof(Cplx)), H + H / 2 + 1);
    const int units_a = (budget_a - H / 2 - 1) / H;
    if (units_a < 1) return cudaErrorInvalidValue;
    int csa = 8;
    while (csa > 1 && csa > units_a) csa >>= 1;
    int lga = 0;
    while ((2 << lga) * csa <= units_a && (2 << lga) <= L) ++lga;
    const size_t smem_a = (static_cast<size_t>(H) * ((1 << lga) * csa) + H / 2 + 1) * sizeof(Cplx);
    cudaError_t err = cudaFuncSetAttribute(k_dct_pass_a<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem_a));
    if (err != cudaSuccess) return err;
    k_dct_pass_a<TA><<<dim3(static_cast<unsigned>(L >> lga), (n + csa - 1) / csa), 256, smem_a, st>>>(
        A, m, n, lda, p, l1, lga, csa, sgn, T, info);
    // pass B shape
    const int budget_b = std::max(kDctSmem / static_cast<int>(sizeof(Cplx)), L + L / 2 + 1);
    const int units_b = (budget_b - L / 2 - 1) / L;
    if (units_b < 1) return cudaErrorInvalidValue;
    int csb = 8;
    while (csb > 1 && csb > units_b) csb >>= 1;
    int lgb = 0;
    while ((2 << lgb) * csb <= units_b && (2 << lgb) <= H) ++lgb;
    const size_t smem_b = (static_cast<size_t>(L) * ((1 << lgb) * csb) + L / 2 + 1) * sizeof(Cplx);
    err = cudaFuncSetAttribute(k_dct_pass_b, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_b));
    if (err != cudaSuccess) return err;
    if (np > n) {
        err = cudaMemsetAsync(As + static_cast<int64_t>(n) * lds, 0,
                              sizeof(double) * static_cast<size_t>(np - n) * static_cast<size_t>(lds), st);
        if (err != cudaSuccess) return err;
    }
    const double w0 = std::sqrt(1.0 / static_cast<double>(N)), w1 = std::sqrt(2.0 / static_cast<double>(N));
    const double scale = scale_sample ? std::sqrt(static_cast<double>(N) / static_cast<double>(s)) : 1.0;
    k_dct_pass_b<<<dim3(static_cast<unsigned>(H >> lgb), (n + csb - 1) / csb), 256, smem_b, st>>>(
        T, p, l1, n, lgb, csb, idx, s, w0, w1, scale, As, lds, info);
    return cudaGetLastError();
}

cudaError_t launch_dct_sample(const double* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, void* T,
                              int8_t* sgn, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                              cudaStream_t st, bool scale_sample) {
    return dct_sample_t<double>(A, m, n, lda, s, seed, T, sgn, idx, As, lds, np, info, st, scale_sample);
}

cudaError_t launch_dct_sample_f32(const float* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, void* T,
                                  int8_t* sgn, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                                  cudaStream_t st, bool scale_sample) {
    return dct_sample_t<float>(A, m, n, lda, s, seed, T, sgn, idx, As, lds, np, info, st, scale_sample);
}

}  // namespace rpq
