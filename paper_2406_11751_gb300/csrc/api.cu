// C ABI of the library (declared in include/rpcholqr.h): plans, the full rpCholesky-QR call,
// the individual steps, and the FP64 tensor-pipe probe.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace rpq {
// sample.cu
void launch_sample_rows(const double* rows, int32_t n, int32_t s, double scale, double* As, int64_t lds,
                        int32_t np, int32_t* info, cudaStream_t st);
void launch_sample_indices(uint64_t seed, uint64_t stream_id, int64_t m, int32_t s, int64_t* idx,
                           cudaStream_t st);
void launch_sample_gather(const double* A, int64_t m, int32_t n, int64_t lda, int32_t s, uint64_t seed,
                          uint64_t stream_id, double scale, double* As, int64_t lds, int32_t np,
                          int64_t* idx_out, int32_t* info, cudaStream_t st);
// smallfactor.cu
cudaError_t launch_householder(double* W, int64_t lds, int s, int n, int np, double* Rs,
                               double* Rs_user, int32_t* info, cudaStream_t st);
size_t householder_smem_bytes(int s, int n);
cudaError_t launch_cholesky(const double* G, int64_t ldg, int n, int np, double* R, double* R_user,
                            int32_t* info, cudaStream_t st);
void launch_triu_mul(const double* R1, int64_t ld1, const double* Rs, int64_t lds, int n, double* R,
                     int64_t ldr, const int32_t* info, cudaStream_t st);
// rowpass.cu
void launch_prep_tri(const double* T, int64_t ldt, int n, int np, double* frag, double* diag,
                     const int32_t* info, cudaStream_t st);
cudaError_t launch_rowpass(bool syrk, int np, const double* X, int64_t ldx, double* Y, int64_t ldy,
                           int64_t m, int n, const double* frag, const double* diag, double* gpart,
                           int32_t* info, int grid, cudaStream_t st);
void launch_gram_reduce(const double* gpart, int nparts, int np, int n, double* G, int64_t ldg,
                        const int32_t* info, cudaStream_t st);
cudaError_t launch_rowpass_ex(bool syrk, int np, const double* X, int64_t ldx, double* Y, int64_t ldy,
                              int64_t m, int n, const double* frag, const double* diag, double* gpart,
                              int32_t* info, int grid, cudaStream_t st, bool check_finite, int32_t* rowexp,
                              int rowexp_mode, int32_t* colexp);
void launch_fill_noexp(int32_t* p, int n, cudaStream_t st);
// probe.cu
cudaError_t run_fp64_mma_probe(int iters, double* flops_per_s);
// smallfactor.cu
void launch_fill_identity(double* W, int np, const int32_t* info, cudaStream_t st);
void launch_triu_inv(const double* T, int64_t ldt, int n, int np, double* W, const int32_t* info,
                     cudaStream_t st);
// ozaki.cu
size_t ozaki_yblocks_bytes(int K, int N);
int32_t ozaki_no_exp();
void launch_ozaki_slice_cols(const double* Y, int64_t ldy, int K, int N, uint8_t* blocks, int32_t* yexp,
                             const int32_t* info, cudaStream_t st);
cudaError_t launch_ozaki_gemm(bool sub, const double* X, int64_t ldx, const int32_t* xexp, int K,
                              const uint8_t* yblocks, const int32_t* yexp, int N, const double* B,
                              int64_t ldb, double* C, int64_t ldc, int64_t m, int32_t* info, int grid,
                              cudaStream_t st, long spin, bool y_upper, const uint8_t* aimg, int img_nkw,
                              const int32_t* bexp, int64_t ld_bexp);
size_t ozaki_image_bytes(int64_t m, int K);
void launch_slice_images(const double* X, int64_t ldx, int64_t m, int K, const int32_t* xexp, uint8_t* img,
                         const int32_t* info, cudaStream_t st);
void launch_slice_block_images(const double* X, int64_t ldx, int64_t m, int nc, uint8_t* img, int img_nkw, int kw0,
                               int32_t* bexp, const int32_t* info, cudaStream_t st);
int ozaki_gram_halves(int np);
int ozaki_gram_tiles(int np, bool images);
cudaError_t launch_ozaki_gram(const double* X, int64_t ldx, int64_t m, int n, int np, const int32_t* colexp,
                              int nranges, double* gpart, int32_t* info, cudaStream_t st, long spin,
                              const uint8_t* gimg, bool accum);
void launch_slice_col_images(const double* X, int64_t ldx, int64_t m, int n, int np, const int32_t* colexp,
                             uint8_t* img, const int32_t* info, cudaStream_t st);
void launch_row_exp(const double* X, int64_t ldx, int64_t m, int K, int32_t* rowexp, cudaStream_t st);
void launch_col_exp(const double* X, int64_t ldx, int64_t m, int n, int32_t* colexp, cudaStream_t st);
cudaError_t launch_gemm_sub_fp64(const double* X, int64_t ldx, const double* Y, int64_t ldy, const double* B,
                                 int64_t ldb, double* C, int64_t ldc, int64_t m, int K, int N,
                                 const int32_t* info, int grid, cudaStream_t st);
cudaError_t launch_syrk_fp64(const double* X, int64_t ldx, int64_t m, int n, int np, int ranges, double* gpart,
                             const int32_t* info, cudaStream_t st);
void launch_sample_gather_f32(const float* A, int64_t m, int32_t n, int64_t lda, int32_t s, uint64_t seed,
                              uint64_t stream_id, double scale, double* As, int64_t lds, int32_t np,
                              int64_t* idx_out, int32_t* info, cudaStream_t st);
int f32_pad(int n);
void launch_prep_f32(const double* T, int64_t ldt, int n, float* T32, float* rinv32, int fail_status,
                     int32_t* info, cudaStream_t st);
cudaError_t launch_rowsolve_f32(const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t m, int n,
                                const float* T32, const float* rinv32, int32_t* info, bool check_finite,
                                cudaStream_t st);
int launch_syrk_f32(const float* X, int64_t ldx, int64_t m, int n, int max_ranges, double* gpart,
                    const int32_t* info, cudaStream_t st);
void launch_f64_to_f32(const double* src, int64_t lds, int n, float* dst, int64_t ldd, cudaStream_t st);
void launch_gather_owned_rows(const double* A, int64_t m_local, int32_t n, int64_t lda, int64_t row_offset,
                              int64_t m, int32_t s, uint64_t seed, uint64_t stream_id, double scale, double* As,
                              int64_t ld_as, int32_t* info, cudaStream_t st);
void launch_sample_to_colmajor(const double* src, int64_t ld_src, int32_t s, int32_t n, int32_t np, double* dst,
                               int64_t lds, cudaStream_t st);
void launch_sum_parts(const double* parts, int32_t nparts, int32_t n, double* G, cudaStream_t st);
bool smooth_supported(int64_t m);
size_t smooth_buffer_bytes(int64_t max_m, int max_n);
cudaError_t launch_smoothed_sample(const double* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, double* T,
                                   int64_t* idx, double* As, int64_t lds, int np, int32_t* info, cudaStream_t st, bool scale_sample);
cudaError_t launch_smoothed_sample_f32(const float* A, int64_t m, int n, int64_t lda, int s, uint64_t seed,
                                       double* T, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                                       cudaStream_t st, bool scale_sample);
void launch_colmajor_to_rows(const double* src, int64_t lds, int s, int n, double* dst, int64_t ldd,
                             cudaStream_t st);
size_t smooth_dct_buffer_bytes(int64_t max_m, int max_n);
cudaError_t launch_dct_sample(const double* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, void* T,
                              int8_t* sgn, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                              cudaStream_t st, bool scale_sample);
cudaError_t launch_dct_sample_f32(const float* A, int64_t m, int n, int64_t lda, int s, uint64_t seed, void* T,
                                  int8_t* sgn, int64_t* idx, double* As, int64_t lds, int np, int32_t* info,
                                  cudaStream_t st, bool scale_sample);
void launch_pass2_gate(const double* R1, const double* W, int n, int np, double tau, const int32_t* info,
                       int32_t* gates, cudaStream_t st);
void launch_gate_merge(int32_t* info, const int32_t* gates, cudaStream_t st);
void launch_scholqr3_shift(double* G, int64_t ldg, int n, int64_t m, const int32_t* info, cudaStream_t st);
void launch_fill_uniform(double* A, int64_t count, uint64_t seed, cudaStream_t st);
// persist.cu
struct BatchLayout {
    int64_t mat_stride, off_rs, off_r1, off_g, off_frag_s, off_frag_1, off_diag_s, off_diag_1;
    size_t mats_bytes, ctr_off, order_off, pre_off, items_off, queue_off, total;
    int64_t max_items;
};
BatchLayout batch_layout(int32_t capacity, int32_t max_n, int32_t max_s, int sms);
size_t batch_smem_bytes(int32_t max_n, int32_t max_s);
int batch_max_np();
cudaError_t launch_batch_persistent(int32_t count, const double* const* A, const int64_t* m, const int32_t* n,
                                    const int64_t* lda, const int32_t* s, const uint64_t* seed, double* const* Q,
                                    const int64_t* ldq, double* const* R, int32_t* info, void* ws, int32_t capacity,
                                    int64_t max_m, int32_t max_n, int32_t max_s, int sms, int scale_sample,
                                    long spin, int grid, cudaStream_t st);
cudaError_t prepare_batch_persistent(int32_t max_n, int32_t max_s, int sms, int* grid);
}  // namespace rpq

using namespace rpq;

constexpr int64_t kDefaultSpinLimit = int64_t{1} << 24;

// Launch parameters the autotuner chooses (rpcholqr_autotune); 0 = the built-in rule.
struct Tuning {
    int32_t split_sub = 0;      // SPLIT64 first pass: width of the FP64 diagonal-block solves (16 or 32)
    int32_t gram_ranges = 0;    // SPLIT64 Gram: row ranges (split-K factor of G = A1^T A1)
    int32_t syrk_ranges = 0;    // FP64 Gram of wide panels: row ranges
};
// One row of the autotuner's table: the parameters measured best for (mode, padded n, ceil(log2 m)).
struct TuneEntry {
    int32_t mode = 0, np = 0, m_log2 = 0;
    Tuning t;
    double ms = 0.0;
};
constexpr int64_t kMaxBatchCount = 1 << 16;   // matrices one rpcholqr_factor_batched call may take
constexpr int32_t kMaxNF32 = 512;              // widest FP32 plan (the FP32 row solve stages T in shared memory)
constexpr int kTriuInvMaxN = 512;              // widest R1^{-1} of the warp-per-column kernel

struct rpcholqr_plan_s {
    int device = 0;
    rpcholqr_mode mode = RPCHOLQR_FP64;
    int64_t max_m = 0;
    int32_t max_n = 0, max_s = 0, np = 0;
    int grid = 0;  // CTAs of the row passes (one per SM)
    int nparts = 0;  // Gram partials in gpart (gram_parts)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double* As = nullptr;       // max_s x np, column-major
    double* Rs = nullptr;       // np x np
    double* R1 = nullptr;       // np x np
    double* G = nullptr;        // np x np
    double* frag_s = nullptr;   // np*np
    double* diag_s = nullptr;   // np/8*64
    double* frag_1 = nullptr;
    double* diag_1 = nullptr;
    double* gpart = nullptr;    // grid x np x np
    int32_t* info_ws = nullptr; // 2 ints (for step calls without a caller info)
    // staging for rpcholqr_factor_host
    double* hA = nullptr;
    double* hQ = nullptr;
    double* hR = nullptr;
    int32_t* hinfo = nullptr;
    size_t staged_elems = 0;
    // rpcholqr_factor_host's copy pipeline (SPLIT64): a copy stream, chunk events, the sample indices
    // (device and pinned host) and the sampled rows (pinned host and device)
    cudaStream_t hcopy = nullptr;
    cudaEvent_t hev[2 * 4] = {};     // 2 x kHostChunks
    int64_t* hidx_dev = nullptr;
    int64_t* hidx_host = nullptr;
    double* hrows_host = nullptr;
    double* hrows_dev = nullptr;
    // phase timing
    int32_t timing_slots = 0;
    int32_t timed_calls = 0;
    cudaEvent_t* events = nullptr;  // timing_slots x (RPCHOLQR_NUM_PHASES + 1)
    // per-launch timing of the timed calls: timing_slots x kMaxTimedLaunches event pairs, the class
    // and algorithmic FP64 flops of each launch, and the launches recorded per slot
    cudaEvent_t* kevents = nullptr;
    int8_t* kclass = nullptr;
    bool kuntimed = false;      // launches enqueued now are a gated-off branch: not counted in any class
    double* kflops = nullptr;
    int32_t* klaunches = nullptr;
    int32_t cur_slot = -1;          // the slot of the call being issued (-1: not timed)
    int64_t launches = 0;
    // autotuned launch parameters (rpcholqr_autotune, or loaded by rpcholqr_plan_create) and the
    // parameters of the call being issued
    std::vector<TuneEntry> tune_table;
    Tuning cur_tune;
    int cur_np = 0;             // padded width of the current call (select_tuning)
    bool tune_forced = false;   // rpcholqr_autotune is timing a candidate: cur_tune is not looked up
    // options (rpcholqr_plan_set_option)
    int64_t spin_limit = kDefaultSpinLimit;   // polls of a pipeline wait before TIMEOUT
    int32_t scale_sample = 1;                 // sample scaled by sqrt(m/s) (Remark r_exp)
    // rpcholqr_factor_batched's workspace (RPCHOLQR_OPT_BATCH_CAPACITY or the first batched call)
    void* batch_ws = nullptr;
    int32_t batch_capacity = 0;
    int batch_grid = 0;        // CTAs of the persistent kernel
    // SPLIT64 buffers (separate allocation)
    void* split_ws = nullptr;
    double* A1 = nullptr;       // max_m x np
    int32_t* xexp = nullptr;    // max_m
    int32_t* colexp = nullptr;  // np
    int32_t* yexp = nullptr;    // np
    uint8_t* yblocks = nullptr; // Ozaki column slices (K, N <= np)
    // stage images (np > 128; separate allocation img_ws), img_rows rows at a time: the wide first pass's
    // row slices of finished column blocks, then the Gram's column slices of A1, then pass 2's row slices
    // of A1; when they cover every row each pass is a single launch over all rows
    void* img_ws = nullptr;
    uint8_t* aimg = nullptr;
    int32_t* bexp = nullptr;    // per pair of 64-column blocks of the image, the row bounds of that pair
    int64_t img_rows = 0;
    int64_t img_rows_opt = 0;   // RPCHOLQR_OPT_IMAGE_ROWS (0: automatic)
    double* W = nullptr;        // np x np
    int32_t* gates = nullptr;   // split pass-2 gate words: {split status, pivot, fp64 status, pivot, used fp64}
    // FP32 buffers (separate allocation)
    float* T32 = nullptr;       // pad32(max_n)^2: R_s or R1 in FP32, identity-padded
    float* rinv32 = nullptr;    // pad32(max_n)
    // smoothing (allocated by rpcholqr_plan_set_smoothing)
    int32_t smoothing = 0;          // 0 none, 1 Walsh-Hadamard, 2 cosine
    int32_t smooth_capacity = 0;    // the largest kind the buffers below were sized for
    void* smooth_ws = nullptr;
    double* smooth_T = nullptr;     // transform buffer, 8-column blocks of m' rows (complex for the cosine)
    int64_t* smooth_idx = nullptr;  // max_s sample rows of F A
    int8_t* smooth_sgn = nullptr;   // max_m Rademacher signs (cosine transform)
};

namespace {

struct WsLayout {
    size_t As, Rs, R1, G, frag_s, diag_s, frag_1, diag_1, gpart, info, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Per-CTA (or per-row-range) Gram partials a plan holds: one per SM for panels up to 128 columns (the
// fused pass writes one per CTA) and in the FP32 mode; for wide panels (np x np doubles each) at most one
// per 1024 rows of max_m and at most 1 GiB of them.
int gram_parts(rpcholqr_mode mode, int64_t max_m, int32_t max_n, int grid) {
    const int64_t np = pad_np(max_n);
    if (np <= kMaxNP || mode == RPCHOLQR_FP32) return grid;
    int64_t parts = (max_m + 1023) / 1024;
    const int64_t cap = (int64_t{1} << 30) / (np * np * static_cast<int64_t>(sizeof(double)));
    if (parts > cap) parts = cap;
    if (parts > grid) parts = grid;
    return parts < 1 ? 1 : static_cast<int>(parts);
}

WsLayout ws_layout(int32_t max_n, int32_t max_s, int grid) {
    const size_t np = static_cast<size_t>(pad_np(max_n));
    WsLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L.As = take(sizeof(double) * static_cast<size_t>(max_s) * np);   // sample, s x np column-major
    L.Rs = take(sizeof(double) * np * np);
    L.R1 = take(sizeof(double) * np * np);
    L.G = take(sizeof(double) * np * np);
    L.frag_s = take(sizeof(double) * np * np);
    L.diag_s = take(sizeof(double) * (np / 8) * 64);
    L.frag_1 = take(sizeof(double) * np * np);
    L.diag_1 = take(sizeof(double) * (np / 8) * 64);
    L.gpart = take(sizeof(double) * static_cast<size_t>(grid) * np * np);
    L.info = take(sizeof(int32_t) * 2);
    L.total = off;
    return L;
}

int default_grid(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        sms = 152;
    return sms;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

rpcholqr_status check_launch() {
    return cudaGetLastError() == cudaSuccess ? RPCHOLQR_OK : RPCHOLQR_ERR_CUDA;
}

rpcholqr_status reset_info(int32_t* info, cudaStream_t st) {
    if (cudaMemsetAsync(info, 0, sizeof(int32_t), st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    if (cudaMemsetAsync(info + 1, 0xFF, sizeof(int32_t), st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    return RPCHOLQR_OK;
}

// The sample's scale sqrt(m/s) (Remark r_exp) unless the plan turned it off.
double sample_scale(const rpcholqr_plan_s* p, int64_t m, int32_t s) {
    return p->scale_sample ? std::sqrt(static_cast<double>(m) / static_cast<double>(s)) : 1.0;
}

bool shape_ok(const rpcholqr_plan_s* p, int64_t m, int32_t n, int32_t s) {
    return n >= 1 && n <= p->max_n && s >= n && s <= p->max_s && m >= s && m <= p->max_m;
}

// Records the start of `phase` (or the end of the call for phase == RPCHOLQR_NUM_PHASES) when
// the plan times this call.
constexpr int kMaxTimedLaunches = 1024;   // per timed call

struct PhaseMarks {
    rpcholqr_plan_s* p;
    cudaStream_t st;
    int slot;
    PhaseMarks(rpcholqr_plan_s* plan, cudaStream_t stream) : p(plan), st(stream), slot(-1) {
        if (p->events && p->timed_calls < p->timing_slots) slot = p->timed_calls++;
        p->cur_slot = slot;
        if (slot >= 0) p->klaunches[slot] = 0;
    }
    ~PhaseMarks() { p->cur_slot = -1; }
    void mark(int phase) const {
        if (slot >= 0) cudaEventRecord(p->events[slot * (RPCHOLQR_NUM_PHASES + 1) + phase], st);
    }
};

// Events around one launch of kernel class `cls` (rpcholqr_plan_collect_kernel_timing) when the current
// call is timed; `flops` = the launch's algorithmic FP64 flops.
struct KTimer {
    rpcholqr_plan_s* p;
    cudaStream_t st;
    int k = -1;
    KTimer(rpcholqr_plan_s* plan, cudaStream_t stream, int cls, double flops) : p(plan), st(stream) {
        const int slot = p->cur_slot;
        if (slot < 0 || !p->kevents || p->kuntimed || p->klaunches[slot] >= kMaxTimedLaunches) return;
        k = slot * kMaxTimedLaunches + p->klaunches[slot]++;
        p->kclass[k] = static_cast<int8_t>(cls);
        p->kflops[k] = flops;
        cudaEventRecord(p->kevents[2 * k], st);
    }
    ~KTimer() {
        if (k >= 0) cudaEventRecord(p->kevents[2 * k + 1], st);
    }
};

// The kernel class and algorithmic FP64 flops of a split product (launch_ozaki_gemm picks the kernel the
// same way): C = B - X Y with K <= 32 and N <= 128 runs k_ozaki_update, the other subtract forms and
// C = X Y k_ozaki_gemm_ws; an upper-triangular Y needs sum_j 2 min(j + 1, K) flops per row.
int ozaki_class(bool sub, int K, int N) {
    if (sub) return K <= 32 && N <= 128 ? RPCHOLQR_KERNEL_SPLIT_UPDATE : RPCHOLQR_KERNEL_SPLIT_GEMM_SUB;
    return RPCHOLQR_KERNEL_SPLIT_GEMM;
}
double ozaki_flops(bool sub, bool y_upper, int64_t m, int K, int N) {
    if (sub || !y_upper) return 2.0 * m * K * N;
    double per_row = 0.0;
    for (int j = 0; j < N; ++j) per_row += 2.0 * (j + 1 < K ? j + 1 : K);
    return per_row * m;
}

constexpr int kBlk = 64;   // column block of the FP64 blocked solves (n > 128)
// Blocks of the split mode's first pass: the FP64 row passes solve split_sub-column diagonal blocks
// (FP64 work per row n * split_sub); the rest of the solve runs as split tensor-core updates, K =
// kSplitBlk across blocks and K = split_sub inside one (n <= 128; wider, 64-column blocks).  At
// m = 2^20, n = 128, sub-blocks of 16 measured the same step time as 32 (13.75 vs 13.79 ms: the FP64
// work halves, the extra K = 16 updates cost as much), so up to 128 columns the blocks are not split; at
// m = 2^23, n = 512, 16 took the step from 558 to 540 ms (row passes 159 -> 96 ms, updates 32 -> 76 ms),
// so wider matrices take 16.
constexpr int kSplitBlk = 32;
constexpr int kSplitSub = 32;
constexpr int kSplitSubWide = 16;
// Split mode: the explicit-inverse second pass is used while ||R1||_F ||R1^{-1}||_F / n <= this
// (1.1-1.25 for well-sampled incoherent A; the estimate lies in [kappa(A1)/n, kappa(A1)]; at 3.3
// (kappa(A1) ~ 30) the explicit inverse already costs 10x in residual).
constexpr double kSplitPass2Tau = 2.0;

int ceil_log2(int64_t m) {
    int l = 0;
    while ((int64_t{1} << l) < m) ++l;
    return l;
}

// The launch parameters of a call on an m x n matrix: the plan's table entry of the same mode and padded
// width nearest in log2 m (none: the built-in rules).  Every public call that runs these kernels sets
// them first.
void select_tuning(rpcholqr_plan_s* p, int64_t m, int n) {
    p->cur_np = pad_np(n);
    if (p->tune_forced) return;
    Tuning t;
    const int np = pad_np(n), lm = ceil_log2(m);
    int best_d = 1 << 30;
    for (const TuneEntry& e : p->tune_table) {
        if (e.mode != p->mode || e.np != np) continue;
        const int d = e.m_log2 > lm ? e.m_log2 - lm : lm - e.m_log2;
        if (d < best_d) {
            best_d = d;
            t = e.t;
        }
    }
    p->cur_tune = t;
}

// Width of the SPLIT64 first pass's FP64 diagonal-block solves for the current call.
int split_sub(const rpcholqr_plan_s* p) {
    const int v = p->cur_tune.split_sub;
    return v == 16 || v == 32 ? v : (p->cur_np > kMaxNP ? kSplitSubWide : kSplitSub);
}

// CTAs of a row pass over m rows: one per 128-row panel, at most one per SM.
int row_grid(const rpcholqr_plan_s* p, int64_t m) {
    const int64_t panels = (m + 127) / 128;
    return static_cast<int>(panels < p->grid ? panels : p->grid);
}

// The smoothed sample of the plan's kind into p->As (column-major, ld s, np columns).
template <typename TA>
cudaError_t plan_smoothed_sample(rpcholqr_plan_s* p, const TA* A, int64_t m, int n, int64_t lda, int s,
                                 uint64_t seed, int np, int32_t* info, cudaStream_t st);
template <>
cudaError_t plan_smoothed_sample<double>(rpcholqr_plan_s* p, const double* A, int64_t m, int n, int64_t lda, int s,
                                         uint64_t seed, int np, int32_t* info, cudaStream_t st) {
    p->launches += 3;
    if (p->smoothing == 2)
        return launch_dct_sample(A, m, n, lda, s, seed, p->smooth_T, p->smooth_sgn, p->smooth_idx, p->As, s, np,
                                 info, st, p->scale_sample != 0);
    return launch_smoothed_sample(A, m, n, lda, s, seed, p->smooth_T, p->smooth_idx, p->As, s, np, info, st,
                                  p->scale_sample != 0);
}
template <>
cudaError_t plan_smoothed_sample<float>(rpcholqr_plan_s* p, const float* A, int64_t m, int n, int64_t lda, int s,
                                        uint64_t seed, int np, int32_t* info, cudaStream_t st) {
    p->launches += 3;
    if (p->smoothing == 2)
        return launch_dct_sample_f32(A, m, n, lda, s, seed, p->smooth_T, p->smooth_sgn, p->smooth_idx, p->As, s,
                                     np, info, st, p->scale_sample != 0);
    return launch_smoothed_sample_f32(A, m, n, lda, s, seed, p->smooth_T, p->smooth_idx, p->As, s, np, info, st,
                                      p->scale_sample != 0);
}

void free_events(rpcholqr_plan_s* p) {
    if (p->events)
        for (int i = 0; i < p->timing_slots * (RPCHOLQR_NUM_PHASES + 1); ++i) cudaEventDestroy(p->events[i]);
    if (p->kevents)
        for (int i = 0; i < 2 * p->timing_slots * kMaxTimedLaunches; ++i) cudaEventDestroy(p->kevents[i]);
    delete[] p->events;
    delete[] p->kevents;
    delete[] p->kclass;
    delete[] p->kflops;
    delete[] p->klaunches;
    p->events = nullptr;
    p->kevents = nullptr;
    p->kclass = nullptr;
    p->kflops = nullptr;
    p->klaunches = nullptr;
    p->timing_slots = 0;
    p->timed_calls = 0;
    p->cur_slot = -1;
}

const char* mode_name(int32_t mode) {
    return mode == RPCHOLQR_SPLIT64 ? "split" : mode == RPCHOLQR_FP32 ? "fp32" : "fp64";
}

// The tuning table as JSON: {"gpu": ..., "sms": ..., "entries": [{"mode": ..., "np": ..., "m_log2": ...,
// "split_sub": ..., "gram_ranges": ..., "syrk_ranges": ..., "ms": ...}, ...]}.
std::string tune_json(const rpcholqr_plan_s* p) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) {
        cudaGetLastError();
        prop.name[0] = 0;
    }
    std::string out = "{\n  \"gpu\": \"" + std::string(prop.name) + "\",\n  \"sms\": " + std::to_string(p->grid) +
                      ",\n  \"entries\": [";
    for (size_t i = 0; i < p->tune_table.size(); ++i) {
        const TuneEntry& e = p->tune_table[i];
        char buf[320];
        std::snprintf(buf, sizeof buf,
                      "%s\n    {\"mode\": \"%s\", \"np\": %d, \"m_log2\": %d, \"split_sub\": %d, "
                      "\"gram_ranges\": %d, \"syrk_ranges\": %d, \"ms\": %.4f}",
                      i ? "," : "", mode_name(e.mode), e.np, e.m_log2, e.t.split_sub, e.t.gram_ranges,
                      e.t.syrk_ranges, e.ms);
        out += buf;
    }
    out += "\n  ]\n}\n";
    return out;
}

// Reads the "entries" of a tuning table written by tune_json (whitespace and key order free; other keys
// ignored).  False on malformed text.
bool parse_tune_json(const char* text, std::vector<TuneEntry>& out) {
    const char* q = std::strstr(text, "\"entries\"");
    if (!q) return false;
    q = std::strchr(q, '[');
    if (!q) return false;
    ++q;
    for (;;) {
        while (*q == ' ' || *q == '\n' || *q == '\r' || *q == '\t' || *q == ',') ++q;
        if (*q == ']') return true;
        if (*q != '{') return false;
        const char* end = std::strchr(q, '}');
        if (!end) return false;
        const std::string obj(q + 1, end);
        TuneEntry e;
        bool have_mode = false, have_np = false, have_m = false;
        size_t pos = 0;
        while ((pos = obj.find('"', pos)) != std::string::npos) {
            const size_t kend = obj.find('"', pos + 1);
            if (kend == std::string::npos) return false;
            const std::string key = obj.substr(pos + 1, kend - pos - 1);
            size_t v = obj.find(':', kend);
            if (v == std::string::npos) return false;
            ++v;
            while (v < obj.size() && (obj[v] == ' ' || obj[v] == '\n' || obj[v] == '\t')) ++v;
            if (v < obj.size() && obj[v] == '"') {
                const size_t vend = obj.find('"', v + 1);
                if (vend == std::string::npos) return false;
                const std::string val = obj.substr(v + 1, vend - v - 1);
                if (key == "mode") {
                    if (val == "fp64") e.mode = RPCHOLQR_FP64;
                    else if (val == "split") e.mode = RPCHOLQR_SPLIT64;
                    else if (val == "fp32") e.mode = RPCHOLQR_FP32;
                    else return false;
                    have_mode = true;
                }
                pos = vend + 1;
            } else {
                char* after = nullptr;
                const double num = std::strtod(obj.c_str() + v, &after);
                if (after == obj.c_str() + v) return false;
                const int iv = static_cast<int>(num);
                if (key == "np") { e.np = iv; have_np = true; }
                else if (key == "m_log2") { e.m_log2 = iv; have_m = true; }
                else if (key == "split_sub") e.t.split_sub = iv;
                else if (key == "gram_ranges") e.t.gram_ranges = iv;
                else if (key == "syrk_ranges") e.t.syrk_ranges = iv;
                else if (key == "ms") e.ms = num;
                pos = static_cast<size_t>(after - obj.c_str());
            }
        }
        if (!have_mode || !have_np || !have_m || e.np < 1 || e.m_log2 < 0 || e.m_log2 > 62 ||
            e.t.split_sub < 0 || e.t.gram_ranges < 0 || e.t.syrk_ranges < 0)
            return false;
        out.push_back(e);
        q = end + 1;
    }
}

// The table from JSON text (starting with '{') or from the file it names.
bool load_tune_json(const char* json_or_path, std::vector<TuneEntry>& out) {
    const char* t = json_or_path;
    while (*t == ' ' || *t == '\n' || *t == '\t' || *t == '\r') ++t;
    if (*t == '{') return parse_tune_json(t, out);
    FILE* f = std::fopen(json_or_path, "rb");
    if (!f) return false;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
    std::fclose(f);
    return parse_tune_json(text.c_str(), out);
}

void put_tune_entry(rpcholqr_plan_s* p, const TuneEntry& e) {
    for (TuneEntry& x : p->tune_table)
        if (x.mode == e.mode && x.np == e.np && x.m_log2 == e.m_log2) {
            x = e;
            return;
        }
    p->tune_table.push_back(e);
}

}  // namespace

extern "C" {

const char* rpcholqr_status_string(int status) {
    switch (status) {
        case RPCHOLQR_OK: return "RPCHOLQR_OK";
        case RPCHOLQR_ERR_ARG: return "RPCHOLQR_ERR_ARG";
        case RPCHOLQR_ERR_NONFINITE: return "RPCHOLQR_ERR_NONFINITE";
        case RPCHOLQR_ERR_SINGULAR_SKETCH: return "RPCHOLQR_ERR_SINGULAR_SKETCH";
        case RPCHOLQR_ERR_NOT_SPD: return "RPCHOLQR_ERR_NOT_SPD";
        case RPCHOLQR_ERR_TIMEOUT: return "RPCHOLQR_ERR_TIMEOUT";
        case RPCHOLQR_ERR_CUDA: return "RPCHOLQR_ERR_CUDA";
        case RPCHOLQR_ERR_NOMEM: return "RPCHOLQR_ERR_NOMEM";
        case RPCHOLQR_ERR_UNSUPPORTED: return "RPCHOLQR_ERR_UNSUPPORTED";
        default: return "RPCHOLQR_UNKNOWN_STATUS";
    }
}

// ---- stage images of the wide split passes (np > 128) ---------------------------------------------------
// Rows of one chunk of images when they cannot cover every row: 8 GiB of images.
int64_t image_chunk_rows(int np) {
    int64_t rows = (int64_t{1} << 33) / static_cast<int64_t>(np * 16) / 128 * 128;
    return rows < 128 ? 128 : rows;
}
int image_cols(int np) { return (np + 127) / 128 * 128; }
// Image rows a plan takes: `request` rows (rounded up to 128), or automatically every row when their images
// take at most a quarter of the device's memory (2^23 x 512: 69 GB of the GB300's 288 GB; each wide pass is
// then one launch per step instead of one per chunk), else one chunk.
int64_t image_rows(int device, int64_t max_m, int np, int64_t request) {
    const int64_t all = (max_m + 127) / 128 * 128;
    if (request > 0) {
        const int64_t r = (request + 127) / 128 * 128;
        return r < all ? r : all;
    }
    size_t total = 0;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) total = prop.totalGlobalMem;
    else cudaGetLastError();
    const size_t full = ozaki_image_bytes(all, image_cols(np));
    if (total > 0 && full <= total / 4) return all;
    const int64_t chunk = image_chunk_rows(np);
    return chunk < all ? chunk : all;
}
// Bytes of the image buffers for `rows` image rows: the images and the row bounds of each pair of blocks.
size_t image_bytes(int np, int64_t rows) {
    return align256(ozaki_image_bytes(rows, image_cols(np))) +
           align256(sizeof(int32_t) * static_cast<size_t>(rows) * ((np + kBlk - 1) / kBlk));
}

rpcholqr_status rpcholqr_workspace_size(rpcholqr_plan p, int64_t max_m, int32_t max_n, int32_t max_s,
                                        size_t* bytes) {
    if (!bytes || max_n < 1 || max_n > RPCHOLQR_MAX_N || max_s < max_n || max_m < max_s)
        return RPCHOLQR_ERR_ARG;
    const rpcholqr_mode mode = p ? p->mode : RPCHOLQR_FP64;
    const int grid = p ? p->grid : 152;
    const int32_t ws_n = mode == RPCHOLQR_FP32 ? (max_n + 63) / 64 * 64 : max_n;
    size_t total = ws_layout(ws_n, max_s, gram_parts(mode, max_m, max_n, grid)).total;
    const size_t np = static_cast<size_t>(pad_np(max_n));
    if (mode == RPCHOLQR_SPLIT64)   // A1, row/column bounds, column slices, R1^{-1}, gate words
        total += align256(sizeof(double) * static_cast<size_t>(max_m) * np) +
                 align256(sizeof(int32_t) * static_cast<size_t>(max_m)) + 2 * align256(sizeof(int32_t) * np) +
                 align256(ozaki_yblocks_bytes(static_cast<int>(np), static_cast<int>(np))) +
                 align256(sizeof(double) * np * np) + align256(sizeof(int32_t) * 8);
    if (mode == RPCHOLQR_SPLIT64 && np > static_cast<size_t>(kMaxNP)) {   // stage images
        int device = 0;
        if (p) device = p->device;
        else if (cudaGetDevice(&device) != cudaSuccess) cudaGetLastError();
        const int64_t rows = image_rows(device, max_m, static_cast<int>(np), p ? p->img_rows_opt : 0);
        total += image_bytes(static_cast<int>(np), rows);
    }
    if (mode == RPCHOLQR_FP32) {
        const size_t n32 = static_cast<size_t>(f32_pad(max_n));
        total += align256(sizeof(float) * n32 * n32) + sizeof(float) * n32;
    }
    *bytes = total;
    return RPCHOLQR_OK;
}

// (Re)allocates the stage images for `request` rows (0: automatic, see image_rows; if every row does not
// fit, one chunk).  The new buffer is allocated before the old one is freed: when it cannot be had the
// plan keeps its images as they were and RPCHOLQR_ERR_NOMEM is returned.
static rpcholqr_status alloc_images(rpcholqr_plan_s* p, int64_t request) {
    const int64_t all = (p->max_m + 127) / 128 * 128;
    int64_t rows = image_rows(p->device, p->max_m, p->np, request);
    void* buf = nullptr;
    for (int attempt = 0; attempt < 2 && !buf; ++attempt) {
        if (cudaMalloc(&buf, image_bytes(p->np, rows)) == cudaSuccess) break;
        cudaGetLastError();
        buf = nullptr;
        if (request > 0 || rows < all) break;
        rows = image_chunk_rows(p->np) < all ? image_chunk_rows(p->np) : all;   // every row did not fit
        if (rows >= all) break;
    }
    if (!buf) return RPCHOLQR_ERR_NOMEM;
    if (p->img_ws) {
        cudaFree(p->img_ws);
        p->ws_bytes -= image_bytes(p->np, p->img_rows);
    }
    p->img_ws = buf;
    char* c = static_cast<char*>(buf);
    p->aimg = reinterpret_cast<uint8_t*>(c);
    p->bexp = reinterpret_cast<int32_t*>(c + align256(ozaki_image_bytes(rows, image_cols(p->np))));
    p->img_rows = rows;
    p->ws_bytes += image_bytes(p->np, rows);
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_plan_create(rpcholqr_plan* plan, int device, rpcholqr_mode mode,
                                     int64_t max_m, int32_t max_n, int32_t max_s, const char* autotune_json) {
    if (!plan) return RPCHOLQR_ERR_ARG;
    *plan = nullptr;
    std::vector<TuneEntry> table;
    if (autotune_json && !load_tune_json(autotune_json, table)) return RPCHOLQR_ERR_ARG;
    if (max_n < 1 || max_n > RPCHOLQR_MAX_N || max_s < max_n || max_m < max_s) return RPCHOLQR_ERR_ARG;
    if (mode != RPCHOLQR_FP64 && mode != RPCHOLQR_SPLIT64 && mode != RPCHOLQR_FP32) return RPCHOLQR_ERR_UNSUPPORTED;
    if (mode == RPCHOLQR_FP32 && max_n > kMaxNF32) return RPCHOLQR_ERR_UNSUPPORTED;
    if (householder_smem_bytes(max_s, max_n) > 200 * 1024) return RPCHOLQR_ERR_UNSUPPORTED;
    DeviceGuard guard(device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    auto* p = new (std::nothrow) rpcholqr_plan_s();
    if (!p) return RPCHOLQR_ERR_NOMEM;
    p->device = device;
    p->mode = mode;
    p->max_m = max_m;
    p->max_n = max_n;
    p->max_s = max_s;
    p->np = pad_np(max_n);
    p->grid = default_grid(device);
    p->tune_table = table;
    // the FP32 Gram works on 64 x 64 tiles: size the shared FP64 buffers for max_n rounded up to 64
    const int32_t ws_n = mode == RPCHOLQR_FP32 ? (max_n + 63) / 64 * 64 : max_n;
    p->nparts = gram_parts(mode, max_m, max_n, p->grid);
    const WsLayout L = ws_layout(ws_n, max_s, p->nparts);
    if (cudaMalloc(&p->ws, L.total) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return RPCHOLQR_ERR_NOMEM;
    }
    p->ws_bytes = L.total;
    char* b = static_cast<char*>(p->ws);
    p->As = reinterpret_cast<double*>(b + L.As);
    p->Rs = reinterpret_cast<double*>(b + L.Rs);
    p->R1 = reinterpret_cast<double*>(b + L.R1);
    p->G = reinterpret_cast<double*>(b + L.G);
    p->frag_s = reinterpret_cast<double*>(b + L.frag_s);
    p->diag_s = reinterpret_cast<double*>(b + L.diag_s);
    p->frag_1 = reinterpret_cast<double*>(b + L.frag_1);
    p->diag_1 = reinterpret_cast<double*>(b + L.diag_1);
    p->gpart = reinterpret_cast<double*>(b + L.gpart);
    p->info_ws = reinterpret_cast<int32_t*>(b + L.info);
    if (mode == RPCHOLQR_SPLIT64) {
        const size_t np = static_cast<size_t>(p->np);
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
        const size_t oA1 = take(sizeof(double) * static_cast<size_t>(max_m) * np);
        const size_t oX = take(sizeof(int32_t) * static_cast<size_t>(max_m));
        const size_t oC = take(sizeof(int32_t) * np);
        const size_t oY = take(sizeof(int32_t) * np);
        const size_t oB = take(ozaki_yblocks_bytes(p->np, p->np));
        const size_t oW = take(sizeof(double) * np * np);
        const size_t oG = take(sizeof(int32_t) * 8);
        if (cudaMalloc(&p->split_ws, off) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(p->ws);
            delete p;
            return RPCHOLQR_ERR_NOMEM;
        }
        char* c = static_cast<char*>(p->split_ws);
        p->A1 = reinterpret_cast<double*>(c + oA1);
        p->xexp = reinterpret_cast<int32_t*>(c + oX);
        p->colexp = reinterpret_cast<int32_t*>(c + oC);
        p->yexp = reinterpret_cast<int32_t*>(c + oY);
        p->yblocks = reinterpret_cast<uint8_t*>(c + oB);
        p->W = reinterpret_cast<double*>(c + oW);
        p->gates = reinterpret_cast<int32_t*>(c + oG);
        if (cudaMemset(p->gates, 0, sizeof(int32_t) * 8) != cudaSuccess) cudaGetLastError();
        p->ws_bytes += off;
        if (np > static_cast<size_t>(kMaxNP) && alloc_images(p, 0) != RPCHOLQR_OK) {
            cudaFree(p->split_ws);
            cudaFree(p->ws);
            delete p;
            return RPCHOLQR_ERR_NOMEM;
        }
    }
    if (mode == RPCHOLQR_FP32) {
        const size_t n32 = static_cast<size_t>(f32_pad(max_n));
        const size_t oT = 0, oR = align256(sizeof(float) * n32 * n32);
        const size_t total = oR + sizeof(float) * n32;
        if (cudaMalloc(&p->split_ws, total) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(p->ws);
            delete p;
            return RPCHOLQR_ERR_NOMEM;
        }
        char* c = static_cast<char*>(p->split_ws);
        p->T32 = reinterpret_cast<float*>(c + oT);
        p->rinv32 = reinterpret_cast<float*>(c + oR);
        p->ws_bytes += total;
    }
    *plan = p;
    return RPCHOLQR_OK;
}

// (Re)allocates the persistent batched kernel's workspace for up to `capacity` matrices (0 frees it).
static rpcholqr_status reserve_batch(rpcholqr_plan_s* p, int32_t capacity) {
    if (capacity == p->batch_capacity) return RPCHOLQR_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    if (p->batch_ws) {
        if (cudaDeviceSynchronize() != cudaSuccess) return RPCHOLQR_ERR_CUDA;
        cudaFree(p->batch_ws);
        p->batch_ws = nullptr;
        p->batch_capacity = 0;
    }
    if (capacity == 0) return RPCHOLQR_OK;
    if (prepare_batch_persistent(p->max_n, p->max_s, p->grid, &p->batch_grid) != cudaSuccess) {
        cudaGetLastError();
        return RPCHOLQR_ERR_CUDA;
    }
    const BatchLayout L = batch_layout(capacity, p->max_n, p->max_s, p->grid);
    if (cudaMalloc(&p->batch_ws, L.total) != cudaSuccess) {
        cudaGetLastError();
        p->batch_ws = nullptr;
        return RPCHOLQR_ERR_NOMEM;
    }
    p->batch_capacity = capacity;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_plan_set_option(rpcholqr_plan p, int32_t option, int64_t value) {
    if (!p) return RPCHOLQR_ERR_ARG;
    switch (option) {
        case RPCHOLQR_OPT_SPIN_LIMIT:
            if (value < 1 || value > (int64_t{1} << 40)) return RPCHOLQR_ERR_ARG;
            p->spin_limit = value;
            return RPCHOLQR_OK;
        case RPCHOLQR_OPT_SCALE_SAMPLE:
            if (value != 0 && value != 1) return RPCHOLQR_ERR_ARG;
            p->scale_sample = static_cast<int32_t>(value);
            return RPCHOLQR_OK;
        case RPCHOLQR_OPT_DETERMINISTIC:
            // every reduction is a fixed-order sum; no run-to-run varying variant is built
            if (value == 1) return RPCHOLQR_OK;
            return value == 0 ? RPCHOLQR_ERR_UNSUPPORTED : RPCHOLQR_ERR_ARG;
        case RPCHOLQR_OPT_BATCH_CAPACITY:
            if (value < 0 || value > kMaxBatchCount) return RPCHOLQR_ERR_ARG;
            return reserve_batch(p, static_cast<int32_t>(value));
        case RPCHOLQR_OPT_IMAGE_ROWS: {
            if (value < 0) return RPCHOLQR_ERR_ARG;
            if (p->mode != RPCHOLQR_SPLIT64 || p->np <= kMaxNP) return RPCHOLQR_ERR_UNSUPPORTED;
            DeviceGuard guard(p->device);
            if (!guard.ok) return RPCHOLQR_ERR_CUDA;
            if (cudaDeviceSynchronize() != cudaSuccess) return RPCHOLQR_ERR_CUDA;   // no call still reads them
            const rpcholqr_status rc = alloc_images(p, value);
            if (rc == RPCHOLQR_OK) p->img_rows_opt = value;
            return rc;
        }
        default: return RPCHOLQR_ERR_ARG;
    }
}

rpcholqr_status rpcholqr_plan_get_option(rpcholqr_plan p, int32_t option, int64_t* value) {
    if (!p || !value) return RPCHOLQR_ERR_ARG;
    switch (option) {
        case RPCHOLQR_OPT_SPIN_LIMIT: *value = p->spin_limit; return RPCHOLQR_OK;
        case RPCHOLQR_OPT_SCALE_SAMPLE: *value = p->scale_sample; return RPCHOLQR_OK;
        case RPCHOLQR_OPT_DETERMINISTIC: *value = 1; return RPCHOLQR_OK;
        case RPCHOLQR_OPT_BATCH_CAPACITY: *value = p->batch_capacity; return RPCHOLQR_OK;
        case RPCHOLQR_OPT_IMAGE_ROWS: *value = p->img_rows; return RPCHOLQR_OK;
        default: return RPCHOLQR_ERR_ARG;
    }
}

rpcholqr_status rpcholqr_plan_destroy(rpcholqr_plan plan) {
    if (!plan) return RPCHOLQR_OK;
    DeviceGuard guard(plan->device);
    cudaDeviceSynchronize();
    cudaFree(plan->ws);
    cudaFree(plan->hA);
    cudaFree(plan->hQ);
    cudaFree(plan->hR);
    cudaFree(plan->hinfo);
    if (plan->hcopy) cudaStreamDestroy(plan->hcopy);
    for (cudaEvent_t e : plan->hev)
        if (e) cudaEventDestroy(e);
    cudaFree(plan->hidx_dev);
    cudaFreeHost(plan->hidx_host);
    cudaFreeHost(plan->hrows_host);
    cudaFree(plan->hrows_dev);
    cudaFree(plan->split_ws);
    cudaFree(plan->img_ws);
    cudaFree(plan->smooth_ws);
    cudaFree(plan->batch_ws);
    free_events(plan);
    delete plan;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_sample_indices(uint64_t seed, uint64_t stream_id, int64_t m, int32_t s,
                                        int64_t* idx, void* stream) {
    if (!idx || m < 1 || s < 1) return RPCHOLQR_ERR_ARG;
    launch_sample_indices(seed, stream_id, m, s, idx, static_cast<cudaStream_t>(stream));
    return check_launch();
}

static rpcholqr_status sketch_internal(rpcholqr_plan p, const double* A, int64_t m, int32_t n,
                                       int64_t lda, int32_t s, uint64_t seed, uint64_t stream_id,
                                       double* Rs_user, int32_t* info, cudaStream_t st,
                                       const PhaseMarks* pm) {
    const int np = pad_np(n);
    const double scale = sample_scale(p, m, s);
    if (pm) pm->mark(RPCHOLQR_PHASE_SAMPLE);
    const int64_t lds = s;
    if (p->smoothing) {
        if (plan_smoothed_sample<double>(p, A, m, n, lda, s, seed, np, info, st) != cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    } else {
        launch_sample_gather(A, m, n, lda, s, seed, stream_id, scale, p->As, lds, np, nullptr, info, st);
        ++p->launches;
    }
    if (check_launch() != RPCHOLQR_OK) return RPCHOLQR_ERR_CUDA;
    if (pm) pm->mark(RPCHOLQR_PHASE_SKETCH_QR);
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_SKETCH_QR, 2.0 * s * n * n - 2.0 * n * n * n / 3.0);
        if (launch_householder(p->As, lds, s, n, np, p->Rs, Rs_user, info, st) != cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    }
    ++p->launches;
    return RPCHOLQR_OK;
}

static rpcholqr_status ozaki_gemm_internal(rpcholqr_plan p, bool sub, const double* X, int64_t m, int K,
                                           int64_t ldx, const double* Y, int N, int64_t ldy, const double* B,
                                           int64_t ldb, double* C, int64_t ldc, int32_t* info, cudaStream_t st,
                                           bool xexp_ready = false, int64_t row0 = 0, bool y_ready = false,
                                           bool y_upper = false, const uint8_t* aimg = nullptr, int img_nkw = 0,
                                           const int32_t* bexp = nullptr, int64_t ld_bexp = 0);

// Diagonal-block setups for the blocked solve with T (n x n, ld ldt): block J (64 columns, the last
// one ragged) gets frag + 4096 J and diag + 512 J.
static void prep_blocks(rpcholqr_plan_s* p, const double* T, int64_t ldt, int n, double* frag, double* diag,
                        const int32_t* info, cudaStream_t st, int blk = kBlk) {
    for (int J = 0; J * blk < n; ++J) {
        const int nj = n - J * blk < blk ? n - J * blk : blk;
        launch_prep_tri(T + static_cast<int64_t>(J) * blk * ldt + J * blk, ldt, nj, pad16(nj),
                        frag + J * blk * blk, diag + J * (blk / 8) * 64, info, st);
        ++p->launches;
    }
}

// Right-looking blocked row solve for the split mode, Y = X T^{-1}, two-level: over kSplitBlk-column
// blocks J, each solved as two kSplitSub-column halves.  A half is solved by the FP64 row pass,
// Y[:, h] <- (current X[:, h]) T[h, h]^{-1}; after the first half, the second half is updated by one
// split tensor-core product with K = N = kSplitSub; after the block, every later column is updated at
// once, Y[:, >J] = (X or Y)[:, >J] - Y[:, J] T[J, >J], by one split product with K = kSplitBlk (one
// exactness stage) and N = the remaining width.  The FP64 work per row is n * kSplitSub.  The diagonal
// blocks must have been set up by prep_blocks with blk = kSplitSub.  The row passes store (first half)
// and max-merge the row bounds of Y into p->xexp (the updates' left operands use the bound over the
// columns solved so far) and their column bounds into p->colexp.  Marks PASS1 / PASS1_UPDATE /
// PASS1_SOLVE2 as the first row pass / the first update / the rest when pm is given.  row0: X's first
// row within the matrix whose row bounds p->xexp holds (a block of rows is solved on its own).
static rpcholqr_status solve_split_right(rpcholqr_plan_s* p, const double* X, int64_t ldx, const double* T,
                                         int64_t ldt, int64_t m, int n, double* Y, int64_t ldy, const double* frag,
                                         const double* diag, int32_t* info, cudaStream_t st, const PhaseMarks* pm,
                                         int64_t row0 = 0) {
    const int grid = row_grid(p, m);
    const int blk = kSplitBlk, sub = split_sub(p);
    bool first_update = true;
    auto update = [&](int c0, int K, int c1, int N, const double* B, int64_t ldb) -> rpcholqr_status {
        if (pm && first_update) pm->mark(RPCHOLQR_PHASE_PASS1_UPDATE);
        rpcholqr_status rc = ozaki_gemm_internal(p, true, Y + c0, m, K, ldy, T + static_cast<int64_t>(c0) * ldt + c1,
                                                 N, ldt, B, ldb, Y + c1, ldy, info, st, true, row0);
        if (pm && first_update) pm->mark(RPCHOLQR_PHASE_PASS1_SOLVE2);
        first_update = false;
        return rc;
    };
    for (int J = 0; J * blk < n; ++J) {
        const int c0 = J * blk;
        const int nj = n - c0 < blk ? n - c0 : blk;
        for (int h = 0; h * sub < nj; ++h) {
            const int c1 = c0 + h * sub;
            const int nh = nj - h * sub < sub ? nj - h * sub : sub;
            // column c1 still holds A only in the very first half; later ones were written by an update
            const double* src = c1 == 0 ? X : Y;
            const int64_t lsrc = c1 == 0 ? ldx : ldy;
            const int js = c1 / sub;
            {
                KTimer kt(p, st, RPCHOLQR_KERNEL_ROWPASS, static_cast<double>(m) * nh * nh);
                if (launch_rowpass_ex(false, pad16(nh), src + c1, lsrc, Y + c1, ldy, m, nh, frag + js * sub * sub,
                                      diag + js * (sub / 8) * 64, nullptr, info, grid, st, true, p->xexp + row0,
                                      c1 == 0 ? 1 : 2, p->colexp + c1) != cudaSuccess)
                    return RPCHOLQR_ERR_CUDA;
            }
            ++p->launches;
            if (h == 0 && nj > nh) {
                const rpcholqr_status rc = update(c1, nh, c1 + nh, nj - nh, (J == 0 ? X : Y) + c1 + nh,
                                                  J == 0 ? ldx : ldy);
                if (rc != RPCHOLQR_OK) return rc;
            }
        }
        const int rest = n - c0 - nj;
        if (rest > 0) {
            const rpcholqr_status rc = update(c0, nj, c0 + nj, rest, (J == 0 ? X : Y) + c0 + nj, J == 0 ? ldx : ldy);
            if (rc != RPCHOLQR_OK) return rc;
        }
    }
    if (pm && first_update) {
        pm->mark(RPCHOLQR_PHASE_PASS1_UPDATE);
        pm->mark(RPCHOLQR_PHASE_PASS1_SOLVE2);
    }
    return check_launch();
}

// The SPLIT64 first pass above 128 columns, Y = X T^{-1} (T = R_s upper triangular), left-looking over
// 64-column blocks, one row chunk (p->img_rows rows) at a time so that the chunk's stage image holds the
// slices of every finished block: block J of a chunk is first Y[:, J] = X[:, J] - Y[:, <J] T[<J, J], one
// split product over the image of blocks < J (each pair of blocks one exactness window, sliced against
// the row's bound over that pair alone), then its sub-block FP64 row passes joined by K = sub split
// updates (as in solve_blocked), and the finished block is sliced into the image (an odd block together
// with its even partner, which was sliced alone before).  The row passes max-merge
// the bounds of the whole row into p->xexp (pass 2 slices against them) and of each column into
// p->colexp.  Marks PASS1_UPDATE / PASS1_SOLVE2 around the first chunk's first product.
static rpcholqr_status solve_split_wide(rpcholqr_plan_s* p, const double* X, int64_t ldx, const double* T,
                                        int64_t ldt, int64_t m, int n, double* Y, int64_t ldy, const double* frag,
                                        const double* diag, int32_t* info, cudaStream_t st, const PhaseMarks* pm) {
    const int img_nkw = (n + 31) / 32;
    const int sub = split_sub(p);
    bool marked = false;
    for (int64_t r0 = 0; r0 < m; r0 += p->img_rows) {
        const int64_t rows = m - r0 < p->img_rows ? m - r0 : p->img_rows;
        const int grid = row_grid(p, rows);
        const double* Xc = X + r0 * ldx;
        double* Yc = Y + r0 * ldy;
        for (int J = 0; J * kBlk < n; ++J) {
            const int c0 = J * kBlk;
            const int nj = n - c0 < kBlk ? n - c0 : kBlk;
            if (J > 0) {
                const bool mark = pm && !marked;
                if (mark) pm->mark(RPCHOLQR_PHASE_PASS1_UPDATE);
                rpcholqr_status rc = ozaki_gemm_internal(p, true, Yc, rows, c0, ldy, T + c0, nj, ldt, Xc + c0, ldx,
                                                         Yc + c0, ldy, info, st, true, r0, false, false, p->aimg,
                                                         img_nkw, p->bexp, p->img_rows);
                if (rc != RPCHOLQR_OK) return rc;
                if (mark) {
                    pm->mark(RPCHOLQR_PHASE_PASS1_SOLVE2);
                    marked = true;
                }
            }
            for (int h = 0; h * sub < nj; ++h) {
                const int c1 = c0 + h * sub;
                const int nh = nj - h * sub < sub ? nj - h * sub : sub;
                const bool from_input = J == 0 && h == 0;
                const double* hsrc = (from_input ? Xc : Yc) + c1;
                const int64_t lh = from_input ? ldx : ldy;
                const int js = c1 / sub;
                {
                    KTimer kt(p, st, RPCHOLQR_KERNEL_ROWPASS, static_cast<double>(rows) * nh * nh);
                    if (launch_rowpass_ex(false, pad16(nh), hsrc, lh, Yc + c1, ldy, rows, nh, frag + js * sub * sub,
                                          diag + js * (sub / 8) * 64, nullptr, info, grid, st, true, p->xexp + r0,
                                          c1 == 0 ? 1 : 2, p->colexp + c1) != cudaSuccess)
                        return RPCHOLQR_ERR_CUDA;
                }
                ++p->launches;
                const int rest = c0 + nj - (c1 + nh);
                if (rest > 0) {
                    // the block's first sub-block update reads its input columns (X for block 0, else the
                    // product's output in Y), later ones the updated columns
                    const double* B = (from_input ? Xc : Yc) + c1 + nh;
                    const int64_t ldb = from_input ? ldx : ldy;
                    rpcholqr_status rc = ozaki_gemm_internal(p, true, Yc + c1, rows, nh, ldy,
                                                             T + static_cast<int64_t>(c1) * ldt + c1 + nh, rest, ldt,
                                                             B, ldb, Yc + c1 + nh, ldy, info, st, true, r0);
                    if (rc != RPCHOLQR_OK) return rc;
                }
            }
            if (c0 + nj < n) {
                // the products' exactness windows are pairs of blocks (K = 128) with their own row bound: an
                // even block is sliced alone (the last window of block J + 1's update), an odd one re-slices
                // its pair
                const int g0 = (J & 1) ? c0 - kBlk : c0;
                launch_slice_block_images(Yc + g0, ldy, rows, c0 + nj - g0, p->aimg, img_nkw, g0 / 32,
                                          p->bexp + static_cast<int64_t>(J >> 1) * p->img_rows, info, st);
                ++p->launches;
            }
        }
    }
    return check_launch();
}

// Left-looking blocked row solve Y = X T^{-1} (T upper triangular, n x n, ld ldt) over 64-column
// blocks J:  Y[:, J] = X[:, J] - Y[:, <J] T[<J, J]  (FP64 mma, or the split tensor-core product when
// split), then Y[:, J] <- Y[:, J] T[J, J]^{-1} by the row pass (NP = 64; split: two 32-column row
// passes and a K = 32 split update between them, so the FP64 work per row is n * 32).  Y may equal X
// (ldy == ldx).  The diagonal blocks must have been set up by prep_blocks (split: with blk =
// kSplitSub).  split: the row passes store (block 0) and
// max-merge (later blocks) the row bounds of Y into p->xexp and max-merge its column bounds into
// p->colexp, both needed by the split products; marks PASS1 / PASS1_UPDATE / PASS1_SOLVE2 when
// pass1_marks (blocks 2.. fall in PASS1_SOLVE2).
static rpcholqr_status solve_blocked(rpcholqr_plan_s* p, const double* X, int64_t ldx, const double* T, int64_t ldt,
                              int64_t m, int n, double* Y, int64_t ldy, const double* frag, const double* diag,
                              bool split, bool check_finite, int32_t* info, cudaStream_t st,
                              const PhaseMarks* pm, bool pass1_marks) {
    const int grid = row_grid(p, m);
    for (int J = 0; J * kBlk < n; ++J) {
        const int c0 = J * kBlk;
        const int nj = n - c0 < kBlk ? n - c0 : kBlk;
        const double* src = X + c0;
        int64_t lsrc = ldx;
        if (J > 0) {
            if (pm && pass1_marks && J == 1) pm->mark(RPCHOLQR_PHASE_PASS1_UPDATE);
            if (split) {
                rpcholqr_status rc = ozaki_gemm_internal(p, true, Y, m, c0, ldy, T + c0, nj, ldt, X + c0, ldx,
                                                         Y + c0, ldy, info, st, true);
                if (rc != RPCHOLQR_OK) return rc;
            } else {
                {
                    KTimer kt(p, st, RPCHOLQR_KERNEL_FP64_GEMM, 2.0 * m * c0 * nj);
                    if (launch_gemm_sub_fp64(Y, ldy, T + c0, ldt, X + c0, ldx, Y + c0, ldy, m, c0, nj, info,
                                             2 * p->grid, st) != cudaSuccess)
                        return RPCHOLQR_ERR_CUDA;
                }
                ++p->launches;
            }
            src = Y + c0;
            lsrc = ldy;
            if (pm && pass1_marks && J == 1) pm->mark(RPCHOLQR_PHASE_PASS1_SOLVE2);
        }
        if (split) {
            // sub-column FP64 solves (sub = the call's diagonal-block width, 16 or 32), each followed by
            // one K = sub split update of the block's remaining columns (diagonal tables from prep_blocks
            // with blk = sub)
            const int sub = split_sub(p);
            for (int h = 0; h * sub < nj; ++h) {
                const int c1 = c0 + h * sub;
                const int nh = nj - h * sub < sub ? nj - h * sub : sub;
                const double* hsrc = h == 0 ? src : Y + c1;
                const int64_t lh = h == 0 ? lsrc : ldy;
                const int js = c1 / sub;
                {
                    KTimer kt(p, st, RPCHOLQR_KERNEL_ROWPASS, static_cast<double>(m) * nh * nh);
                    if (launch_rowpass_ex(false, pad16(nh), hsrc, lh, Y + c1, ldy, m, nh, frag + js * sub * sub,
                                          diag + js * (sub / 8) * 64, nullptr, info, grid, st, check_finite, p->xexp,
                                          c1 == 0 ? 1 : 2, p->colexp + c1) != cudaSuccess)
                        return RPCHOLQR_ERR_CUDA;
                }
                ++p->launches;
                const int rest = c0 + nj - (c1 + nh);
                if (rest > 0) {
                    // the first sub-block's update reads the block's input columns, later ones updated columns
                    const bool from_input = J == 0 && h == 0;
                    const double* B = (from_input ? X : Y) + c1 + nh;
                    const int64_t ldb = from_input ? ldx : ldy;
                    rpcholqr_status rc = ozaki_gemm_internal(p, true, Y + c1, m, nh, ldy,
                                                             T + static_cast<int64_t>(c1) * ldt + c1 + nh, rest, ldt,
                                                             B, ldb, Y + c1 + nh, ldy, info, st, true);
                    if (rc != RPCHOLQR_OK) return rc;
                }
            }
            continue;
        }
        {
            KTimer kt(p, st, RPCHOLQR_KERNEL_ROWPASS, static_cast<double>(m) * nj * nj);
            if (launch_rowpass_ex(false, pad16(nj), src, lsrc, Y + c0, ldy, m, nj, frag + J * kBlk * kBlk,
                                  diag + J * (kBlk / 8) * 64, nullptr, info, grid, st, check_finite,
                                  nullptr, 0, nullptr) != cudaSuccess)
                return RPCHOLQR_ERR_CUDA;
        }
        ++p->launches;
    }
    if (pm && pass1_marks && n <= kBlk) {
        pm->mark(RPCHOLQR_PHASE_PASS1_UPDATE);
        pm->mark(RPCHOLQR_PHASE_PASS1_SOLVE2);
    }
    return check_launch();
}

// W = R1^{-1} (np x np, identity-padded) for the split second pass: the warp-per-column back
// substitution up to kTriuInvMaxN columns; wider, the FP64 blocked row solve of the identity's first n
// rows by R1 (row i of W solves w_i^T R1 = e_i^T), with R1's diagonal-block tables in frag_1 / diag_1.
static rpcholqr_status inverse_r1(rpcholqr_plan_s* p, int n, int np, int32_t* info, cudaStream_t st) {
    if (n <= kTriuInvMaxN) {
        launch_triu_inv(p->R1, np, n, np, p->W, info, st);
        ++p->launches;
        return check_launch();
    }
    launch_fill_identity(p->W, np, info, st);
    ++p->launches;
    prep_blocks(p, p->R1, np, n, p->frag_1, p->diag_1, info, st);
    return solve_blocked(p, p->W, np, p->R1, np, n, n, p->W, np, p->frag_1, p->diag_1, false, false, info, st,
                         nullptr, false);
}

// Row-range partials of G = X^T X in FP64 (n > 128) and their fixed-order sum into G (ld ldg).
static rpcholqr_status gram_fp64_wide(rpcholqr_plan_s* p, const double* X, int64_t ldx, int64_t m, int n, double* G,
                               int64_t ldg, int32_t* info, cudaStream_t st) {
    const int np = pad_np(n);
    const int nb = np / kBlk;
    const int tiles = nb * (nb + 1) / 2;
    int ranges = 2 * p->grid / tiles;   // two CTAs per SM fit
    if (p->cur_tune.syrk_ranges > 0) ranges = p->cur_tune.syrk_ranges;   // autotuned split-K factor
    if (ranges < 1) ranges = 1;
    if (ranges > p->nparts) ranges = p->nparts;
    const int64_t max_ranges = (m + 31) / 32;
    if (ranges > max_ranges) ranges = static_cast<int>(max_ranges);
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_FP64_SYRK, static_cast<double>(m) * n * n);
        if (launch_syrk_fp64(X, ldx, m, n, np, ranges, p->gpart, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    }
    launch_gram_reduce(p->gpart, ranges, np, n, G, ldg, info, st);
    p->launches += 2;
    return check_launch();
}

static rpcholqr_status precondition_internal(rpcholqr_plan p, const double* A, int64_t m, int32_t n,
                                             int64_t lda, const double* Rs, int64_t ldrs, double* A1,
                                             int64_t ld1, double* G_user, int32_t* info,
                                             cudaStream_t st, const PhaseMarks* pm) {
    const int np = pad_np(n);
    double* G = G_user ? G_user : p->G;
    const int64_t ldg = G_user ? n : np;
    if (pm) pm->mark(RPCHOLQR_PHASE_PREP_RS);
    if (np > kMaxNP) {
        // wide: blocked solve into A1, then a separate Gram pass
        prep_blocks(p, Rs, ldrs, n, p->frag_s, p->diag_s, info, st);
        if (pm) pm->mark(RPCHOLQR_PHASE_PASS1);
        rpcholqr_status rc = solve_blocked(p, A, lda, Rs, ldrs, m, n, A1, ld1, p->frag_s, p->diag_s, false, true,
                                           info, st, pm, true);
        if (rc != RPCHOLQR_OK) return rc;
        if (pm) pm->mark(RPCHOLQR_PHASE_GRAM_REDUCE);
        return gram_fp64_wide(p, A1, ld1, m, n, G, ldg, info, st);
    }
    launch_prep_tri(Rs, ldrs, n, np, p->frag_s, p->diag_s, info, st);
    ++p->launches;
    if (check_launch() != RPCHOLQR_OK) return RPCHOLQR_ERR_CUDA;
    const int grid = row_grid(p, m);
    if (pm) pm->mark(RPCHOLQR_PHASE_PASS1);
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_ROWPASS, 2.0 * m * n * n);
        if (launch_rowpass(true, np, A, lda, A1, ld1, m, n, p->frag_s, p->diag_s, p->gpart, info, grid, st) !=
            cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    }
    ++p->launches;
    if (pm) {
        pm->mark(RPCHOLQR_PHASE_PASS1_UPDATE);
        pm->mark(RPCHOLQR_PHASE_PASS1_SOLVE2);
        pm->mark(RPCHOLQR_PHASE_GRAM_REDUCE);
    }
    launch_gram_reduce(p->gpart, grid, np, n, G, ldg, info, st);
    ++p->launches;
    return check_launch();
}

static rpcholqr_status solve_internal(rpcholqr_plan p, const double* X, int64_t m, int32_t n,
                                      int64_t ldx, const double* T, int64_t ldt, double* Y, int64_t ldy,
                                      int32_t* info, cudaStream_t st, const PhaseMarks* pm) {
    const int np = pad_np(n);
    if (pm) pm->mark(RPCHOLQR_PHASE_PREP_R1);
    if (np > kMaxNP) {
        prep_blocks(p, T, ldt, n, p->frag_1, p->diag_1, info, st);
        if (pm) pm->mark(RPCHOLQR_PHASE_PASS2);
        return solve_blocked(p, X, ldx, T, ldt, m, n, Y, ldy, p->frag_1, p->diag_1, false, false, info, st,
                             nullptr, false);
    }
    launch_prep_tri(T, ldt, n, np, p->frag_1, p->diag_1, info, st);
    ++p->launches;
    if (check_launch() != RPCHOLQR_OK) return RPCHOLQR_ERR_CUDA;
    const int grid = row_grid(p, m);
    if (pm) pm->mark(RPCHOLQR_PHASE_PASS2);
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_ROWPASS, static_cast<double>(m) * n * n);
        if (launch_rowpass(false, np, X, ldx, Y, ldy, m, n, p->frag_1, p->diag_1, nullptr, info, grid, st) !=
            cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    }
    ++p->launches;
    return RPCHOLQR_OK;
}

// C = X Y (sub = false) or C = B - X Y (sub = true) on the tensor cores; X row bounds computed here.
// xexp_ready: p->xexp already holds the row bounds of X (written by the row pass that produced X);
// row0: X's first row within the matrix whose bounds p->xexp holds; y_ready: p->yblocks already holds
// the slices of this Y; y_upper: Y is upper triangular (the product skips its zero K stages).
static rpcholqr_status ozaki_gemm_internal(rpcholqr_plan p, bool sub, const double* X, int64_t m, int K,
                                           int64_t ldx, const double* Y, int N, int64_t ldy, const double* B,
                                           int64_t ldb, double* C, int64_t ldc, int32_t* info, cudaStream_t st,
                                           bool xexp_ready, int64_t row0, bool y_ready, bool y_upper,
                                           const uint8_t* aimg, int img_nkw, const int32_t* bexp, int64_t ld_bexp) {
    int32_t* xexp = p->xexp + row0;
    if (!xexp_ready) {
        launch_row_exp(X, ldx, m, K, xexp, st);
        ++p->launches;
    }
    if (!y_ready) {
        launch_ozaki_slice_cols(Y, ldy, K, N, p->yblocks, p->yexp, info, st);
        ++p->launches;
    }
    if (check_launch() != RPCHOLQR_OK) return RPCHOLQR_ERR_CUDA;
    const int64_t tiles = ((m + 127) / 128) * ((N + 63) / 64);
    const int grid = static_cast<int>(tiles < p->grid ? tiles : p->grid);
    {
        KTimer kt(p, st, ozaki_class(sub, K, N), ozaki_flops(sub, y_upper, m, K, N));
        if (launch_ozaki_gemm(sub, X, ldx, xexp, K, p->yblocks, p->yexp, N, B, ldb, C, ldc, m, info, grid, st,
                              static_cast<long>(p->spin_limit), y_upper, aimg,
                              img_nkw > 0 ? img_nkw : (K + 31) / 32, bexp, ld_bexp) !=
            cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    }
    ++p->launches;
    return RPCHOLQR_OK;
}

// G (n x n, ld ldg) = X^T X on the tensor cores: column bounds, per-range partials, fixed-order sum.
// colexp_ready: p->colexp already holds the column bounds of X.
static rpcholqr_status ozaki_gram_internal(rpcholqr_plan p, const double* X, int64_t m, int n, int64_t ldx,
                                           double* G, int64_t ldg, int32_t* info, cudaStream_t st,
                                           bool colexp_ready = false) {
    const int np = pad_np(n);
    if (!colexp_ready) {
        launch_col_exp(X, ldx, m, n, p->colexp, st);
        p->launches += 2;
    }
    // row ranges: the fewest that make (tiles x ranges) a whole number of waves over the SMs, so no SM
    // idles in the last wave (p->gpart holds p->nparts partials)
    const int nh = ozaki_gram_tiles(np, p->aimg != nullptr);
    int nranges = p->grid / nh;
    if (nranges > p->nparts) nranges = p->nparts;
    for (int r = nranges > 1 ? nranges : 1; r <= p->nparts; ++r)
        if ((static_cast<int64_t>(r) * nh) % p->grid == 0) {
            nranges = r;
            break;
        }
    if (p->cur_tune.gram_ranges > 0) nranges = p->cur_tune.gram_ranges;   // autotuned split-K factor
    if (nranges > p->nparts) nranges = p->nparts;
    if (nranges < 1) nranges = 1;
    const int64_t max_ranges = (m + 31) / 32;
    if (nranges > max_ranges) nranges = static_cast<int>(max_ranges);
    if (p->aimg) {
        // above 128 columns: the column slices made once per row chunk into stage images; the chunks'
        // partials are summed into the same nranges partials in chunk order
        for (int64_t r0 = 0; r0 < m; r0 += p->img_rows) {
            const int64_t rows = m - r0 < p->img_rows ? m - r0 : p->img_rows;
            launch_slice_col_images(X + r0 * ldx, ldx, rows, n, np, p->colexp, p->aimg, info, st);
            ++p->launches;
            KTimer kt(p, st, RPCHOLQR_KERNEL_SPLIT_GRAM, static_cast<double>(rows) * n * n);
            if (launch_ozaki_gram(X + r0 * ldx, ldx, rows, n, np, p->colexp, nranges, p->gpart, info, st,
                                  static_cast<long>(p->spin_limit), p->aimg, r0 > 0) != cudaSuccess)
                return RPCHOLQR_ERR_CUDA;
            ++p->launches;
        }
    } else {
        KTimer kt(p, st, RPCHOLQR_KERNEL_SPLIT_GRAM, static_cast<double>(m) * n * n);
        if (launch_ozaki_gram(X, ldx, m, n, np, p->colexp, nranges, p->gpart, info, st,
                              static_cast<long>(p->spin_limit), nullptr, false) != cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
        ++p->launches;
    }
    launch_gram_reduce(p->gpart, nranges, np, n, G, ldg, info, st);
    ++p->launches;
    return check_launch();
}

// SPLIT64 factorisation: see rpcholqr_mode.  A1 lives in the plan's buffer, Q receives only Q.
static rpcholqr_status factor_split(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                    int32_t s, uint64_t seed, double* Q, int64_t ldq, double* R,
                                    int32_t* info, cudaStream_t st, const PhaseMarks& pm) {
    const int np = pad_np(n);
    rpcholqr_status rc = sketch_internal(p, A, m, n, lda, s, seed, 0, nullptr, info, st, &pm);
    if (rc != RPCHOLQR_OK) return rc;
    double* A1 = p->A1;
    const int64_t ld1 = np;
    pm.mark(RPCHOLQR_PHASE_PREP_RS);
    launch_fill_noexp(p->colexp, n, st);   // column bounds of A1, atomically max-merged by the row passes
    ++p->launches;
    // A1 = A R_s^{-1}: FP64 row passes on the diagonal blocks, split tensor-core updates for the rest.
    // Up to 128 columns: 32-column blocks, right-looking (every update one K stage, wide N); above:
    // 64-column blocks, left-looking (long K windows; fewer passes over the trailing columns).
    if (np <= kMaxNP) {
        prep_blocks(p, p->Rs, np, n, p->frag_s, p->diag_s, info, st, split_sub(p));
        pm.mark(RPCHOLQR_PHASE_PASS1);
        rc = solve_split_right(p, A, lda, p->Rs, np, m, n, A1, ld1, p->frag_s, p->diag_s, info, st, &pm);
    } else {
        prep_blocks(p, p->Rs, np, n, p->frag_s, p->diag_s, info, st, split_sub(p));
        pm.mark(RPCHOLQR_PHASE_PASS1);
        rc = p->aimg ? solve_split_wide(p, A, lda, p->Rs, np, m, n, A1, ld1, p->frag_s, p->diag_s, info, st, &pm)
                     : solve_blocked(p, A, lda, p->Rs, np, m, n, A1, ld1, p->frag_s, p->diag_s, true, true, info, st,
                                     &pm, true);
    }
    if (rc != RPCHOLQR_OK) return rc;
    pm.mark(RPCHOLQR_PHASE_GRAM_REDUCE);
    if ((rc = ozaki_gram_internal(p, A1, m, n, ld1, p->G, np, info, st, true)) != RPCHOLQR_OK) return rc;
    pm.mark(RPCHOLQR_PHASE_CHOLESKY);
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_CHOLESKY, static_cast<double>(n) * n * n / 3.0);
        if (launch_cholesky(p->G, np, n, np, p->R1, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    }
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_PREP_R1);
    if ((rc = inverse_r1(p, n, np, info, st)) != RPCHOLQR_OK) return rc;
    launch_pass2_gate(p->R1, p->W, n, np, kSplitPass2Tau, info, p->gates, st);
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_PASS2);
    // Q = A1 R1^{-1}: the split product with the explicit inverse when A1 is well conditioned, else the
    // FP64 row-wise substitution; both are launched, the gate words make the other one return at once
    if (p->aimg) {
        // above 128 columns: A1 sliced once per row chunk into stage images, then the product copies them
        // (the same slices, so the same bits as slicing inside the product).  The chunk stays at most 8 GiB
        // of images even when the buffer holds every row: one launch over all 2^23 rows of a 512-column
        // A1 measured 95 ms against 74.6 ms for eight 2^20-row launches (the first pass and the Gram are
        // single launches)
        const int64_t chunk = p->img_rows < image_chunk_rows(p->np) ? p->img_rows : image_chunk_rows(p->np);
        for (int64_t r0 = 0; r0 < m; r0 += chunk) {
            const int64_t rows = m - r0 < chunk ? m - r0 : chunk;
            launch_slice_images(A1 + r0 * ld1, ld1, rows, n, p->xexp + r0, p->aimg, p->gates, st);
            ++p->launches;
            if ((rc = ozaki_gemm_internal(p, false, A1 + r0 * ld1, rows, n, ld1, p->W, n, np, nullptr, 0, Q + r0 * ldq,
                                          ldq, p->gates, st, true, r0, r0 > 0, true, p->aimg)) != RPCHOLQR_OK)
                return rc;
        }
    } else if ((rc = ozaki_gemm_internal(p, false, A1, m, n, ld1, p->W, n, np, nullptr, 0, Q, ldq, p->gates, st,
                                         true, 0, false, true)) != RPCHOLQR_OK) {
        return rc;
    }
    // the FP64 branch is timed as a whole in the PASS2 phase but kept out of the kernel classes: with the
    // gate on the split product (the usual case) its launches return at once and carry no work
    p->kuntimed = true;
    rc = solve_internal(p, A1, m, n, ld1, p->R1, np, Q, ldq, p->gates + 2, st, nullptr);
    p->kuntimed = false;
    if (rc != RPCHOLQR_OK) return rc;
    launch_gate_merge(info, p->gates, st);
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_RECOVER_R);
    launch_triu_mul(p->R1, np, p->Rs, np, n, R, n, info, st);
    ++p->launches;
    pm.mark(RPCHOLQR_NUM_PHASES);
    return check_launch();
}

rpcholqr_status rpcholqr_factor(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                int32_t s, uint64_t seed, double* Q, int64_t ldq, double* R,
                                int32_t* info, void* stream) {
    if (!p || !A || !Q || !R || !info || p->mode == RPCHOLQR_FP32) return RPCHOLQR_ERR_ARG;
    if (!shape_ok(p, m, n, s) || lda < n || ldq < n) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int np = pad_np(n);
    const PhaseMarks pm(p, st);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    if (p->mode == RPCHOLQR_SPLIT64) return factor_split(p, A, m, n, lda, s, seed, Q, ldq, R, info, st, pm);
    if ((rc = sketch_internal(p, A, m, n, lda, s, seed, 0, nullptr, info, st, &pm)) != RPCHOLQR_OK) return rc;
    if ((rc = precondition_internal(p, A, m, n, lda, p->Rs, np, Q, ldq, nullptr, info, st, &pm)) !=
        RPCHOLQR_OK)
        return rc;
    pm.mark(RPCHOLQR_PHASE_CHOLESKY);
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_CHOLESKY, static_cast<double>(n) * n * n / 3.0);
        if (launch_cholesky(p->G, np, n, np, p->R1, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    }
    ++p->launches;
    if ((rc = solve_internal(p, Q, m, n, ldq, p->R1, np, Q, ldq, info, st, &pm)) != RPCHOLQR_OK) return rc;
    pm.mark(RPCHOLQR_PHASE_RECOVER_R);
    launch_triu_mul(p->R1, np, p->Rs, np, n, R, n, info, st);
    ++p->launches;
    pm.mark(RPCHOLQR_NUM_PHASES);
    return check_launch();
}

rpcholqr_status rpcholqr_factor_batched(rpcholqr_plan p, int32_t count, const double* const* A, const int64_t* m,
                                        const int32_t* n, const int64_t* lda, const int32_t* s, const uint64_t* seed,
                                        double* const* Q, const int64_t* ldq, double* const* R, int32_t* info,
                                        void* stream) {
    if (!p || count < 1 || count > kMaxBatchCount || !A || !m || !n || !lda || !s || !seed || !Q || !ldq || !R ||
        !info)
        return RPCHOLQR_ERR_ARG;
    if (p->mode != RPCHOLQR_FP64 || pad_np(p->max_n) > batch_max_np() || p->smoothing)
        return RPCHOLQR_ERR_UNSUPPORTED;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    if (count > p->batch_capacity) {
        const rpcholqr_status rc = reserve_batch(p, count);
        if (rc != RPCHOLQR_OK) return rc;
    }
    if (launch_batch_persistent(count, A, m, n, lda, s, seed, Q, ldq, R, info, p->batch_ws, p->batch_capacity,
                                p->max_m, p->max_n, p->max_s, p->grid, p->scale_sample,
                                static_cast<long>(p->spin_limit), p->batch_grid,
                                static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return RPCHOLQR_ERR_CUDA;
    }
    p->launches += 2;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_factor_f32(rpcholqr_plan p, const float* A, int64_t m, int32_t n, int64_t lda,
                                    int32_t s, uint64_t seed, float* Q, int64_t ldq, float* R, int32_t* info,
                                    void* stream) {
    if (!p || !A || !Q || !R || !info || p->mode != RPCHOLQR_FP32) return RPCHOLQR_ERR_ARG;
    if (!shape_ok(p, m, n, s) || lda < n || ldq < n) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int np = pad_np(n);
    const PhaseMarks pm(p, st);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    // sample (widened to FP64) and the FP64 Householder R_s
    pm.mark(RPCHOLQR_PHASE_SAMPLE);
    const double scale = sample_scale(p, m, s);
    if (p->smoothing) {
        if (plan_smoothed_sample<float>(p, A, m, n, lda, s, seed, np, info, st) != cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    } else {
        launch_sample_gather_f32(A, m, n, lda, s, seed, 0, scale, p->As, s, np, nullptr, info, st);
        ++p->launches;
    }
    pm.mark(RPCHOLQR_PHASE_SKETCH_QR);
    if (launch_householder(p->As, s, s, n, np, p->Rs, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    ++p->launches;
    // pass 1 in FP32: A1 = A R_s^{-1} into Q, then the Gram partials and their FP64 sum
    pm.mark(RPCHOLQR_PHASE_PREP_RS);
    launch_prep_f32(p->Rs, np, n, p->T32, p->rinv32, RPCHOLQR_ERR_SINGULAR_SKETCH, info, st);
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_PASS1);
    if (launch_rowsolve_f32(A, lda, Q, ldq, m, n, p->T32, p->rinv32, info, true, st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_PASS1_UPDATE);
    pm.mark(RPCHOLQR_PHASE_PASS1_SOLVE2);
    pm.mark(RPCHOLQR_PHASE_GRAM_REDUCE);
    const int np64 = (n + 63) / 64 * 64;
    const int ranges = launch_syrk_f32(Q, ldq, m, n, p->nparts, p->gpart, info, st);
    launch_gram_reduce(p->gpart, ranges, np64, n, p->G, np, info, st);
    p->launches += 2;
    // FP64 Cholesky, pass 2 in FP32 (in place), R = R1 R_s in FP64 rounded to FP32
    pm.mark(RPCHOLQR_PHASE_CHOLESKY);
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_CHOLESKY, static_cast<double>(n) * n * n / 3.0);
        if (launch_cholesky(p->G, np, n, np, p->R1, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    }
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_PREP_R1);
    launch_prep_f32(p->R1, np, n, p->T32, p->rinv32, RPCHOLQR_ERR_NOT_SPD, info, st);
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_PASS2);
    if (launch_rowsolve_f32(Q, ldq, Q, ldq, m, n, p->T32, p->rinv32, info, false, st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    ++p->launches;
    pm.mark(RPCHOLQR_PHASE_RECOVER_R);
    launch_triu_mul(p->R1, np, p->Rs, np, n, p->frag_s, n, info, st);
    launch_f64_to_f32(p->frag_s, n, n, R, n, st);
    p->launches += 2;
    pm.mark(RPCHOLQR_NUM_PHASES);
    return check_launch();
}

rpcholqr_status rpcholqr_plan_enable_timing(rpcholqr_plan p, int32_t max_calls) {
    if (!p || max_calls < 0) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    free_events(p);
    if (max_calls == 0) return RPCHOLQR_OK;
    if (max_calls > 4096) return RPCHOLQR_ERR_ARG;
    const int total = max_calls * (RPCHOLQR_NUM_PHASES + 1);
    const int ktotal = 2 * max_calls * kMaxTimedLaunches;
    p->events = new (std::nothrow) cudaEvent_t[total]();
    p->kevents = new (std::nothrow) cudaEvent_t[ktotal]();
    p->kclass = new (std::nothrow) int8_t[max_calls * kMaxTimedLaunches]();
    p->kflops = new (std::nothrow) double[max_calls * kMaxTimedLaunches]();
    p->klaunches = new (std::nothrow) int32_t[max_calls]();
    p->timing_slots = max_calls;   // free_events destroys what was created so far
    if (!p->events || !p->kevents || !p->kclass || !p->kflops || !p->klaunches) {
        free_events(p);
        return RPCHOLQR_ERR_NOMEM;
    }
    for (int i = 0; i < total; ++i)
        if (cudaEventCreate(&p->events[i]) != cudaSuccess) {
            free_events(p);
            return RPCHOLQR_ERR_CUDA;
        }
    for (int i = 0; i < ktotal; ++i)
        if (cudaEventCreate(&p->kevents[i]) != cudaSuccess) {
            free_events(p);
            return RPCHOLQR_ERR_CUDA;
        }
    p->timed_calls = 0;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_plan_collect_kernel_timing(rpcholqr_plan p, float* ms_per_class, int64_t* launches_per_class,
                                                    double* flops_per_class) {
    if (!p) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    for (int c = 0; c < RPCHOLQR_NUM_KERNEL_CLASSES; ++c) {
        if (ms_per_class) ms_per_class[c] = 0.f;
        if (launches_per_class) launches_per_class[c] = 0;
        if (flops_per_class) flops_per_class[c] = 0.0;
    }
    const int n = p->kevents ? p->timed_calls : 0;
    for (int slot = 0; slot < n; ++slot)
        for (int i = 0; i < p->klaunches[slot]; ++i) {
            const int k = slot * kMaxTimedLaunches + i;
            if (cudaEventSynchronize(p->kevents[2 * k + 1]) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p->kevents[2 * k], p->kevents[2 * k + 1]) != cudaSuccess)
                return RPCHOLQR_ERR_CUDA;
            const int c = p->kclass[k];
            if (ms_per_class) ms_per_class[c] += ms;
            if (launches_per_class) ++launches_per_class[c];
            if (flops_per_class) flops_per_class[c] += p->kflops[k];
        }
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_plan_collect_timing(rpcholqr_plan p, float* ms_per_phase, int32_t* calls,
                                             int64_t* launches) {
    if (!p) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    if (ms_per_phase)
        for (int ph = 0; ph < RPCHOLQR_NUM_PHASES; ++ph) ms_per_phase[ph] = 0.f;
    const int n = p->events ? p->timed_calls : 0;
    for (int c = 0; c < n; ++c) {
        cudaEvent_t* ev = p->events + c * (RPCHOLQR_NUM_PHASES + 1);
        if (cudaEventSynchronize(ev[RPCHOLQR_NUM_PHASES]) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
        for (int ph = 0; ph < RPCHOLQR_NUM_PHASES; ++ph) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
            if (ms_per_phase) ms_per_phase[ph] += ms;
        }
    }
    if (calls) *calls = n;
    if (launches) *launches = p->launches;
    p->timed_calls = 0;
    p->launches = 0;
    return RPCHOLQR_OK;
}

// rpcholqr_factor_host for SPLIT64 (n <= 128, contiguous host matrices): the copies overlap the work.
// A goes to the device in kHostChunks row blocks on a copy stream; meanwhile the sample indices are
// computed on the device and read back, the host gathers the s sampled rows from its own copy of A
// and sends them ahead, and the sketch QR runs; pass 1 then solves each row block as soon as it has
// arrived.  After the Gram matrix, the Cholesky factor and R1^{-1}, pass 2 runs block by block and
// each block of Q is copied back while the next is computed.  Every step is the one rpcholqr_factor
// takes, on the same rows, so the results are identical to it.
constexpr int kHostChunks = 4;   // 8 measured the same (53.7 vs 54.5 matrices/s end to end)
static_assert(2 * kHostChunks <= static_cast<int>(sizeof(rpcholqr_plan_s::hev) / sizeof(cudaEvent_t)),
              "one arrival and one completion event per row block");
static rpcholqr_status factor_host_split(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int32_t s,
                                         uint64_t seed, double* Q, double* R, int32_t* info_host, cudaStream_t st) {
    const int np = pad_np(n);
    const int64_t ld1 = np;
    double* dA = p->hA;
    double* dQ = p->hQ;
    int32_t* info = p->hinfo;
    if (!p->hcopy) {
        if (cudaStreamCreateWithFlags(&p->hcopy, cudaStreamNonBlocking) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
        for (cudaEvent_t& e : p->hev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    }
    if (!p->hidx_dev) {
        const size_t ms = static_cast<size_t>(p->max_s);
        if (cudaMalloc(&p->hidx_dev, ms * sizeof(int64_t)) != cudaSuccess ||
            cudaMallocHost(&p->hidx_host, ms * sizeof(int64_t)) != cudaSuccess ||
            cudaMallocHost(&p->hrows_host, ms * p->max_n * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&p->hrows_dev, ms * p->max_n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return RPCHOLQR_ERR_NOMEM;
        }
    }
    int64_t rows_per = (m + kHostChunks - 1) / kHostChunks;
    rows_per = (rows_per + 127) / 128 * 128;
    const int nchunks = static_cast<int>((m + rows_per - 1) / rows_per);
    auto chunk = [&](int c, int64_t& r0, int64_t& rows) {
        r0 = c * rows_per;
        rows = m - r0 < rows_per ? m - r0 : rows_per;
    };
    const size_t row_bytes = static_cast<size_t>(n) * sizeof(double);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    // the sample first: indices on the device, rows gathered on the host and sent before A (a copy
    // engine serves its queue in order, so the sample must not wait behind the row blocks of A)
    launch_sample_indices(seed, 0, m, s, p->hidx_dev, st);
    if (cudaMemcpyAsync(p->hidx_host, p->hidx_dev, static_cast<size_t>(s) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    for (int j = 0; j < s; ++j) std::memcpy(p->hrows_host + static_cast<size_t>(j) * n, A + p->hidx_host[j] * n, row_bytes);
    if (cudaMemcpyAsync(p->hrows_dev, p->hrows_host, static_cast<size_t>(s) * row_bytes, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    // A in row blocks on the copy stream (st has nothing queued that touches the staging buffers)
    for (int c = 0; c < nchunks; ++c) {
        int64_t r0, rows;
        chunk(c, r0, rows);
        if (cudaMemcpyAsync(dA + r0 * n, A + r0 * n, static_cast<size_t>(rows) * row_bytes, cudaMemcpyHostToDevice,
                            p->hcopy) != cudaSuccess ||
            cudaEventRecord(p->hev[c], p->hcopy) != cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    }
    launch_sample_rows(p->hrows_dev, n, s, sample_scale(p, m, s), p->As, s, np,
                       info, st);
    if (launch_householder(p->As, s, s, n, np, p->Rs, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    p->launches += 3;
    // pass 1, block by block as A arrives
    launch_fill_noexp(p->colexp, n, st);
    prep_blocks(p, p->Rs, np, n, p->frag_s, p->diag_s, info, st, split_sub(p));
    for (int c = 0; c < nchunks; ++c) {
        int64_t r0, rows;
        chunk(c, r0, rows);
        if (cudaStreamWaitEvent(st, p->hev[c], 0) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
        if ((rc = solve_split_right(p, dA + r0 * n, n, p->Rs, np, rows, n, p->A1 + r0 * ld1, ld1, p->frag_s,
                                    p->diag_s, info, st, nullptr, r0)) != RPCHOLQR_OK)
            return rc;
    }
    if ((rc = ozaki_gram_internal(p, p->A1, m, n, ld1, p->G, np, info, st, true)) != RPCHOLQR_OK) return rc;
    {
        KTimer kt(p, st, RPCHOLQR_KERNEL_CHOLESKY, static_cast<double>(n) * n * n / 3.0);
        if (launch_cholesky(p->G, np, n, np, p->R1, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    }
    if ((rc = inverse_r1(p, n, np, info, st)) != RPCHOLQR_OK) return rc;
    launch_pass2_gate(p->R1, p->W, n, np, kSplitPass2Tau, info, p->gates, st);
    p->launches += 2;
    // pass 2 block by block; each block of Q goes back while the next is computed
    for (int c = 0; c < nchunks; ++c) {
        int64_t r0, rows;
        chunk(c, r0, rows);
        if ((rc = ozaki_gemm_internal(p, false, p->A1 + r0 * ld1, rows, n, ld1, p->W, n, np, nullptr, 0, dQ + r0 * n, n,
                                      p->gates, st, true, r0, c > 0, true)) != RPCHOLQR_OK)
            return rc;
        p->kuntimed = true;     // the gated-off FP64 branch (see factor_split)
        rc = solve_internal(p, p->A1 + r0 * ld1, rows, n, ld1, p->R1, np, dQ + r0 * n, n, p->gates + 2, st, nullptr);
        p->kuntimed = false;
        if (rc != RPCHOLQR_OK) return rc;
        if (cudaEventRecord(p->hev[kHostChunks + c], st) != cudaSuccess ||
            cudaStreamWaitEvent(p->hcopy, p->hev[kHostChunks + c], 0) != cudaSuccess ||
            cudaMemcpyAsync(Q + r0 * n, dQ + r0 * n, static_cast<size_t>(rows) * row_bytes, cudaMemcpyDeviceToHost,
                            p->hcopy) != cudaSuccess)
            return RPCHOLQR_ERR_CUDA;
    }
    launch_gate_merge(info, p->gates, st);
    launch_triu_mul(p->R1, np, p->Rs, np, n, p->hR, n, info, st);
    p->launches += 2;
    if (cudaMemcpyAsync(R, p->hR, static_cast<size_t>(n) * n * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(info_host, info, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    if (check_launch() != RPCHOLQR_OK) return RPCHOLQR_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess && cudaStreamSynchronize(p->hcopy) == cudaSuccess
               ? RPCHOLQR_OK
               : RPCHOLQR_ERR_CUDA;
}

rpcholqr_status rpcholqr_factor_host(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                     int32_t s, uint64_t seed, double* Q, int64_t ldq, double* R,
                                     int32_t* info_host, void* stream) {
    if (!p || !A || !Q || !R || !info_host) return RPCHOLQR_ERR_ARG;
    if (!shape_ok(p, m, n, s) || lda < n || ldq < n) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t elems = static_cast<size_t>(m) * static_cast<size_t>(n);
    if (elems > p->staged_elems || !p->hR) {
        cudaFree(p->hA); cudaFree(p->hQ); cudaFree(p->hR); cudaFree(p->hinfo);
        p->hA = p->hQ = p->hR = nullptr; p->hinfo = nullptr; p->staged_elems = 0;
        const size_t nn = static_cast<size_t>(p->max_n) * p->max_n;
        if (cudaMalloc(&p->hA, elems * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&p->hQ, elems * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&p->hR, nn * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&p->hinfo, 2 * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return RPCHOLQR_ERR_NOMEM;
        }
        p->staged_elems = elems;
    }
    if (p->mode == RPCHOLQR_SPLIT64 && !p->smoothing && pad_np(n) <= kMaxNP && lda == n && ldq == n &&
        m >= 128 * kHostChunks)
        return factor_host_split(p, A, m, n, s, seed, Q, R, info_host, st);
    const size_t row_bytes = static_cast<size_t>(n) * sizeof(double);
    // contiguous host matrices (ld = n) go as one linear copy; strided ones row by row (2-D copy)
    const cudaError_t ein =
        lda == n ? cudaMemcpyAsync(p->hA, A, elems * sizeof(double), cudaMemcpyHostToDevice, st)
                 : cudaMemcpy2DAsync(p->hA, row_bytes, A, static_cast<size_t>(lda) * sizeof(double), row_bytes,
                                     static_cast<size_t>(m), cudaMemcpyHostToDevice, st);
    if (ein != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    rpcholqr_status rc = rpcholqr_factor(p, p->hA, m, n, n, s, seed, p->hQ, n, p->hR, p->hinfo, stream);
    if (rc != RPCHOLQR_OK) return rc;
    const cudaError_t eout =
        ldq == n ? cudaMemcpyAsync(Q, p->hQ, elems * sizeof(double), cudaMemcpyDeviceToHost, st)
                 : cudaMemcpy2DAsync(Q, static_cast<size_t>(ldq) * sizeof(double), p->hQ, row_bytes, row_bytes,
                                     static_cast<size_t>(m), cudaMemcpyDeviceToHost, st);
    if (eout != cudaSuccess ||
        cudaMemcpyAsync(R, p->hR, static_cast<size_t>(n) * n * sizeof(double), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(info_host, p->hinfo, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? RPCHOLQR_OK : RPCHOLQR_ERR_CUDA;
}

rpcholqr_status rpcholqr_sketch_r(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                  int32_t s, uint64_t seed, double* Rs, int32_t* info, void* stream) {
    if (!p || !A || !Rs || !info) return RPCHOLQR_ERR_ARG;
    if (!shape_ok(p, m, n, s) || lda < n) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    return sketch_internal(p, A, m, n, lda, s, seed, 0, Rs, info, st, nullptr);
}

rpcholqr_status rpcholqr_precondition_gram(rpcholqr_plan p, const double* A, int64_t m, int32_t n,
                                           int64_t lda, const double* Rs, double* A1, int64_t ld1,
                                           double* G, int32_t* info, void* stream) {
    if (!p || !A || !Rs || !A1 || !G || !info) return RPCHOLQR_ERR_ARG;
    if (n < 1 || n > p->max_n || m < 1 || m > p->max_m || lda < n || ld1 < n) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    return precondition_internal(p, A, m, n, lda, Rs, n, A1, ld1, G, info, st, nullptr);
}

rpcholqr_status rpcholqr_cholesky(rpcholqr_plan p, const double* G, int32_t n, double* R1,
                                  int32_t* info, void* stream) {
    if (!p || !G || !R1 || !info || n < 1 || n > p->max_n) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    const int np = pad_np(n);
    return launch_cholesky(G, n, n, np, p->R1, R1, info, st) == cudaSuccess ? RPCHOLQR_OK
                                                                             : RPCHOLQR_ERR_CUDA;
}

rpcholqr_status rpcholqr_solve_rows(rpcholqr_plan p, const double* X, int64_t m, int32_t n, int64_t ldx,
                                    const double* T, double* Y, int64_t ldy, int32_t* info,
                                    void* stream) {
    if (!p || !X || !T || !Y || !info) return RPCHOLQR_ERR_ARG;
    if (n < 1 || n > p->max_n || m < 1 || m > p->max_m || ldx < n || ldy < n) return RPCHOLQR_ERR_ARG;
    if (X == Y && ldx != ldy) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    return solve_internal(p, X, m, n, ldx, T, n, Y, ldy, info, st, nullptr);
}

rpcholqr_status rpcholqr_triu_mul(const double* R1, const double* Rs, int32_t n, double* R, void* stream) {
    if (!R1 || !Rs || !R || n < 1) return RPCHOLQR_ERR_ARG;
    launch_triu_mul(R1, n, Rs, n, n, R, n, nullptr, static_cast<cudaStream_t>(stream));
    return check_launch();
}

rpcholqr_status rpcholqr_ozaki_gemm(rpcholqr_plan p, const double* X, int64_t m, int32_t K, int64_t ldx,
                                    const double* Y, int32_t N, int64_t ldy, double* C, int64_t ldc,
                                    int32_t* info, void* stream) {
    if (!p || !X || !Y || !C || !info || p->mode != RPCHOLQR_SPLIT64) return RPCHOLQR_ERR_ARG;
    if (m < 1 || m > p->max_m || K < 1 || K > p->np || N < 1 || N > p->np || ldx < K || ldy < N || ldc < N)
        return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, K);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    return ozaki_gemm_internal(p, false, X, m, K, ldx, Y, N, ldy, nullptr, 0, C, ldc, info, st);
}

rpcholqr_status rpcholqr_ozaki_update(rpcholqr_plan p, const double* X, int64_t m, int32_t K, int64_t ldx,
                                      const double* Y, int32_t N, int64_t ldy, const double* B, int64_t ldb,
                                      double* C, int64_t ldc, int32_t* info, void* stream) {
    if (!p || !X || !Y || !B || !C || !info || p->mode != RPCHOLQR_SPLIT64) return RPCHOLQR_ERR_ARG;
    if (m < 1 || m > p->max_m || K < 1 || K > p->np || N < 1 || N > p->np || ldx < K || ldy < N || ldb < N ||
        ldc < N)
        return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, K);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    return ozaki_gemm_internal(p, true, X, m, K, ldx, Y, N, ldy, B, ldb, C, ldc, info, st);
}

rpcholqr_status rpcholqr_ozaki_gram(rpcholqr_plan p, const double* X, int64_t m, int32_t n, int64_t ldx,
                                    double* G, int32_t* info, void* stream) {
    if (!p || !X || !G || !info || p->mode != RPCHOLQR_SPLIT64) return RPCHOLQR_ERR_ARG;
    if (m < 1 || m > p->max_m || n < 1 || n > p->max_n || ldx < n) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    return ozaki_gram_internal(p, X, m, n, ldx, G, n, info, st);
}

// One Cholesky-QR step in FP64: Q = X R^{-1} with R = chol(X^T X) written to R_out (np x np, ld np).
static rpcholqr_status cholqr_step(rpcholqr_plan p, const double* X, int64_t m, int32_t n, int64_t ldx,
                                   double* Q, int64_t ldq, double* R_out, int32_t* info, cudaStream_t st,
                                   bool shifted = false) {
    const int np = pad_np(n);
    if (np > kMaxNP) {
        rpcholqr_status rc = gram_fp64_wide(p, X, ldx, m, n, p->G, np, info, st);
        if (rc != RPCHOLQR_OK) return rc;
        if (shifted) {
            launch_scholqr3_shift(p->G, np, n, m, info, st);
            ++p->launches;
        }
        if (launch_cholesky(p->G, np, n, np, R_out, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
        ++p->launches;
        return solve_internal(p, X, m, n, ldx, R_out, np, Q, ldq, info, st, nullptr);
    }
    launch_prep_tri(nullptr, 0, 0, np, p->frag_s, p->diag_s, info, st);   // identity preconditioner
    const int64_t panels = (m + 127) / 128;
    const int grid = static_cast<int>(panels < p->grid ? panels : p->grid);
    if (launch_rowpass(true, np, X, ldx, Q, ldq, m, n, p->frag_s, p->diag_s, p->gpart, info, grid, st) !=
        cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    launch_gram_reduce(p->gpart, grid, np, n, p->G, np, info, st);
    if (shifted) {
        launch_scholqr3_shift(p->G, np, n, m, info, st);
        ++p->launches;
    }
    if (launch_cholesky(p->G, np, n, np, R_out, nullptr, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    p->launches += 4;
    return solve_internal(p, Q, m, n, ldq, R_out, np, Q, ldq, info, st, nullptr);
}

static rpcholqr_status cholqr_args(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                   const double* Q, int64_t ldq, const double* R, const int32_t* info) {
    if (!p || !A || !Q || !R || !info) return RPCHOLQR_ERR_ARG;
    if (n < 1 || n > p->max_n || m < n || m > p->max_m || lda < n || ldq < n) return RPCHOLQR_ERR_ARG;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_cholqr(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                double* Q, int64_t ldq, double* R, int32_t* info, void* stream) {
    rpcholqr_status rc = cholqr_args(p, A, m, n, lda, Q, ldq, R, info);
    if (rc != RPCHOLQR_OK) return rc;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = reset_info(info, st)) != RPCHOLQR_OK) return rc;
    if ((rc = cholqr_step(p, A, m, n, lda, Q, ldq, p->R1, info, st)) != RPCHOLQR_OK) return rc;
    const size_t np = static_cast<size_t>(pad_np(n));
    if (cudaMemcpy2DAsync(R, sizeof(double) * n, p->R1, sizeof(double) * np, sizeof(double) * n,
                          static_cast<size_t>(n), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_cholqr2(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                 double* Q, int64_t ldq, double* R, int32_t* info, void* stream) {
    rpcholqr_status rc = cholqr_args(p, A, m, n, lda, Q, ldq, R, info);
    if (rc != RPCHOLQR_OK) return rc;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = reset_info(info, st)) != RPCHOLQR_OK) return rc;
    if ((rc = cholqr_step(p, A, m, n, lda, Q, ldq, p->Rs, info, st)) != RPCHOLQR_OK) return rc;   // R_a
    if ((rc = cholqr_step(p, Q, m, n, ldq, Q, ldq, p->R1, info, st)) != RPCHOLQR_OK) return rc;   // R_b
    const int np = pad_np(n);
    launch_triu_mul(p->R1, np, p->Rs, np, n, R, n, info, st);
    ++p->launches;
    return check_launch();
}

rpcholqr_status rpcholqr_scholqr3(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                  double* Q, int64_t ldq, double* R, int32_t* info, void* stream) {
    rpcholqr_status rc = cholqr_args(p, A, m, n, lda, Q, ldq, R, info);
    if (rc != RPCHOLQR_OK) return rc;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    select_tuning(p, m, n);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int np = pad_np(n);
    if ((rc = reset_info(info, st)) != RPCHOLQR_OK) return rc;
    if ((rc = cholqr_step(p, A, m, n, lda, Q, ldq, p->Rs, info, st, true)) != RPCHOLQR_OK) return rc;   // R_1
    if ((rc = cholqr_step(p, Q, m, n, ldq, Q, ldq, p->R1, info, st)) != RPCHOLQR_OK) return rc;         // R_2
    launch_triu_mul(p->R1, np, p->Rs, np, n, R, n, info, st);                                       // R_2 R_1
    if ((rc = cholqr_step(p, Q, m, n, ldq, Q, ldq, p->R1, info, st)) != RPCHOLQR_OK) return rc;         // R_3
    if (cudaMemcpy2DAsync(p->Rs, sizeof(double) * np, R, sizeof(double) * n, sizeof(double) * n,
                          static_cast<size_t>(n), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    launch_triu_mul(p->R1, np, p->Rs, np, n, R, n, info, st);                                       // R_3 R_2 R_1
    p->launches += 2;
    return check_launch();
}

rpcholqr_status rpcholqr_gather_owned_rows(const double* A_local, int64_t m_local, int32_t n, int64_t lda,
                                           int64_t row_offset, int64_t m, int32_t s, uint64_t seed, double* As,
                                           int64_t ld_as, int32_t* info, void* stream) {
    if (!As || !info || n < 1 || s < 1 || m < 1 || m_local < 0 || row_offset < 0 || row_offset > m - m_local ||
        ld_as < n || (m_local > 0 && (!A_local || lda < n)))
        return RPCHOLQR_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    const double scale = std::sqrt(static_cast<double>(m) / static_cast<double>(s));
    launch_gather_owned_rows(A_local, m_local, n, lda, row_offset, m, s, seed, 0, scale, As, ld_as, info, st);
    return check_launch();
}

rpcholqr_status rpcholqr_sketch_r_from_sample(rpcholqr_plan p, const double* As, int32_t s, int32_t n,
                                              int64_t ld_as, double* Rs, int32_t* info, void* stream) {
    if (!p || !As || !Rs || !info || n < 1 || n > p->max_n || s < n || s > p->max_s || ld_as < n)
        return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    const int np = pad_np(n);
    launch_sample_to_colmajor(As, ld_as, s, n, np, p->As, s, st);
    if (launch_householder(p->As, s, s, n, np, p->Rs, Rs, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    p->launches += 2;
    return check_launch();
}

rpcholqr_status rpcholqr_sum_partials(const double* parts, int32_t nparts, int32_t n, double* G, void* stream) {
    if (!parts || !G || nparts < 1 || n < 1) return RPCHOLQR_ERR_ARG;
    launch_sum_parts(parts, nparts, n, G, static_cast<cudaStream_t>(stream));
    return check_launch();
}

rpcholqr_status rpcholqr_autotune(rpcholqr_plan p, int32_t nclasses, const int64_t* m, const int32_t* n,
                                  const int32_t* s, int32_t reps, const char* out_json) {
    if (!p || nclasses < 1 || !m || !n || !s || reps < 1) return RPCHOLQR_ERR_ARG;
    if (p->mode == RPCHOLQR_FP32) return RPCHOLQR_ERR_UNSUPPORTED;
    for (int c = 0; c < nclasses; ++c)
        if (!shape_ok(p, m[c], n[c], s[c])) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *A = nullptr, *Q = nullptr, *R = nullptr;
    int32_t* info = nullptr;
    rpcholqr_status rc = RPCHOLQR_OK;
    auto cleanup = [&] {
        p->tune_forced = false;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        cudaFree(A);
        cudaFree(Q);
        cudaFree(R);
        cudaFree(info);
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return RPCHOLQR_ERR_CUDA;
    }
    for (int c = 0; c < nclasses && rc == RPCHOLQR_OK; ++c) {
        const int64_t mc = m[c];
        const int nc = n[c], sc = s[c], np = pad_np(nc);
        const size_t bytes = sizeof(double) * static_cast<size_t>(mc) * nc;
        if (cudaMalloc(&A, bytes) != cudaSuccess || cudaMalloc(&Q, bytes) != cudaSuccess ||
            cudaMalloc(&R, sizeof(double) * nc * nc) != cudaSuccess || cudaMalloc(&info, 2 * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            rc = RPCHOLQR_ERR_NOMEM;
            break;
        }
        launch_fill_uniform(A, static_cast<int64_t>(mc) * nc, 20240617ull + c, st);
        // candidates: the built-in rules first, then the alternatives of each parameter
        std::vector<Tuning> cands(1);
        if (p->mode == RPCHOLQR_SPLIT64) {
            cands.clear();
            const int nh = ozaki_gram_tiles(np, p->aimg != nullptr);
            const int plain = p->grid / nh > 0 ? p->grid / nh : 1;
            for (int sub : {kSplitSub, 16})   // the built-in width first; gram_ranges 0 = the wave rule
                for (int gr : {0, plain, 2 * plain}) {
                    Tuning t;
                    t.split_sub = sub;
                    t.gram_ranges = gr > p->nparts ? p->nparts : gr;
                    cands.push_back(t);
                }
        } else if (np > kMaxNP) {
            const int nb = np / kBlk, tiles = nb * (nb + 1) / 2;
            for (int f : {1, 4}) {
                Tuning t;
                t.syrk_ranges = f * p->grid / tiles > 0 ? f * p->grid / tiles : 1;
                cands.push_back(t);
            }
        }
        TuneEntry best;
        best.mode = p->mode;
        best.np = np;
        best.m_log2 = ceil_log2(mc);
        best.ms = -1.0;
        for (const Tuning& t : cands) {
            p->tune_forced = true;
            p->cur_tune = t;
            float tot = 0.f;
            for (int r = 0; r <= reps && rc == RPCHOLQR_OK; ++r) {   // r = 0: untimed warm-up
                if (r == 1) cudaEventRecord(e0, st);
                rc = rpcholqr_factor(p, A, mc, nc, nc, sc, 1 + r, Q, nc, R, info, st);
            }
            if (rc != RPCHOLQR_OK) break;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&tot, e0, e1) != cudaSuccess) {
                rc = RPCHOLQR_ERR_CUDA;
                break;
            }
            const double ms = tot / reps;
            if (best.ms < 0.0 || ms < best.ms) {
                best.ms = ms;
                best.t = t;
            }
        }
        p->tune_forced = false;
        if (rc == RPCHOLQR_OK) put_tune_entry(p, best);
        cudaFree(A);
        cudaFree(Q);
        cudaFree(R);
        cudaFree(info);
        A = Q = R = nullptr;
        info = nullptr;
    }
    cleanup();
    if (rc != RPCHOLQR_OK) return rc;
    if (out_json) {
        FILE* f = std::fopen(out_json, "wb");
        if (!f) return RPCHOLQR_ERR_ARG;
        const std::string text = tune_json(p);
        const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
        if (std::fclose(f) != 0 || !ok) return RPCHOLQR_ERR_ARG;
    }
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_autotune_table(rpcholqr_plan p, char* out, size_t capacity, size_t* length) {
    if (!p || !length) return RPCHOLQR_ERR_ARG;
    const std::string text = tune_json(p);
    *length = text.size();
    if (out && capacity > 0) {
        const size_t k = text.size() < capacity - 1 ? text.size() : capacity - 1;
        std::memcpy(out, text.data(), k);
        out[k] = 0;
    }
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_autotune_parse(const char* json_or_path, int32_t* entries) {
    if (!json_or_path || !entries) return RPCHOLQR_ERR_ARG;
    std::vector<TuneEntry> t;
    if (!load_tune_json(json_or_path, t)) return RPCHOLQR_ERR_ARG;
    *entries = static_cast<int32_t>(t.size());
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_plan_set_smoothing(rpcholqr_plan p, int32_t kind) {
    if (!p || kind < 0 || kind > 2) return RPCHOLQR_ERR_ARG;
    if (kind > p->smooth_capacity) {
        if (!smooth_supported(p->max_m)) return RPCHOLQR_ERR_UNSUPPORTED;
        DeviceGuard guard(p->device);
        if (!guard.ok) return RPCHOLQR_ERR_CUDA;
        const size_t tb = align256(kind == 2 ? smooth_dct_buffer_bytes(p->max_m, p->max_n)
                                             : smooth_buffer_bytes(p->max_m, p->max_n));
        const size_t ib = align256(sizeof(int64_t) * static_cast<size_t>(p->max_s));
        const size_t total = tb + ib + static_cast<size_t>(p->max_m);
        void* ws = nullptr;
        cudaStreamSynchronize(nullptr);
        if (cudaMalloc(&ws, total) != cudaSuccess) {
            cudaGetLastError();
            return RPCHOLQR_ERR_NOMEM;
        }
        if (p->smooth_ws) {
            cudaDeviceSynchronize();
            cudaFree(p->smooth_ws);
        }
        p->smooth_ws = ws;
        p->smooth_T = static_cast<double*>(ws);
        p->smooth_idx = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + tb);
        p->smooth_sgn = reinterpret_cast<int8_t*>(static_cast<char*>(ws) + tb + ib);
        p->smooth_capacity = kind;
        p->ws_bytes += total;
    }
    p->smoothing = kind;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_smoothed_sample(rpcholqr_plan p, const double* A, int64_t m, int32_t n, int64_t lda,
                                         int32_t s, uint64_t seed, double* As, int64_t ld_as, int32_t* info,
                                         void* stream) {
    if (!p || !A || !As || !info || !p->smoothing) return RPCHOLQR_ERR_ARG;
    if (n < 1 || n > p->max_n || s < 1 || s > p->max_s || m < 1 || m > p->max_m || lda < n || ld_as < n)
        return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpcholqr_status rc = reset_info(info, st);
    if (rc != RPCHOLQR_OK) return rc;
    const int np = pad_np(n);
    if (plan_smoothed_sample<double>(p, A, m, n, lda, s, seed, np, info, st) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    launch_colmajor_to_rows(p->As, s, s, n, As, ld_as, st);
    return check_launch();
}

rpcholqr_status rpcholqr_plan_split_pass2_fp64(rpcholqr_plan p, int32_t* used_fp64) {
    if (!p || !used_fp64 || p->mode != RPCHOLQR_SPLIT64) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    return cudaMemcpy(used_fp64, p->gates + 4, sizeof(int32_t), cudaMemcpyDeviceToHost) == cudaSuccess
               ? RPCHOLQR_OK
               : RPCHOLQR_ERR_CUDA;
}

rpcholqr_status rpcholqr_probe_fp64_mma(int device, int32_t iters, double* flops_per_s) {
    if (!flops_per_s || iters < 1) return RPCHOLQR_ERR_ARG;
    DeviceGuard guard(device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    return run_fp64_mma_probe(iters, flops_per_s) == cudaSuccess ? RPCHOLQR_OK : RPCHOLQR_ERR_CUDA;
}

}  // extern "C"
