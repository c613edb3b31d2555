// Batches of independent tall-skinny matrices in ONE persistent kernel launch (rpcholqr_factor_batched):
// Algorithm alg_2 (Section 4) for every matrix of the batch, FP64 arithmetic, n <= 128.  The workload is
// that of block-Krylov and LOBPCG solvers, which orthogonalise many blocks of uneven size (Section 1).
//
// A one-CTA setup kernel reads the device-resident shape arrays, checks every shape against the plan
// (ERR_ARG for a matrix that does not fit), orders the matrices by decreasing cost m n^2 (largest first,
// so that the longest chains start first) and writes a work list of items in four sections:
//   SKETCH(i)     sample + gather + scale (Remark r_exp), Householder QR of the sample, fragment tables
//                 of R_s; zeroes the matrix's Gram accumulator;                        signals done0[i]
//   PASS1(i, b)   A1 = A R_s^{-1} on the panels b, b + P_i, b + 2 P_i, ... (P_i parts) into Q, and the
//                 Gram partial of those panels, added into the accumulator when turn[i] == b, so the
//                 parts are summed in the order b = 0, 1, ...;                          turn[i] = b + 1
//   CHOL(i)       waits turn[i] == P_i; Cholesky G1 = R1^T R1, fragment tables of R1, R = R1 R_s;
//                                                                                         done2[i] = 1
//   PASS2(i, b)   Q = A1 R1^{-1} in place on the same panels; waits done2[i].
// The persistent kernel's CTAs (one per SM) take items from the list in order with one atomic counter.
// An item only waits for items earlier in the list, which running CTAs took before it, so the waits
// always end (no CTA needs another to be resident); the launch is still cooperative, so every CTA is
// resident.  Every wait is bounded by the plan's spin limit (with a short sleep between polls): a wait
// that gives up sets RPCHOLQR_ERR_TIMEOUT for its matrix, and the items after it skip the matrix's
// work but still pass its counters on, so no other wait depends on the one that gave up.
//
// Bits: P_i is the single call's pass-1 grid (one CTA per 128-row panel, at most one per SM), the
// panels of part b are those CTA b of the single call solves, each part's Gram partial is accumulated
// by the same code, and the parts are summed in the single call's order; the sample, the Householder
// QR (the cluster kernel's per-column arithmetic is the same for one CTA of the same size), the
// Cholesky factorisation (the same virtual-thread layout), the fragment tables and R = R1 R_s are the
// same device functions.  So every matrix's Q, R and status are bit-identical to rpcholqr_factor on
// an FP64 plan, whatever else is in the batch.
#include <algorithm>

#include "philox.cuh"
#include "rowpass.cuh"
#include "smallfactor.cuh"

namespace rpq {
namespace {

constexpr int kPThreads = kClusterQrThreads;   // the Householder QR's bits are those of 256-thread CTAs
constexpr int kBatchMaxNP = 128;
constexpr int kPanelRowsForParts = 128;        // the single call sizes its pass-1 grid by 128-row panels

enum : int { kItemSketch = 0, kItemPass1 = 1, kItemChol = 2, kItemPass2 = 3 };

struct BatchArgs {
    int32_t count;
    const double* const* A;
    const int64_t* m;
    const int32_t* n;
    const int64_t* lda;
    const int32_t* s;
    const uint64_t* seed;
    double* const* Q;
    const int64_t* ldq;
    double* const* R;
    int32_t* info;
    // workspace (see batch_layout)
    double* mats;
    int64_t mat_stride;    // doubles per matrix
    int64_t off_rs, off_r1, off_g, off_frag_s, off_frag_1, off_diag_s, off_diag_1;   // within a matrix
    int32_t* ctr;          // 4 per matrix: done0, turn, done2, parts
    int32_t* order;        // count: matrices by decreasing cost
    int64_t* pre;          // count + 1: prefix sums of parts in that order
    uint64_t* items;
    int32_t* queue;        // [0] next item, [1] number of items, [2] abort (a wait gave up)
    // limits and options
    int64_t max_m;
    int32_t max_n, max_s, sms, scale_sample;
    long spin;
};

__host__ __device__ inline uint64_t item_code(int type, int i, int64_t b) {
    return (static_cast<uint64_t>(type) << 62) | (static_cast<uint64_t>(i) << 32) | static_cast<uint64_t>(b);
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 polls *flag until it reaches `target` (at most `limit` polls, sleeping between them); the
// outcome is shared through *ok_s.  Every thread of the CTA calls this.  A wait that gives up raises the
// launch's abort word, after which every other wait gives up at its next poll: one failed dependency
// costs the launch one bounded wait, not one per item.
__device__ __forceinline__ bool cta_wait_geq(const int32_t* flag, int target, long limit, int* ok_s,
                                             int32_t* abort) {
    if (threadIdx.x == 0) {
        int ok = 0;
        for (long it = 0; it < limit; ++it) {
            if (ld_acquire(flag) >= target) { ok = 1; break; }
            if (*reinterpret_cast<volatile int32_t*>(abort)) break;
            __nanosleep(it < 32 ? 64 : 512);
        }
        if (!ok) atomicExch(abort, 1);
        *ok_s = ok;
    }
    __syncthreads();
    const bool ok = *ok_s != 0;
    __syncthreads();
    return ok;
}

// Publishes everything the CTA wrote, then raises *flag to at least `value` (counters never go back).
__device__ __forceinline__ void cta_signal(int32_t* flag, int value) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicMax(flag, value);
    }
}

struct MatWs {
    double *As, *Rs, *R1, *G, *frag_s, *frag_1, *diag_s, *diag_1;
};
__device__ __forceinline__ MatWs mat_ws(const BatchArgs& a, int i) {
    double* base = a.mats + static_cast<int64_t>(i) * a.mat_stride;
    return {base, base + a.off_rs, base + a.off_r1, base + a.off_g, base + a.off_frag_s, base + a.off_frag_1,
            base + a.off_diag_s, base + a.off_diag_1};
}

__global__ void __launch_bounds__(1024) k_batch_setup(BatchArgs a) {
    __shared__ int nvalid_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < a.count; i += nt) {
        const int64_t m = a.m[i];
        const int n = a.n[i], s = a.s[i];
        const bool ok = a.A[i] && a.Q[i] && a.R[i] && n >= 1 && n <= a.max_n && s >= n && s <= a.max_s &&
                        m >= s && m <= a.max_m && a.lda[i] >= n && a.ldq[i] >= n;
        a.info[2 * i] = ok ? 0 : RPCHOLQR_ERR_ARG;
        a.info[2 * i + 1] = -1;
        int parts = 0;
        if (ok) {
            const int64_t panels = (m + kPanelRowsForParts - 1) / kPanelRowsForParts;
            parts = static_cast<int>(panels < a.sms ? panels : a.sms);
        }
        a.ctr[4 * i + 0] = 0;
        a.ctr[4 * i + 1] = 0;
        a.ctr[4 * i + 2] = 0;
        a.ctr[4 * i + 3] = parts;
    }
    __syncthreads();
    // rank by decreasing cost (ties by index); matrices that do not fit (cost -1) come last
    for (int i = tid; i < a.count; i += nt) {
        auto cost = [&](int j) {
            return a.ctr[4 * j + 3] > 0 ? static_cast<double>(a.m[j]) * a.n[j] * a.n[j] : -1.0;
        };
        const double ci = cost(i);
        int rank = 0;
        for (int j = 0; j < a.count; ++j) {
            const double cj = cost(j);
            rank += (cj > ci || (cj == ci && j < i)) ? 1 : 0;
        }
        a.order[rank] = i;
    }
    __syncthreads();
    if (tid == 0) {
        int64_t acc = 0;
        int nv = 0;
        for (int r = 0; r < a.count; ++r) {
            a.pre[r] = acc;
            const int p = a.ctr[4 * a.order[r] + 3];
            acc += p;
            nv += p > 0 ? 1 : 0;
        }
        a.pre[a.count] = acc;
        a.queue[0] = 0;
        a.queue[1] = static_cast<int32_t>(2 * nv + 2 * acc);
        a.queue[2] = 0;
        nvalid_s = nv;
    }
    __syncthreads();
    const int nv = nvalid_s;
    const int64_t P = a.pre[a.count];
    const int64_t base1 = nv, base2 = nv + P, base3 = 2 * static_cast<int64_t>(nv) + P;
    for (int r = tid; r < nv; r += nt) {
        a.items[r] = item_code(kItemSketch, a.order[r], 0);
        a.items[base2 + r] = item_code(kItemChol, a.order[r], 0);
    }
    for (int64_t k = tid; k < P; k += nt) {
        int lo = 0, hi = nv - 1;   // the rank r with pre[r] <= k < pre[r + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (a.pre[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const int64_t b = k - a.pre[lo];
        a.items[base1 + k] = item_code(kItemPass1, a.order[lo], b);
        a.items[base3 + k] = item_code(kItemPass2, a.order[lo], b);
    }
}

// ---- the four item kinds ----------------------------------------------------------------------------
__device__ void item_sketch(const BatchArgs& a, int i, double* psm) {
    const MatWs w = mat_ws(a, i);
    const int n = a.n[i], s = a.s[i], np = pad16(n);
    const int64_t m = a.m[i], lda = a.lda[i];
    const double* A = a.A[i];
    int32_t* info = a.info + 2 * i;
    const int tid = threadIdx.x;
    for (int e = tid; e < np * np; e += kPThreads) w.G[e] = 0.0;
    // sample rows (Philox, stream 0), then A_s = scale * A[idx, :] column-major (ld s)
    int64_t* rows = reinterpret_cast<int64_t*>(psm);
    for (int j = tid; j < s; j += kPThreads) rows[j] = sample_row(a.seed[i], 0, m, j);
    __syncthreads();
    const double scale = a.scale_sample ? sqrt(static_cast<double>(m) / static_cast<double>(s)) : 1.0;
    bool bad = false;
    for (int e = tid; e < np * s; e += kPThreads) {
        const int c = e / s, j = e - c * s;
        double v = 0.0;
        if (c < n) {
            const double x = A[rows[j] * lda + c];
            bad |= !isfinite(x);
            v = scale * x;
        }
        w.As[static_cast<int64_t>(c) * s + j] = v;
    }
    if (__syncthreads_or(bad) && tid == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
    __syncthreads();
    if (load_status(info) == 0) hh_factor<false>(w.As, s, s, n, np, w.Rs, nullptr, info, 0u, 1u, psm);
    __syncthreads();
    if (load_status(info) == 0)
        for (int e = tid; e < np * np + (np / 8) * 64; e += kPThreads)
            prep_tri_entry(w.Rs, np, n, np, w.frag_s, w.diag_s, e);
    cta_signal(&a.ctr[4 * i + 0], 1);
}

template <int NP, bool SYRK, class BeforeEmit, class Emit>
__device__ __forceinline__ bool item_rows(const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m, int n,
                                          const double* frag, const double* diag, bool check, int64_t part,
                                          int64_t parts, double* psm, BeforeEmit before, Emit emit) {
    return rowpass_panels<NP, SYRK, rowpass_warps(NP) * 32 == kPThreads, false>(
        X, ldx, Y, ldy, m, n, frag, diag, check, nullptr, 0, nullptr, part, parts, psm, before, emit);
}

template <bool SYRK, class BeforeEmit, class Emit>
__device__ __forceinline__ bool item_rows_np(int np, const double* X, int64_t ldx, double* Y, int64_t ldy, int64_t m,
                                             int n, const double* frag, const double* diag, bool check, int64_t part,
                                             int64_t parts, double* psm, BeforeEmit before, Emit emit) {
    switch (np) {
#define RPQ_NP(V) \
    case V: return item_rows<V, SYRK>(X, ldx, Y, ldy, m, n, frag, diag, check, part, parts, psm, before, emit);
        RPQ_NP(16) RPQ_NP(32) RPQ_NP(48) RPQ_NP(64) RPQ_NP(80) RPQ_NP(96) RPQ_NP(112) RPQ_NP(128)
#undef RPQ_NP
        default: return false;
    }
}

__device__ void item_pass1(const BatchArgs& a, int i, int64_t b, double* psm, int* ok_s, int* go_s) {
    const MatWs w = mat_ws(a, i);
    int32_t* info = a.info + 2 * i;
    int32_t* turn = &a.ctr[4 * i + 1];
    const int parts = a.ctr[4 * i + 3];
    const int n = a.n[i], np = pad16(n);
    if (!cta_wait_geq(&a.ctr[4 * i + 0], 1, a.spin, ok_s, a.queue + 2) && threadIdx.x == 0)
        set_status(info, RPCHOLQR_ERR_TIMEOUT);
    __syncthreads();
    // wait for this part's turn to add its Gram partial (parts are summed in the order b = 0, 1, ...)
    auto before = [&] {
        if (!cta_wait_geq(turn, static_cast<int>(b), a.spin, ok_s, a.queue + 2) && threadIdx.x == 0)
            set_status(info, RPCHOLQR_ERR_TIMEOUT);
        __syncthreads();
        if (threadIdx.x == 0) *go_s = load_status(info) == 0;
        __syncthreads();
    };
    double* G = w.G;
    auto emit = [&](int pr, int pc, double v) {
        if (*go_s) G[pr * np + pc] += v;
    };
    bool bad = false;
    if (load_status(info) == 0) {
        bad = item_rows_np<true>(np, a.A[i], a.lda[i], a.Q[i], a.ldq[i], a.m[i], n, w.frag_s, w.diag_s, true, b,
                                 parts, psm, before, emit);
    } else {
        before();   // keep the turns moving for the parts after this one
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(info, RPCHOLQR_ERR_NONFINITE);
    cta_signal(turn, static_cast<int>(b) + 1);
}

__device__ void item_chol(const BatchArgs& a, int i, double* psm, int* ok_s) {
    const MatWs w = mat_ws(a, i);
    int32_t* info = a.info + 2 * i;
    const int parts = a.ctr[4 * i + 3];
    const int n = a.n[i], np = pad16(n);
    if (!cta_wait_geq(&a.ctr[4 * i + 1], parts, a.spin, ok_s, a.queue + 2) && threadIdx.x == 0)
        set_status(info, RPCHOLQR_ERR_TIMEOUT);
    __syncthreads();
    if (load_status(info) == 0 && cholesky_small<kPThreads>(w.G, np, n, np, w.R1, nullptr, info, psm)) {
        __syncthreads();
        for (int e = threadIdx.x; e < np * np + (np / 8) * 64; e += kPThreads)
            prep_tri_entry(w.R1, np, n, np, w.frag_1, w.diag_1, e);
        double* R = a.R[i];
        for (int e = threadIdx.x; e < n * n; e += kPThreads) {
            const int r = e / n, c = e - r * n;
            R[e] = triu_mul_entry(w.R1, np, w.Rs, np, r, c);
        }
    }
    cta_signal(&a.ctr[4 * i + 2], 1);
}

__device__ void item_pass2(const BatchArgs& a, int i, int64_t b, double* psm, int* ok_s) {
    const MatWs w = mat_ws(a, i);
    int32_t* info = a.info + 2 * i;
    const int parts = a.ctr[4 * i + 3];
    const int n = a.n[i], np = pad16(n);
    if (!cta_wait_geq(&a.ctr[4 * i + 2], 1, a.spin, ok_s, a.queue + 2) && threadIdx.x == 0)
        set_status(info, RPCHOLQR_ERR_TIMEOUT);
    __syncthreads();
    if (load_status(info) == 0) {
        double* Q = a.Q[i];
        item_rows_np<false>(np, Q, a.ldq[i], Q, a.ldq[i], a.m[i], n, w.frag_1, w.diag_1, false, b, parts, psm,
                            [] {}, [](int, int, double) {});
    }
}

__global__ void __launch_bounds__(kPThreads, 1) k_batch_persistent(BatchArgs a) {
    extern __shared__ __align__(16) double psm[];
    __shared__ uint64_t item_s;
    __shared__ int ok_s, go_s;
    const int total = a.queue[1];
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(&a.queue[0], 1);
            item_s = it < total ? a.items[it] : ~0ull;
        }
        __syncthreads();
        const uint64_t item = item_s;
        __syncthreads();
        if (item == ~0ull) break;
        const int type = static_cast<int>(item >> 62);
        const int i = static_cast<int>((item >> 32) & 0x3FFFFFFFu);
        const int64_t b = static_cast<int64_t>(item & 0xFFFFFFFFu);
        switch (type) {
            case kItemSketch: item_sketch(a, i, psm); break;
            case kItemPass1: item_pass1(a, i, b, psm, &ok_s, &go_s); break;
            case kItemChol: item_chol(a, i, psm, &ok_s); break;
            default: item_pass2(a, i, b, psm, &ok_s); break;
        }
        __syncthreads();
    }
}

}  // namespace

// ---- host side ------------------------------------------------------------------------------------------
struct BatchLayout {
    int64_t mat_stride, off_rs, off_r1, off_g, off_frag_s, off_frag_1, off_diag_s, off_diag_1;
    size_t mats_bytes, ctr_off, order_off, pre_off, items_off, queue_off, total;
    int64_t max_items;
};

static int64_t round32(int64_t x) { return (x + 31) / 32 * 32; }

BatchLayout batch_layout(int32_t capacity, int32_t max_n, int32_t max_s, int sms) {
    BatchLayout L{};
    const int64_t np = pad16(max_n), nn = np * np, dg = (np / 8) * 64;
    int64_t off = round32(static_cast<int64_t>(max_s) * np);
    L.off_rs = off; off += round32(nn);
    L.off_r1 = off; off += round32(nn);
    L.off_g = off; off += round32(nn);
    L.off_frag_s = off; off += round32(nn);
    L.off_frag_1 = off; off += round32(nn);
    L.off_diag_s = off; off += round32(dg);
    L.off_diag_1 = off; off += round32(dg);
    L.mat_stride = off;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    L.mats_bytes = al(sizeof(double) * static_cast<size_t>(off) * capacity);
    L.max_items = static_cast<int64_t>(capacity) * (2 + 2 * static_cast<int64_t>(sms));
    size_t o = L.mats_bytes;
    L.ctr_off = o; o = al(o + sizeof(int32_t) * 4 * capacity);
    L.order_off = o; o = al(o + sizeof(int32_t) * capacity);
    L.pre_off = o; o = al(o + sizeof(int64_t) * (capacity + 1));
    L.items_off = o; o = al(o + sizeof(uint64_t) * L.max_items);
    L.queue_off = o; o = al(o + sizeof(int32_t) * 4);
    L.total = o;
    return L;
}

size_t batch_smem_bytes(int32_t max_n, int32_t max_s) {
    const int npm = pad16(max_n);
    size_t b = 0;
    for (int np = 16; np <= npm; np += 16) b = std::max(b, rowpass_smem_bytes(np));
    b = std::max(b, static_cast<size_t>(npm + kCholParts) * npm * sizeof(double));
    b = std::max(b, static_cast<size_t>(max_s + max_n + 34) * sizeof(double));
    b = std::max(b, static_cast<size_t>(max_s) * sizeof(int64_t));
    return b;
}

int batch_max_np() { return kBatchMaxNP; }

// Sets the persistent kernel's shared-memory limit for these plan limits and returns its grid (one CTA
// per SM times the CTAs an SM holds) in *grid.  Called once per workspace, outside any stream capture.
cudaError_t prepare_batch_persistent(int32_t max_n, int32_t max_s, int sms, int* grid) {
    const size_t smem = batch_smem_bytes(max_n, max_s);
    cudaError_t err = cudaFuncSetAttribute(k_batch_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent, kPThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * per_sm;
    return cudaSuccess;
}

// Launches the setup kernel and the persistent kernel (grid from prepare_batch_persistent) on `st`.
// ws: the batch workspace laid out by batch_layout(capacity, max_n, max_s, sms); count <= capacity.
cudaError_t launch_batch_persistent(int32_t count, const double* const* A, const int64_t* m, const int32_t* n,
                                    const int64_t* lda, const int32_t* s, const uint64_t* seed, double* const* Q,
                                    const int64_t* ldq, double* const* R, int32_t* info, void* ws, int32_t capacity,
                                    int64_t max_m, int32_t max_n, int32_t max_s, int sms, int scale_sample,
                                    long spin, int grid, cudaStream_t st) {
    if (count < 1 || count > capacity || max_n > kBatchMaxNP || grid < 1) return cudaErrorInvalidValue;
    const BatchLayout L = batch_layout(capacity, max_n, max_s, sms);
    char* w = static_cast<char*>(ws);
    BatchArgs a{};
    a.count = count;
    a.A = A; a.m = m; a.n = n; a.lda = lda; a.s = s; a.seed = seed; a.Q = Q; a.ldq = ldq; a.R = R; a.info = info;
    a.mats = reinterpret_cast<double*>(w);
    a.mat_stride = L.mat_stride;
    a.off_rs = L.off_rs; a.off_r1 = L.off_r1; a.off_g = L.off_g; a.off_frag_s = L.off_frag_s;
    a.off_frag_1 = L.off_frag_1; a.off_diag_s = L.off_diag_s; a.off_diag_1 = L.off_diag_1;
    a.ctr = reinterpret_cast<int32_t*>(w + L.ctr_off);
    a.order = reinterpret_cast<int32_t*>(w + L.order_off);
    a.pre = reinterpret_cast<int64_t*>(w + L.pre_off);
    a.items = reinterpret_cast<uint64_t*>(w + L.items_off);
    a.queue = reinterpret_cast<int32_t*>(w + L.queue_off);
    a.max_m = max_m; a.max_n = max_n; a.max_s = max_s; a.sms = sms; a.scale_sample = scale_sample; a.spin = spin;
    k_batch_setup<<<1, 1024, 0, st>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid), 1, 1);
    cfg.blockDim = dim3(kPThreads, 1, 1);
    cfg.dynamicSmemBytes = batch_smem_bytes(max_n, max_s);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    err = cudaLaunchKernelEx(&cfg, k_batch_persistent, a);
    return err == cudaSuccess ? cudaGetLastError() : err;
}

}  // namespace rpq
