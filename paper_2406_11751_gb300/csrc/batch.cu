// Batches of independent matrices (include/rpcholqr.h, "batches of independent matrices"): slot
// plans + streams, round-robin dealing with fork/join events, CUDA-graph capture and replay, and an
// autotuner for the number of concurrent slots.
#include <new>
#include <vector>

#include "common.cuh"

struct rpcholqr_batch_s {
    int device = 0;
    int slots = 0;         // allocated slots
    int active = 0;        // slots in use (autotuned)
    std::vector<rpcholqr_plan> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

struct BatchDevice {
    int prev = -1;
    bool ok = true;
    explicit BatchDevice(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~BatchDevice() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void release(rpcholqr_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->joins) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto s : b->streams) if (s) cudaStreamDestroy(s);
    for (auto p : b->plans) if (p) rpcholqr_plan_destroy(p);
    delete b;
}

// Enqueue the whole batch: fork from `stream`, deal matrices round-robin, join back into `stream`.
rpcholqr_status enqueue(rpcholqr_batch_s* b, int32_t count, const double* const* A, const int64_t* m,
                        const int32_t* n, const int64_t* lda, const int32_t* s, const uint64_t* seed,
                        double* const* Q, const int64_t* ldq, double* const* R, int32_t* info,
                        cudaStream_t stream) {
    const int S = b->active;
    if (cudaEventRecord(b->fork, stream) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    for (int k = 0; k < S; ++k)
        if (cudaStreamWaitEvent(b->streams[k], b->fork, 0) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    for (int32_t i = 0; i < count; ++i) {
        const int k = i % S;
        const rpcholqr_status rc = rpcholqr_factor(b->plans[k], A[i], m[i], n[i], lda[i], s[i], seed[i], Q[i],
                                                   ldq[i], R[i], info + 2 * static_cast<int64_t>(i), b->streams[k]);
        if (rc != RPCHOLQR_OK) return rc;
    }
    for (int k = 0; k < S; ++k) {
        if (cudaEventRecord(b->joins[k], b->streams[k]) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
        if (cudaStreamWaitEvent(stream, b->joins[k], 0) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    }
    return RPCHOLQR_OK;
}

rpcholqr_status check_args(rpcholqr_batch_s* b, int32_t count, const double* const* A, const int64_t* m,
                           const int32_t* n, const int64_t* lda, const int32_t* s, const uint64_t* seed,
                           double* const* Q, const int64_t* ldq, double* const* R, int32_t* info) {
    if (!b || count < 0 || (count > 0 && (!A || !m || !n || !lda || !s || !seed || !Q || !ldq || !R || !info)))
        return RPCHOLQR_ERR_ARG;
    return RPCHOLQR_OK;
}

}  // namespace

extern "C" {

rpcholqr_status rpcholqr_batch_create(rpcholqr_batch* batch, int device, rpcholqr_mode mode, int64_t max_m,
                                      int32_t max_n, int32_t max_s, int32_t slots) {
    if (!batch || slots < 1 || slots > 64) return RPCHOLQR_ERR_ARG;
    *batch = nullptr;
    if (mode == RPCHOLQR_FP32) return RPCHOLQR_ERR_UNSUPPORTED;   // batches are FP64 matrices
    BatchDevice guard(device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    auto* b = new (std::nothrow) rpcholqr_batch_s();
    if (!b) return RPCHOLQR_ERR_NOMEM;
    b->device = device;
    b->slots = b->active = slots;
    b->plans.assign(slots, nullptr);
    b->streams.assign(slots, nullptr);
    b->joins.assign(slots, nullptr);
    for (int k = 0; k < slots; ++k) {
        const rpcholqr_status rc = rpcholqr_plan_create(&b->plans[k], device, mode, max_m, max_n, max_s, nullptr);
        if (rc != RPCHOLQR_OK) { release(b); return rc; }
        if (cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->joins[k], cudaEventDisableTiming) != cudaSuccess) {
            release(b);
            return RPCHOLQR_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) { release(b); return RPCHOLQR_ERR_CUDA; }
    *batch = b;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_batch_destroy(rpcholqr_batch batch) {
    if (!batch) return RPCHOLQR_OK;
    BatchDevice guard(batch->device);
    cudaDeviceSynchronize();
    release(batch);
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_batch_factor(rpcholqr_batch b, int32_t count, const double* const* A,
                                        const int64_t* m, const int32_t* n, const int64_t* lda,
                                        const int32_t* s, const uint64_t* seed, double* const* Q,
                                        const int64_t* ldq, double* const* R, int32_t* info, void* stream) {
    rpcholqr_status rc = check_args(b, count, A, m, n, lda, s, seed, Q, ldq, R, info);
    if (rc != RPCHOLQR_OK) return rc;
    BatchDevice guard(b->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    return enqueue(b, count, A, m, n, lda, s, seed, Q, ldq, R, info, static_cast<cudaStream_t>(stream));
}

rpcholqr_status rpcholqr_batch_capture(rpcholqr_batch b, int32_t count, const double* const* A,
                                       const int64_t* m, const int32_t* n, const int64_t* lda,
                                       const int32_t* s, const uint64_t* seed, double* const* Q,
                                       const int64_t* ldq, double* const* R, int32_t* info, void* stream) {
    rpcholqr_status rc = check_args(b, count, A, m, n, lda, s, seed, Q, ldq, R, info);
    if (rc != RPCHOLQR_OK) return rc;
    BatchDevice guard(b->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cap);
        return RPCHOLQR_ERR_CUDA;
    }
    rc = enqueue(b, count, A, m, n, lda, s, seed, Q, ldq, R, info, cap);
    cudaGraph_t g = nullptr;
    const cudaError_t end = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != RPCHOLQR_OK || end != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != RPCHOLQR_OK ? rc : RPCHOLQR_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return RPCHOLQR_ERR_CUDA;
    }
    b->graph = g;
    (void)stream;
    return RPCHOLQR_OK;
}

rpcholqr_status rpcholqr_batch_replay(rpcholqr_batch b, void* stream) {
    if (!b || !b->exec) return RPCHOLQR_ERR_ARG;
    BatchDevice guard(b->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RPCHOLQR_OK
                                                                                     : RPCHOLQR_ERR_CUDA;
}

rpcholqr_status rpcholqr_batch_autotune(rpcholqr_batch b, int32_t count, const double* const* A,
                                        const int64_t* m, const int32_t* n, const int64_t* lda,
                                        const int32_t* s, const uint64_t* seed, double* const* Q,
                                        const int64_t* ldq, double* const* R, int32_t* info, int32_t reps,
                                        int32_t* best_slots, float* best_ms, void* stream) {
    rpcholqr_status rc = check_args(b, count, A, m, n, lda, s, seed, Q, ldq, R, info);
    if (rc != RPCHOLQR_OK || reps < 1 || !best_slots || !best_ms) return RPCHOLQR_ERR_ARG;
    BatchDevice guard(b->device);
    if (!guard.ok) return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    float best = -1.f;
    int best_s = b->slots;
    for (int S = 1; S <= b->slots; S *= 2) {
        b->active = S;
        if ((rc = enqueue(b, count, A, m, n, lda, s, seed, Q, ldq, R, info, st)) != RPCHOLQR_OK) break;  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == RPCHOLQR_OK; ++r) rc = enqueue(b, count, A, m, n, lda, s, seed, Q, ldq, R, info, st);
        cudaEventRecord(e1, st);
        if (rc != RPCHOLQR_OK || cudaEventSynchronize(e1) != cudaSuccess) { rc = rc != RPCHOLQR_OK ? rc : RPCHOLQR_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (best < 0.f || ms < best) { best = ms; best_s = S; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->active = best_s;
    *best_slots = best_s;
    *best_ms = best;
    return rc;
}

}  // extern "C"
