// rpcholqr_precondition_gram_noalloc: the fused preconditioning + Gram pass without a plan and
// without any device allocation.
//
// Who needs it: callers that must not allocate device memory once they are running -- for
// example code embedded in a framework whose caching allocator owns all device memory, or a
// service that reserves its memory at start-up and forbids cudaMalloc/cudaFree afterwards because
// they synchronise the device and can fail under memory pressure.  Those callers cannot create an
// rpcholqr_plan (plans cudaMalloc their workspace), so this entry point takes its scratch from a
// fixed array in the library's own device memory instead.
//
// The scratch is one file-scope __device__ array sized for n <= kNoAllocMaxN and at most
// kNoAllocMaxCtas CTAs in the row pass (about 5.3 MB).  Every GPU that loads the library keeps it
// until the process exits.  Host code only sees a host-side stand-in for the array's name, so the
// device address is fetched with cudaGetSymbolAddress once per device, on the first call made on
// that device with it current; that first call should therefore happen before any stream
// capture.  All calls share the array: two calls whose kernels overlap on the GPU race on it.
// The call runs on the current device; a stream that belongs to another device is refused
// (RPCHOLQR_ERR_ARG).  Nothing in the array has to start at zero -- every call rewrites the
// fragment tables and every CTA rewrites all Gram tiles the reduction reads.
#include <mutex>

#include "common.cuh"

namespace rpq {
void launch_prep_tri(const double* T, int64_t ldt, int n, int np, double* frag, double* diag,
                     const int32_t* info, cudaStream_t st);
cudaError_t launch_rowpass(bool syrk, int np, const double* X, int64_t ldx, double* Y, int64_t ldy,
                           int64_t m, int n, const double* frag, const double* diag, double* gpart,
                           int32_t* info, int grid, cudaStream_t st);
void launch_gram_reduce(const double* gpart, int nparts, int np, int n, double* G, int64_t ldg,
                        const int32_t* info, cudaStream_t st);

namespace {
constexpr int kNoAllocMaxN = 64;
constexpr int kNoAllocMaxCtas = 160;
constexpr size_t kFragDoubles = static_cast<size_t>(kNoAllocMaxN) * kNoAllocMaxN;
constexpr size_t kDiagDoubles = static_cast<size_t>(kNoAllocMaxN / 8) * 64;
constexpr size_t kPartDoubles = static_cast<size_t>(kNoAllocMaxCtas) * kNoAllocMaxN * kNoAllocMaxN;
// fragment table | diagonal blocks | per-CTA Gram partials (each slice 256-byte aligned)
constexpr size_t kScratchDoubles = kFragDoubles + kDiagDoubles + kPartDoubles;
static_assert(kFragDoubles % 32 == 0 && kDiagDoubles % 32 == 0, "slices must stay 256-byte aligned");
static_assert(rowpass_ctas_per_sm(kNoAllocMaxN, true) == 1,
              "the partial slice holds one Gram partial per CTA of the grid this file launches");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

}  // namespace rpq

using namespace rpq;

extern "C" rpcholqr_status rpcholqr_precondition_gram_noalloc(const double* A, int64_t m, int32_t n,
                                                              int64_t lda, const double* Rs,
                                                              double* A1, int64_t ld1, double* G,
                                                              int32_t* info, void* stream) {
    if (!A || !Rs || !A1 || !G || !info || m < 1 || n < 1 || lda < n || ld1 < n)
        return RPCHOLQR_ERR_ARG;
    if (n > kNoAllocMaxN) return RPCHOLQR_ERR_UNSUPPORTED;  // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RPCHOLQR_ERR_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return RPCHOLQR_ERR_CUDA;
            }
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return RPCHOLQR_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the scratch address above belongs to the current device: a stream of another device is refused
    // (the default-stream handles always name the current device's default stream)
    if (st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread) {
        int stream_dev = -1;
        if (cudaStreamGetDevice(st, &stream_dev) != cudaSuccess) {
            cudaGetLastError();
            return RPCHOLQR_ERR_ARG;
        }
        if (stream_dev != dev) return RPCHOLQR_ERR_ARG;
    }
    if (cudaMemsetAsync(info, 0, sizeof(int32_t), st) != cudaSuccess ||
        cudaMemsetAsync(info + 1, 0xFF, sizeof(int32_t), st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;

    const int np = pad16(n);
    double* frag = scratch;
    double* diag = scratch + kFragDoubles;
    double* gpart = scratch + kFragDoubles + kDiagDoubles;
    launch_prep_tri(Rs, n, n, np, frag, diag, info, st);
    if (cudaGetLastError() != cudaSuccess) return RPCHOLQR_ERR_CUDA;
    // one CTA per panel of the fused pass (256 rows for n <= 64), at most one per SM; the fused pass
    // launches exactly this grid (one CTA per SM, checked in common.cuh), one Gram partial per CTA
    const int64_t panels = (m + rowpass_rows(np) - 1) / rowpass_rows(np);
    int grid = sms < kNoAllocMaxCtas ? sms : kNoAllocMaxCtas;
    if (panels < grid) grid = static_cast<int>(panels);
    if (launch_rowpass(true, np, A, lda, A1, ld1, m, n, frag, diag, gpart, info, grid, st) != cudaSuccess)
        return RPCHOLQR_ERR_CUDA;
    launch_gram_reduce(gpart, grid, np, n, G, n, info, st);
    return cudaGetLastError() == cudaSuccess ? RPCHOLQR_OK : RPCHOLQR_ERR_CUDA;
}
