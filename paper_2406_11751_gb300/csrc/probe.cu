// FP64 tensor-pipe throughput probe (the denominator of the FP64 roofline on the running GPU).
// Every warp keeps four independent chains of FP64 mma.sync m16n8k16 in flight; 8 warps per CTA,
// two CTAs per SM, so each SM holds 64 chains (the pipe saturates at about 16).
#include "common.cuh"

namespace rpq {

__global__ void __launch_bounds__(256) k_probe_fp64_mma(double* out, int iters, double seed) {
    double c[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) c[j][q] = threadIdx.x * 1e-3 + q + 0.25 * j;  // distinct chains
    double a[8], b[4];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = seed + q * 1e-9;
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = seed - q * 1e-9;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_f64_16816(c[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) s += c[j][q];
    out[static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

cudaError_t run_fp64_mma_probe(int iters, double* flops_per_s) {
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    const int grid = 2 * sms, block = 256;
    double* out = nullptr;
    if ((err = cudaMalloc(&out, sizeof(double) * grid * block)) != cudaSuccess) return err;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_probe_fp64_mma<<<grid, block>>>(out, iters < 8 ? iters : 8, 0.999);  // warm-up
    cudaEventRecord(e0);
    k_probe_fp64_mma<<<grid, block>>>(out, iters, 0.999);
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) {
        const double flops = 2.0 * 2048.0 * 4.0 * static_cast<double>(iters) * grid * (block / 32);
        *flops_per_s = flops / (static_cast<double>(ms) * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return err;
}

}  // namespace rpq
