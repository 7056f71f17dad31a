// FP64 FMA throughput probe: the denominator of the narrow phase's FP64
// utilisation (no FP64 peak is published for this part in the measured-peaks
// file, so it is measured here).  Each thread runs 8 independent dependent
// chains of fused multiply-adds; the grid fills every SM several times over.
#include <cuda_runtime.h>

#include "tms_common.cuh"

namespace {

__global__ void __launch_bounds__(256) k_fp64_fma(double *out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1.2345) out[blockIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" tms_status tms_probe_fp64(double *tflops, void *stream) {
    if (!tflops) return TMS_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TMS_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *out = nullptr;
    if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) return TMS_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fp64_fma<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);   // warm-up
    cudaEventRecord(e0, st);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_fp64_fma<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return TMS_ERR_CUDA;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return TMS_OK;
}
