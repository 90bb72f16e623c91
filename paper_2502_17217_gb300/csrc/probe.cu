// jfnk_measure_fp64_rate: the device's sustained FP64 FMA throughput, measured with independent
// FMA chains in every thread of a full grid (the ceiling of the FP64-bound residual and
// Arnoldi kernels on GB300, reported beside the derived unit-count figure).
#include "jfnk_internal.h"

namespace {

constexpr int kChains = 8, kIters = 4096;

__global__ void k_fp64_chains(double* out, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < kIters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int jfnk_measure_fp64_rate(int device, double* tflops)
{
    if (!tflops) return JFNK_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return JFNK_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 256, blocks = sms * 8;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * (size_t)threads * blocks) != cudaSuccess) return JFNK_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fp64_chains<<<blocks, threads>>>(out, 0.999, 1e-3);  // warm-up
    cudaEventRecord(e0);
    k_fp64_chains<<<blocks, threads>>>(out, 0.999, 1e-3);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.0f) return JFNK_ECUDA;
    *tflops = 2.0 * (double)threads * blocks * kIters * kChains / (ms * 1e-3) / 1e12;
    return JFNK_OK;
}
