// Measured FP32 CUDA-core FMA throughput of the device, the peak against which the low-d
// assignment pass (an ALU-bound scan: d FMAs and about two compare/select operations per
// sample-centroid pair) is reported.  A grid of 4 blocks of 256 threads per SM runs independent
// chains of fma.rn.f32 (8 per thread, so the FMA latency is covered) for a fixed number of
// iterations; CUDA events time the launch.  The result is written only if a runtime flag is set,
// which keeps the chains live without storing them.
#include "../../include/kmeans_aa.h"

#include <cuda_runtime.h>

namespace {

constexpr int CAL_THREADS = 256;
constexpr int CAL_CHAINS = 8;

__global__ void __launch_bounds__(CAL_THREADS) k_fma_chains(int iters, float a, float b, int store, float* out)
{
    float v[CAL_CHAINS];
#pragma unroll
    for (int c = 0; c < CAL_CHAINS; ++c) v[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < CAL_CHAINS; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CAL_CHAINS; ++c) s += v[c];
    if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" kmeans_status kmeans_measure_fp32_fma(int device, int iters, double* fma_per_s, double* ms)
{
    if (!fma_per_s || iters < 1) return KM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return KM_ECUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return KM_ECUDA;
    const int grid = nsm * 4;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KM_ECUDA;
    k_fma_chains<<<grid, CAL_THREADS>>>(iters / 4 + 1, 0.999f, 1e-3f, 0, nullptr);   // warm-up
    cudaEventRecord(e0);
    k_fma_chains<<<grid, CAL_THREADS>>>(iters, 0.999f, 1e-3f, 0, nullptr);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return KM_ECUDA;
    *fma_per_s = (double)grid * CAL_THREADS * (double)iters * 16.0 * CAL_CHAINS / (t * 1e-3);
    if (ms) *ms = t;
    return KM_OK;
}
