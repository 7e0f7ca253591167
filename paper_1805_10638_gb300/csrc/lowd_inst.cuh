// Per-precision entry points of the low-d pass kernels, one instantiation unit each
// (lowd_std_f32.cu, lowd_std_f64.cu, lowd_batch_f32.cu, lowd_batch_f32_v1.cu, lowd_batch_f64.cu),
// dispatched on d (1..16) inside each unit.
#pragma once

#include "km_internal.cuh"

// X(d) for every supported dimension of the low-d path
#define KM_FOR_EACH_D(X) \
    X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

namespace km {

cudaError_t lowd_launch_f32(const PassArgs& a, int d, int nb, size_t smem, cudaStream_t s);
cudaError_t lowd_launch_f64(const PassArgs& a, int d, int nb, size_t smem, cudaStream_t s);
cudaError_t lowd_batch_launch_f32(const BatchPass& b, int d, int grid, size_t smem, cudaStream_t s);
cudaError_t lowd_batch_launch_f64(const BatchPass& b, int d, int grid, size_t smem, cudaStream_t s);
int lowd_occupancy_f32(int d, size_t smem);
int lowd_occupancy_f64(int d, size_t smem);
int lowd_batch_occupancy_f32(int d, size_t smem);
int lowd_batch_occupancy_f64(int d, size_t smem);
// the FP32 pass without update bins and bounds (lowd_ao_f32.cu)
cudaError_t lowd_launch_f32_ao(const PassArgs& a, int d, int nb, size_t smem, cudaStream_t s);
int lowd_occupancy_f32_ao(int d, size_t smem);
// the batched FP32 pass with half the rows per thread in the scan (lowd_batch_f32_v1.cu)
cudaError_t lowd_batch_launch_f32_v1(const BatchPass& b, int d, int grid, size_t smem, cudaStream_t s);
int lowd_batch_occupancy_f32_v1(int d, size_t smem);

}  // namespace km
