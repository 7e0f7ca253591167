// Batched low-d pass kernels, float, the second launch shape the batched autotuner may pick: half
// the rows per thread in the scan (2 for d <= 8, 1 above), one kernel per d.
#include "lowd_pass.cuh"
#include "lowd_inst.cuh"

namespace km {

template <int D>
constexpr int half_rows()
{
    return Shape<D>::R / 2 > 0 ? Shape<D>::R / 2 : 1;
}

#define KM_LAUNCH(DD) \
    case DD:          \
        return launch_batch_one<float, DD, half_rows<DD>()>(b, grid, smem, s);
#define KM_OCC(DD) \
    case DD:       \
        return batch_occ<float, DD, half_rows<DD>()>(smem);

cudaError_t lowd_batch_launch_f32_v1(const BatchPass& b, int d, int grid, size_t smem, cudaStream_t s)
{
    switch (d) {
        KM_FOR_EACH_D(KM_LAUNCH)
        default:
            return cudaErrorInvalidValue;
    }
}

int lowd_batch_occupancy_f32_v1(int d, size_t smem)
{
    switch (d) {
        KM_FOR_EACH_D(KM_OCC)
        default:
            return 1;
    }
}

}  // namespace km
