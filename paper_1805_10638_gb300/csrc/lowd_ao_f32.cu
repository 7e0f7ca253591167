// Assignment-only low-d pass kernels (no update bins, no bounds: the standalone assignment and energy
// calls), float instantiations, one kernel per d.
#include "lowd_pass.cuh"
#include "lowd_inst.cuh"

namespace km {

#define KM_LAUNCH(DD) \
    case DD:          \
        return launch_one_ao<float, DD>(a, nb, smem, s);
#define KM_OCC(DD) \
    case DD:       \
        return pass_occ_ao<float, DD>(smem);

cudaError_t lowd_launch_f32_ao(const PassArgs& a, int d, int nb, size_t smem, cudaStream_t s)
{
    switch (d) {
        KM_FOR_EACH_D(KM_LAUNCH)
        default:
            return cudaErrorInvalidValue;
    }
}

int lowd_occupancy_f32_ao(int d, size_t smem)
{
    switch (d) {
        KM_FOR_EACH_D(KM_OCC)
        default:
            return 1;
    }
}

}  // namespace km
