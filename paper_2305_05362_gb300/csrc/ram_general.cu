// RAM step on rows with arbitrary (non-uniform) meshes.
#include <cuda_runtime.h>

#include "ram_device.cuh"

namespace ram {

cudaError_t launch_general(const Plan &p, ram_dtype, const StepArgs &, cudaStream_t)
{
    for (int o = 2; o <= 4; ++o)
        if (!p.tiles_general_h[o].empty()) return cudaErrorNotSupported;
    return cudaSuccess;
}

cudaError_t launch_row_mass(const Plan &, ram_dtype, const void *, double *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t launch_adjoint(const Plan &, ram_dtype, const StepArgs &, const void *, void *,
                           void *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace ram
