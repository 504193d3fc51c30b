// Sweep kernels with float geometry and float values.
#include "dp_sweep.cuh"

namespace dpk {

cudaError_t launch_sweep(const SweepLaunch<float, float>& L)
{
    if (L.dyn == kDynPolar) return cudaErrorInvalidValue;   // polar grids are FP64
    if (L.dyn == kDynUnitSpeed) {
        if (L.reduced) return cudaErrorInvalidValue;
        return launch_mode<float, float, kDynUnitSpeed, false>(L);
    }
    if (L.reduced) return launch_mode<float, float, kDynOrbit, true>(L);
    return launch_mode<float, float, kDynOrbit, false>(L);
}

}  // namespace dpk
