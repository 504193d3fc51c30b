// Sweep kernels with float geometry and double values.
#include "dp_sweep.cuh"

namespace dpk {

cudaError_t launch_sweep(const SweepLaunch<float, double>& L)
{
    if (L.dyn == kDynPolar) return cudaErrorInvalidValue;   // polar grids are FP64
    if (L.dyn == kDynUnitSpeed) {
        if (L.reduced) return cudaErrorInvalidValue;
        return launch_mode<float, double, kDynUnitSpeed, false>(L);
    }
    if (L.reduced) return launch_mode<float, double, kDynOrbit, true>(L);
    return launch_mode<float, double, kDynOrbit, false>(L);
}

}  // namespace dpk
