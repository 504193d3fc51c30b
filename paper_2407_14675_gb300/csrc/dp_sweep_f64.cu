// Sweep kernels with double geometry and double values.
#include "dp_sweep.cuh"

namespace dpk {

cudaError_t launch_sweep(const SweepLaunch<double, double>& L)
{
    if (L.dyn == kDynUnitSpeed) {
        if (L.reduced) return cudaErrorInvalidValue;
        return launch_mode<double, double, kDynUnitSpeed, false>(L);
    }
    if (L.dyn == kDynPolar) {
        if (L.reduced) return cudaErrorInvalidValue;
        return launch_mode<double, double, kDynPolar, false>(L);
    }
    if (L.reduced) return launch_mode<double, double, kDynOrbit, true>(L);
    return launch_mode<double, double, kDynOrbit, false>(L);
}

}  // namespace dpk
