// Multi-level evaluation sweeps (FP32 geometry and values, frozen feet).
#include "dp_wave.cuh"

namespace dpk {

cudaError_t launch_wave(const WaveArgs& a, int mode, int dyn, int reduced, cudaStream_t st, int sm_count)
{
    if (a.levels < 1 || a.levels > kWaveMaxLevels || !a.feet_lo || !a.sync) return cudaErrorInvalidValue;
    if ((mode == kIncr || mode == kIncrDiag) && (!a.acc || !a.V64)) return cudaErrorInvalidValue;
    if (dyn == kDynPolar) return cudaErrorInvalidValue;   // polar grids are FP64
    if (dyn == kDynUnitSpeed) {
        if (reduced) return cudaErrorInvalidValue;
        return launch_wave_dyn<false, kDynUnitSpeed>(a, mode, st, sm_count);
    }
    if (reduced) return launch_wave_dyn<true, kDynOrbit>(a, mode, st, sm_count);
    return launch_wave_dyn<false, kDynOrbit>(a, mode, st, sm_count);
}

}  // namespace dpk
