// dp_sweep.cuh -- the Jacobi sweep kernel of the semi-Lagrangian scheme.
//
// One launch is one Jacobi sweep V_out = T(V_in) over the stored nodes
// (§3, Eq. (12) value iteration, Eq. (13) policy evaluation, Eq. (14) policy
// improvement).  Grid-stride loop, one thread per node, mass fastest so that
// a warp's 16 corner gathers fall on the same few cache lines.  Each block
// reduces max |V_out - V_in| and folds it into the sweep's FP64 residual slot
// with one atomicMax on the IEEE bit pattern (non-negative doubles order like
// their bits).  A sweep first looks at the previous sweep's residual when the
// host asks it to: if the stopping test passed, it records that and returns
// without touching V, so a queue of sweeps ends at the first converged one.
#pragma once

#include "dp_device.cuh"
#include "dp_host.h"

namespace dpk {

// New value dt + beta w, w = V_j + D.  FP32 storage keeps beta as a sum of two
// floats: its rounding error would otherwise shift the fixed point by
// dt / (1 - beta)^2 * 1e-8.
template <typename G, typename S>
__device__ __forceinline__ S bellman_value(const Geo<G>& g, S vj, G D);
template <>
__device__ __forceinline__ float bellman_value<float, float>(const Geo<float>& g, float vj, float D)
{
    float w = vj + D;
    return fmaf(g.beta_hi, w, fmaf(g.beta_lo, w, g.dt));
}
template <>
__device__ __forceinline__ double bellman_value<float, double>(const Geo<float>& g, double vj, float D)
{
    return g.dt64 + g.beta64 * (vj + (double)D);
}
template <>
__device__ __forceinline__ double bellman_value<double, double>(const Geo<double>& g, double vj, double D)
{
    return g.dt64 + g.beta64 * (vj + D);
}

template <typename S>
__device__ __forceinline__ S warp_max(S v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename G, typename S, int MODE, bool REDUCED, int DYN>
__global__ void __launch_bounds__(kBlock)
sweep_kernel(const __grid_constant__ Geo<G> g, const S* __restrict__ Vin, S* __restrict__ Vout, uint16_t* __restrict__ code,
             Ctl* __restrict__ ctl, unsigned long long* __restrict__ ring, int ring_mask,
             long long sweep, int check_prev, double tol)
{
    if (*(volatile int*)&ctl->stop) return;
    if (check_prev) {
        unsigned long long bits = *(volatile unsigned long long*)&ring[(sweep - 1) & ring_mask];
        if (__longlong_as_double((long long)bits) < tol) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                ctl->stop_sweep = (int)sweep;
                ctl->stop = 1;
            }
            return;
        }
    }

    S resid = (S)0;
    bool bad = false;
    const int stride = gridDim.x * kBlock;
    for (int j = blockIdx.x * kBlock + threadIdx.x; j < g.n_nodes; j += stride) {
        NodeEval<G, S, REDUCED, DYN> ev;
        decode_node(g, j, ev.i);
        const S vj = Vin[j];
        S vnew = (S)0;
        if (!in_target(g, ev.i)) {
            G x[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) x[d] = g.lo[d] + (G)ev.i[d] * g.h[d];
            ev.g = &g;
            ev.V = Vin;
            ev.vj = vj;
            ev.sp.dt = g.dt;
            ev.sp.hdt = g.hdt;
            ev.sp.um = g.um;
#pragma unroll
            for (int d = 0; d < 4; ++d) ev.u0[d] = (G)0;
            ev.nd = node_dyn<G, DYN>(g, ev.sp, x);
            G D;
            if (MODE == kEval) {
                D = ev.at_code(code[j]);
            } else {
                int k;
                if (MODE == kImproveWalk)
                    k = walk_table(ev, g.K, nearest_table_index(g.K, code[j]), D);
                else
                    k = enumerate_table(ev, g.K, D);
                int c = wrap_code(table_code(g.K, k));
                if (MODE != kVI && g.refine) c = fibonacci_refine(ev, g.K, g.fib_stop, k, D, D);
                if (MODE != kVI) code[j] = (uint16_t)c;
            }
            vnew = bellman_value<G, S>(g, vj, D);
        }
        Vout[j] = vnew;
        resid = fmax(resid, (S)fabs(vnew - vj));
        bad = bad || !isfinite(vnew);
    }

    __shared__ S red[kBlock / 32];
    resid = warp_max(resid);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = resid;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->nonfinite, 1);
    if (threadIdx.x < 32) {
        S r = threadIdx.x < kBlock / 32 ? red[threadIdx.x] : (S)0;
        r = warp_max(r);
        if (threadIdx.x == 0)
            atomicMax(&ring[sweep & ring_mask], (unsigned long long)__double_as_longlong((double)r));
    }
}

template <typename G, typename S, int MODE, bool REDUCED, int DYN>
cudaError_t launch_one(const SweepLaunch<G, S>& L)
{
    auto kern = sweep_kernel<G, S, MODE, REDUCED, DYN>;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    long long need = ((long long)L.g.n_nodes + kBlock - 1) / kBlock;
    long long cap = (long long)per_sm * L.sm_count;
    int blocks = (int)(need < cap ? need : cap);
    if (blocks < 1) blocks = 1;
    kern<<<blocks, kBlock, 0, L.stream>>>(L.g, L.Vin, L.Vout, L.code, L.ctl, L.ring, L.ring_mask,
                                          L.sweep, L.check_prev, L.tol);
    return cudaGetLastError();
}

template <typename G, typename S, int DYN, bool REDUCED>
cudaError_t launch_mode(const SweepLaunch<G, S>& L)
{
    switch (L.mode) {
    case kVI: return launch_one<G, S, kVI, REDUCED, DYN>(L);
    case kImproveFull: return launch_one<G, S, kImproveFull, REDUCED, DYN>(L);
    case kImproveWalk: return launch_one<G, S, kImproveWalk, REDUCED, DYN>(L);
    case kEval: return launch_one<G, S, kEval, REDUCED, DYN>(L);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dpk
