// dp_wave.cuh -- several Jacobi evaluation sweeps of policy iteration in one
// launch (FP32 geometry, frozen feet).
//
// With the control frozen, the n_eval evaluation sweeps of modified policy
// iteration (§3, Eq. (13)) apply the same operator V <- b + beta W_f V again
// and again: every sweep streams the same frozen feet and gathers V around
// each node.  One sweep per launch reads the feet and V from DRAM every time.
// Here one persistent launch runs `levels` consecutive sweeps as a wavefront
// over chunks of consecutive nodes: level s of chunk c starts once level s-1
// has finished every chunk that node j of c reads (corners within `reach`
// stored nodes of j, recorded by the improvement sweep that stored the feet)
// and every chunk whose nodes read c's old value (the same range: Jacobi
// double buffering overwrites level s-2's value).  Level s then finds its
// feet and level s-1's values in L2, written a short while before, so DRAM
// sees the feet and V about once per launch instead of once per sweep.  The
// results are bit-identical to `levels` separate sweeps: each node does the
// same arithmetic on the same inputs.
//
// Scheduling.  Work items (level, chunk) are handed out in a fixed order by
// an atomic ticket counter.  The order is by rounds: round rho holds, for
// level s = 0, 1, ..., the window of L chunks [(rho - s) L, (rho - s + 1) L).
// With L at least the dependency distance (in chunks, counter granularity
// included), every item an item waits for has a smaller ticket, so it is held
// by a block that is already running: the item with the smallest unfinished
// ticket never waits, and the launch cannot deadlock, whatever the number of
// resident blocks.  Completion is counted per level and per group of G chunks;
// a block that finished a chunk publishes it with a fence and an atomic add
// (release), a block about to start one polls the counters of its range and
// fences (acquire).  Every wait is bounded (kWaveTimeoutNs, 2 s): past it the
// block sets ctl->wave_err, every other block gives up at its next poll, and
// the host reports DP_ETIMEOUT.
#pragma once

#include <algorithm>

#include "dp_sweep.cuh"

namespace dpk {

struct WaveSched {
    int nC;       // chunks per level
    int levels;
    int Dr;       // reach in chunks: chunk c reads (and is read by) chunks c - Dr .. c + Dr
    int G;        // chunks per completion counter
    int L;        // chunks per window
    int nW;       // windows per level
    __device__ __forceinline__ int count(int rho, int s) const
    {
        const int w = rho - s;
        if (w < 0 || w >= nW) return 0;
        return min(L, nC - w * L);
    }
    __device__ __forceinline__ int round_count(int rho) const
    {
        int c = 0;
        for (int s = 0; s < levels; ++s) c += count(rho, s);
        return c;
    }
};

// The schedule of a launch: every thread computes the same one.  reach <= 0
// (not recorded) is treated as the whole grid, which serialises the levels.
__device__ __forceinline__ WaveSched wave_sched(int n_nodes, int levels, int reach, int blocks)
{
    WaveSched S;
    S.nC = (n_nodes + kWaveChunk - 1) / kWaveChunk;
    S.levels = levels;
    const long long R = reach > 0 ? reach : n_nodes;
    S.Dr = (int)min((R + kWaveChunk - 1) / kWaveChunk, (long long)S.nC);
    // at most 32 counters per range (one per lane of the polling warp)
    S.G = max(1, (2 * S.Dr + 29) / 30);
    const int dist = S.Dr + S.G - 1;          // farthest chunk a wait can cover
    // enough slack that a dependency lies about a resident wave of tickets back
    const int slack = max(0, (blocks - dist + 1) / 2) + 1;
    S.L = max(1, min(S.nC, dist + slack));
    S.nW = (S.nC + S.L - 1) / S.L;
    return S;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile(const int* p)
{
    return *(const volatile int*)p;
}

// Blend at a frozen foot of kind kFootInside with coherent corner loads (the
// values were written by other blocks of this launch): eval_foot's
// arithmetic, either foot format.
template <bool REDUCED, typename W>
__device__ __forceinline__ float eval_foot_coherent(const Geo<float>& g, const float* V, int j, W w, float vj)
{
    const FootCell f = foot_cell_of(g, w);
    int base[4];
    foot_rows<REDUCED>(g, j, f.dr, f.dv, f.dt, base);
    Corners<float> K;
    load_rows_f32<true>(V, base, g.n_m, vj, K);
    return K.blend(f.t);
}

// Q1 interpolation at node j's foot for a policy code, coherent loads:
// D = I[V] - vj (M - vj outside; with ZERO_OUT, 0 outside and on target
// nodes, for increments).  *wself: the node's own weight among the corners.
// interp_delta's arithmetic.
template <bool REDUCED, int DYN, bool ZERO_OUT>
__device__ __noinline__ float recompute_coherent(const Geo<float>& g, const float* V, int j, int code, float vj,
                                                  float* wself)
{
    NodeEval<float, float, REDUCED, DYN> ev;
    decode_node(g, j, ev.i);
    *wself = 0.0f;
    if (ZERO_OUT && in_target(g, ev.i)) return 0.0f;
    setup_node<float, float, DYN>(ev, g, V, vj);
    float s, c, u[4], t[4];
    int cl[4], base[4];
    code_sincos(g, code, s, c);
    heun_cells<float, DYN>(g, ev.sp, ev.nd, s, c, u);
#pragma unroll
    for (int d = 0; d < 4; ++d) u[d] += ev.u0[d];
    if (foot_cell(g, ev.i, u, cl, t) || cell_rows<float, REDUCED>(g, cl, base))
        return ZERO_OUT ? 0.0f : (float)((float)g.M64 - vj);
    Corners<float> K;
    load_rows_f32<true>(V, base, g.n_m, vj, K);
    *wself = self_weight<float, false>(g, ev.i, cl, t);
    return K.blend(t);
}


template <int MODE, bool REDUCED, int DYN>
__global__ void __launch_bounds__(kWaveBlock, 3) wave_kernel(const __grid_constant__ WaveArgs a)
{
    constexpr bool kDiag = MODE == kEvalFeetDiag || MODE == kIncrDiag;
    constexpr bool kInc = MODE == kIncr || MODE == kIncrDiag;
    const Geo<float>& g = a.g;
    Ctl* ctl = a.ctl;
    if (ld_volatile(&ctl->stop)) return;
    if (a.check_prev) {
        unsigned long long bits = *(volatile unsigned long long*)&a.ring[(a.sweep - 1) & a.ring_mask];
        if (__longlong_as_double((long long)bits) < a.tol) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                ctl->stop_sweep = (int)a.sweep;
                ctl->stop = 1;
            }
            return;
        }
    }
    // the schedule and the ticket cursor live in shared memory (warp 0 uses
    // them), keeping the node loop's registers free
    __shared__ WaveSched s_S;
    __shared__ long long s_base;
    __shared__ int s_rho, s_rc, s_next, s_item[2];
    __shared__ float s_red[kWaveBlock / 32];
    int* tickets = a.sync;
    int* done = a.sync + 1;                 // done[level * nC + chunk / G]
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_S = wave_sched(g.n_nodes, a.levels, ld_volatile(&ctl->reach), gridDim.x);
        s_rho = 0;
        s_base = 0;
        s_rc = s_S.round_count(0);
        s_next = atomicAdd(tickets, 1);
    }
    __syncthreads();

    for (;;) {
        if (threadIdx.x < 32) {
            const WaveSched& S = s_S;
            int lev = -1, c = 0;
            if (lane == 0) {
                const long long t = s_next;
                if (t < (long long)a.levels * S.nC) {
                    s_next = atomicAdd(tickets, 1);     // the next ticket, while this one runs
                    int rho = s_rho, rc = s_rc;
                    long long base = s_base;
                    while (t >= base + rc) {
                        base += rc;
                        rc = S.round_count(++rho);
                    }
                    s_rho = rho;
                    s_rc = rc;
                    s_base = base;
                    int off = (int)(t - base), sl = 0;
                    for (;;) {
                        const int k = S.count(rho, sl);
                        if (off < k) break;
                        off -= k;
                        ++sl;
                    }
                    lev = sl;
                    c = (rho - sl) * S.L + off;
                }
            }
            lev = __shfl_sync(0xffffffffu, lev, 0);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (lev > 0) {
                // wait for level lev - 1 on chunks c - Dr .. c + Dr
                const int sb_lo = max(0, c - S.Dr) / S.G, sb_hi = min(S.nC - 1, c + S.Dr) / S.G;
                const int sb = sb_lo + lane;
                const int need = sb <= sb_hi ? min(S.G, S.nC - sb * S.G) : 0;
                const int* cnt = done + (long long)(lev - 1) * S.nC + sb;
                unsigned long long t0 = 0;
                for (int poll = 0;; ++poll) {
                    const bool ok = need == 0 || ld_volatile(cnt) >= need;
                    if (__all_sync(0xffffffffu, ok)) break;
                    if (ld_volatile(&ctl->wave_err)) {
                        lev = -2;
                        break;
                    }
                    const unsigned long long now = global_ns();
                    if (poll == 0) t0 = now;
                    else if (now - t0 > a.timeout_ns) {
                        if (lane == 0) atomicOr(&ctl->wave_err, 1);
                        lev = -2;
                        break;
                    }
                    __nanosleep(128);
                }
                __threadfence();   // acquire: the counted chunks' values before this block's loads
            }
            if (lane == 0) {
                s_item[0] = lev;
                s_item[1] = c;
            }
        }
        __syncthreads();
        const int lev = s_item[0], c = s_item[1];
        if (lev < 0) break;

        const float* Vin = a.V[(a.in0 + lev) & 1];
        float* Vout = a.V[(a.in0 + lev + 1) & 1];
        const int e = a.e0 + lev;
        const bool first = kInc && e == 0, last = kInc && e == a.ne - 1;
        const int j_end = min((c + 1) * kWaveChunk, g.n_nodes);
        float resid = 0.0f;
        bool bad = false;
#pragma unroll 1
        for (int j = c * kWaveChunk + threadIdx.x; j < j_end; j += kWaveBlock) {
            // plain evaluation: 8-byte feet; diagonal-solved evaluation and
            // increments: the word pair
            constexpr bool kF8 = MODE == kEvalFeet8;
            typename std::conditional<kF8, unsigned long long, FootWord>::type w;
            if constexpr (kF8) w = __ldcs(&a.feet_lo[j]);
            else w = FootWord{__ldcs(&a.feet_lo[j]), __ldcs(&a.feet_hi[j])};
            const int kind = foot_kind(w);
            float vnew = 0.0f;
            if constexpr (!kInc) {
                const float vj = ld_coherent(Vin + j);
                float ws = 0.0f;
                if (kind == kFootInside) {
                    if constexpr (kDiag) ws = foot_self_weight(g, w);
                    vnew = bellman_value<float, float>(g, vj, eval_foot_coherent<REDUCED>(g, Vin, j, w, vj));
                } else if (kind == kFootOut) {
                    vnew = bellman_value<float, float>(g, vj, (float)((float)g.M64 - vj));
                } else if (kind == kFootRecompute) {
                    const float D = recompute_coherent<REDUCED, DYN, false>(g, Vin, j, a.code[j], vj, &ws);
                    vnew = bellman_value<float, float>(g, vj, D);
                    if (!kDiag) ws = 0.0f;
                }
                if constexpr (kDiag) {
                    if (kind != kFootTarget) vnew = diag_step(g, vj, vnew, ws);
                }
                Vout[j] = vnew;
                resid = fmaxf(resid, fabsf(vnew - vj));
            } else {
                // increments d' = beta W d at the frozen policy (sweep_nodes'
                // kIncr / kIncrDiag arithmetic)
                float D = 0.0f, ws = 0.0f;
                if (kind == kFootInside) {
                    D = eval_foot_coherent<REDUCED>(g, Vin, j, w, 0.0f);
                    if constexpr (kDiag) ws = foot_self_weight(g, w);
                } else if (kind == kFootRecompute) {
                    D = recompute_coherent<REDUCED, DYN, true>(g, Vin, j, a.code[j], 0.0f, &ws);
                    if (!kDiag) ws = 0.0f;
                }
                if constexpr (kDiag) {
                    const float dj = first ? 0.0f : ld_coherent(Vin + j);
                    const float Dx = first ? D : D - ws * dj;
                    vnew = __fdividef(fmaf(g.beta_hi, Dx, g.beta_lo * Dx), 1.0f - (g.beta_hi + g.beta_lo) * ws);
                } else {
                    vnew = fmaf(g.beta_hi, D, g.beta_lo * D);
                }
                Vout[j] = vnew;
                const float sum = (first ? 0.0f : a.acc[j]) + vnew;
                if (last) a.V64[j] += (double)sum;
                else a.acc[j] = sum;
                resid = fmaxf(resid, fabsf(vnew));
            }
            bad = bad || !isfinite(vnew);
        }
        // residual of this level's chunk, then publish the chunk (release)
        resid = warp_max(resid);
        if (lane == 0) s_red[threadIdx.x >> 5] = resid;
        const bool any_bad = __syncthreads_or(bad);
        if (threadIdx.x < 32) {
            float r = lane < kWaveBlock / 32 ? s_red[lane] : 0.0f;
            r = warp_max(r);
            if (lane == 0) {
                if (any_bad) atomicOr(&ctl->nonfinite, 1);
                atomicMax(&a.ring[(a.sweep + lev) & a.ring_mask],
                          (unsigned long long)__double_as_longlong((double)r));
                __threadfence();
                atomicAdd(&done[(long long)lev * s_S.nC + c / s_S.G], 1);
            }
        }
    }
}

template <int MODE, bool REDUCED, int DYN>
cudaError_t launch_wave_mode(const WaveArgs& a, cudaStream_t st, int sm_count)
{
    auto kern = wave_kernel<MODE, REDUCED, DYN>;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWaveBlock, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const long long chunks = (long long)a.levels * ((a.g.n_nodes + kWaveChunk - 1) / kWaveChunk);
    const long long blocks = std::min<long long>((long long)per_sm * sm_count, chunks);
    cudaError_t e = cudaMemsetAsync(a.sync, 0, wave_sync_ints(a.levels, a.g.n_nodes) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<(int)blocks, kWaveBlock, 0, st>>>(a);
    return cudaGetLastError();
}

template <bool REDUCED, int DYN>
cudaError_t launch_wave_dyn(const WaveArgs& a, int mode, cudaStream_t st, int sm_count)
{
    switch (mode) {
    case kEvalFeet: return launch_wave_mode<kEvalFeet, REDUCED, DYN>(a, st, sm_count);
    case kEvalFeet8: return launch_wave_mode<kEvalFeet8, REDUCED, DYN>(a, st, sm_count);
    case kEvalFeetDiag: return launch_wave_mode<kEvalFeetDiag, REDUCED, DYN>(a, st, sm_count);
    case kIncr: return launch_wave_mode<kIncr, REDUCED, DYN>(a, st, sm_count);
    case kIncrDiag: return launch_wave_mode<kIncrDiag, REDUCED, DYN>(a, st, sm_count);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dpk
