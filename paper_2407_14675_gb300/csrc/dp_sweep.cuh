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
//
// Improvement sweeps with FP32 geometry also store each node's frozen foot
// (cell offsets and fractions of the chosen control: 8 bytes with FP32
// values, 12 with FP64 values).  The evaluation sweeps that follow read it
// (kEvalFeet) and only gather and blend.  With FP64 values the evaluation sweeps run on increments instead
// (kIncr): V_{k+1} - V_k = beta W (V_k - V_{k-1}) at a frozen policy, so the
// increments are swept in FP32 and summed into the FP64 value once.
#pragma once

#include <type_traits>

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
// FP32 geometry with FP64 values: D is blended in FP64.
__device__ __forceinline__ double bellman_value(const Geo<float>& g, double vj, double D)
{
    return g.dt64 + g.beta64 * (vj + D);
}

// State part of the running cost of Eq. (11) (polar dynamics, FP64):
// beta (a - a_bar)^2 + gamma |(e cos w, e sin w) - target|^2, with a from the
// vis-viva relation and (e cos w, e sin w) from the eccentricity vector, whose
// radial and transverse components are r v_t^2 / mu - 1 and -r v_r v_t / mu.
template <typename G>
__device__ __forceinline__ double state_cost_x(const Geo<G>& g, const double x[4])
{
    const double r = x[0], vr = x[1], vt = x[2], mu = (double)g.mu;
    double sn, cs;
    sincos(x[3], &sn, &cs);
    const double a = mu * r / (2.0 * mu - r * (vr * vr + vt * vt));
    const double er = r * vt * vt / mu - 1.0, et = -r * vr * vt / mu;
    const double dx = er * cs - et * sn - g.ex_bar, dy = er * sn + et * cs - g.ey_bar, da = a - g.a_bar;
    return g.cost_b * da * da + g.cost_g * (dx * dx + dy * dy);
}

template <typename G>
__device__ __forceinline__ double state_cost(const Geo<G>& g, const int i[4])
{
    double x[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) x[d] = (double)(g.lo[d] + (G)i[d] * g.h[d]);
    return state_cost_x(g, x);
}

template <typename S>
__device__ __forceinline__ S warp_max(S v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Fills the common fields of an evaluator for grid node ev.i with value vj.
template <typename G, typename S, int DYN, class E>
__device__ __forceinline__ void setup_node(E& ev, const Geo<G>& g, const S* __restrict__ V, S vj)
{
    G x[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) x[d] = g.lo[d] + (G)ev.i[d] * g.h[d];
    ev.g = &g;
    ev.V = V;
    ev.vj = vj;
    ev.sp.dt = g.dt;
    ev.sp.hdt = g.hdt;
    ev.sp.um = g.um;
#pragma unroll
    for (int d = 0; d < 4; ++d) ev.u0[d] = (G)0;
    ev.nd = node_dyn<G, DYN>(g, ev.sp, x);
}

// Corner rows of node j's frozen-foot cell (offsets dr, dv, dt from the node;
// the mass offset is the grid's): base[] as cell_rows gives them.
template <bool REDUCED>
__device__ __forceinline__ void foot_rows(const Geo<float>& g, int j, int dr, int dv, int dt, int base[4])
{
    if (!REDUCED) {
        // full box: the cell's corner index is the node's own index plus offsets
        const int b0 = j + dr * g.stride[0] + dv * g.stride[1] + dt * g.stride[2] + g.foot_dm;
        base[0] = b0;
        base[1] = b0 + g.stride[1];
        base[2] = b0 + g.stride[0];
        base[3] = b0 + g.stride[0] + g.stride[1];
    } else {
        // the four (r, v_r) rows' origins: membership was checked when the
        // foot was stored, so the row lengths are not needed
        int i[4];
        decode_node(g, j, i);
        const int row = (i[0] + dr) * g.n[1] + i[1] + dv;
        const int off = (i[2] + dt) * g.n_m + i[3] + g.foot_dm;
        base[0] = __ldg(&g.row_org[row]) + off;
        base[1] = __ldg(&g.row_org[row + 1]) + off;
        base[2] = __ldg(&g.row_org[row + g.n[1]]) + off;
        base[3] = __ldg(&g.row_org[row + g.n[1] + 1]) + off;
    }
}

// A decoded frozen foot of kind kFootInside: cell offsets and fractions.
struct FootCell {
    int dr, dv, dt;
    float t[4];
};

__device__ __forceinline__ FootCell foot_cell_of(const Geo<float>& g, FootWord w)
{
    FootCell f;
    f.dr = (int)((w.hi >> 8) & 3u) - 2;
    f.dv = (int)((w.hi >> 10) & 15u) - 8;
    f.dt = (int)((w.hi >> 14) & 3u) - 2;
    const unsigned q2 = (unsigned)(w.lo >> 48) | ((w.hi & 0xffu) << 16);
    f.t[0] = (float)(unsigned)(w.lo & 0xffffffu) * (1.0f / kFootQ);
    f.t[1] = (float)(unsigned)((w.lo >> 24) & 0xffffffu) * (1.0f / kFootQ);
    f.t[2] = (float)q2 * (1.0f / kFootQ);
    f.t[3] = g.foot_tm;
    return f;
}

__device__ __forceinline__ FootCell foot_cell_of(const Geo<float>& g, unsigned long long w)
{
    FootCell f;
    f.dr = (int)((w >> 54) & 3u) - 2;
    f.dv = (int)((w >> 56) & 15u) - 8;
    f.dt = (int)((w >> 60) & 3u) - 2;
    f.t[0] = (float)(unsigned)(w & 0x3ffffu) * (1.0f / kFoot8Q);
    f.t[1] = (float)(unsigned)((w >> 18) & 0x3ffffu) * (1.0f / kFoot8Q);
    f.t[2] = (float)(unsigned)((w >> 36) & 0x3ffffu) * (1.0f / kFoot8Q);
    f.t[3] = g.foot_tm;
    return f;
}

// Kind of a stored foot, either format.
__device__ __forceinline__ int foot_kind(FootWord w) { return (int)((w.hi >> 16) & 3u); }
__device__ __forceinline__ int foot_kind(unsigned long long w) { return foot8_kind_of(w); }

// Blend at a frozen foot of kind kFootInside: D = I[V] - vj.  W: the word
// pair (FootWord) or the 8-byte word.
template <bool REDUCED, typename W>
__device__ __forceinline__ float eval_foot(const Geo<float>& g, const float* __restrict__ V, int j, W w, float vj)
{
    const FootCell f = foot_cell_of(g, w);
    int base[4];
    foot_rows<REDUCED>(g, j, f.dr, f.dv, f.dt, base);
    Corners<float> K;
    load_rows<float, float>(V, base, g.n_m, vj, K);
    return K.blend(f.t);
}

// Node j's own weight among the corners of its frozen foot (kind inside):
// per coordinate 1 - t where the cell starts at the node, t where it ends
// there, 0 otherwise.
template <typename W>
__device__ __forceinline__ float foot_self_weight(const Geo<float>& g, W w)
{
    const FootCell f = foot_cell_of(g, w);
    auto wt = [](int off, float t) { return off == 0 ? 1.0f - t : (off == -1 ? t : 0.0f); };
    return wt(f.dr, f.t[0]) * wt(f.dv, f.t[1]) * wt(f.dt, f.t[2]) * wt(g.foot_dm, g.foot_tm);
}

// Blend of increments d at node j's recomputed foot for a policy code: the
// foot of an outside or target node carries no increment.  *wself
// (nullable): node j's own weight among the corners.
template <bool REDUCED, int DYN>
__device__ __forceinline__ float incr_recompute(const Geo<float>& g, const float* __restrict__ d, int j, int code,
                                                float* wself = nullptr)
{
    NodeEval<float, float, REDUCED, DYN> ev;
    decode_node(g, j, ev.i);
    if (wself) *wself = 0.0f;
    if (in_target(g, ev.i)) return 0.0f;
    setup_node<float, float, DYN>(ev, g, d, 0.0f);
    float s, c, u[4], t[4];
    int cl[4];
    code_sincos(g, code, s, c);
    heun_cells<float, DYN>(g, ev.sp, ev.nd, s, c, u);
    Corners<float> K;
    if (foot_cell(g, ev.i, u, cl, t) || load_corners<float, float, float, REDUCED>(g, d, cl, 0.0f, K)) return 0.0f;
    if (wself) *wself = self_weight<float, false>(g, ev.i, cl, t);
    return K.blend(t);
}

// The rare nodes whose foot was not stored (kind kFootRecompute) evaluate
// out of line, so that the registers of the one-step map do not count against
// the gather loop of the evaluation sweeps: (new value, node's own weight).
template <bool REDUCED, int DYN, bool DIAG>
__device__ __noinline__ float2 feet_recompute(const Geo<float>& g, const float* __restrict__ Vin, int j, int c,
                                              float vj)
{
    NodeEval<float, float, REDUCED, DYN> ev;
    decode_node(g, j, ev.i);
    setup_node<float, float, DYN>(ev, g, Vin, vj);
    float ws = 0.0f;
    float D;
    if constexpr (DIAG) D = ev.at_code_w(c, ws);
    else D = ev.at_code(c);
    return make_float2(bellman_value<float, float>(g, vj, D), ws);
}

// The diagonal-solved step of the evaluation: V_j + (T_f(V)_j - V_j) / (1 - beta w_jj).
// The factor only sets the step length (the fixed point is where the change
// T_f(V)_j - V_j vanishes), so FP32 uses the fast division.
__device__ __forceinline__ float diag_step(const Geo<float>& g, float vj, float vplain, float ws)
{
    return vj + __fdividef(vplain - vj, 1.0f - (g.beta_hi + g.beta_lo) * ws);
}
template <typename G>
__device__ __forceinline__ double diag_step(const Geo<G>& g, double vj, double vplain, double ws)
{
    return vj + (vplain - vj) * recip_newton(1.0 - g.beta64 * ws);
}

// Largest distance in stored-node index from node j to a corner of cell cl
// (the cell's lowest corner, and the highest one plus the v_t and mass steps).
template <bool REDUCED>
__device__ __forceinline__ int cell_reach(const Geo<float>& g, int j, const int cl[4])
{
    int base[4];
    cell_rows<float, REDUCED>(g, cl, base);
    const int lo = min(min(base[0], base[1]), min(base[2], base[3]));
    const int hi = max(max(base[0], base[1]), max(base[2], base[3])) + g.n_m + 1;
    return max(j - lo, hi - j);
}

// Sweeps nodes j0, j0 + stride, ... < end of one grid: the per-node work of
// every sweep mode.  Folds max |V_out - V_in| into resid and non-finite
// results into bad.
template <typename G, typename S, int MODE, bool REDUCED, int DYN, bool PREFETCH = true>
__device__ __forceinline__ void sweep_nodes(const Geo<G>& g, const Table<G>& T, const S* __restrict__ Vin,
                                            S* __restrict__ Vout, uint16_t* __restrict__ code,
                                            unsigned long long* __restrict__ feet_lo,
                                            unsigned* __restrict__ feet_hi, float* __restrict__ inc,
                                            float* __restrict__ acc, double* __restrict__ V64, int incr_flags,
                                            int j0, int end, int stride, S& resid, bool& bad,
                                            const Feet64 f64 = Feet64(), int* reach = nullptr,
                                            bool feet8 = true)
{
    constexpr bool kIsVI = MODE == kVI || MODE == kVIDiag;
    constexpr bool kSearch = kIsVI || MODE == kImproveFull || MODE == kImproveWalk;
    constexpr bool kImprove = MODE == kImproveFull || MODE == kImproveWalk;
    constexpr bool kGeo32 = std::is_same<G, float>::value;
    constexpr bool kPolish = kGeo32 && std::is_same<S, double>::value;   // FP32 geometry, FP64 values
    (void)T;
    (void)kSearch;
    if constexpr (MODE == kEvalFeet64 || MODE == kEvalFeet64Diag) {
        // FP64 evaluation from the FP64 frozen feet
        constexpr bool kDiag = MODE == kEvalFeet64Diag;
        constexpr bool kPer = DYN == kDynPolar;
        for (int j = j0; j < end; j += stride) {
            const S vj = Vin[j];
            const unsigned long long w = __ldcs(&f64.w[j]);
            const int kind = (int)((w >> 32) & 3u);
            S vnew = (S)0;
            if (kind != kFootTarget) {
                const double cj = __ldcs(&f64.c[j]);
                double D, ws = 0.0;
                if (kind == kFootOut) {
                    D = g.M64 - (double)vj;
                } else if (kind == kFootInside) {
                    int i[4], cl[4];
                    decode_node(g, j, i);
#pragma unroll
                    for (int d = 0; d < 4; ++d) cl[d] = i[d] + (int)(signed char)((w >> (8 * d)) & 0xffu);
                    if (kPer) cl[3] = cl[3] < 0 ? cl[3] + g.n[3] : (cl[3] >= g.n[3] ? cl[3] - g.n[3] : cl[3]);
                    const double2 ta = __ldcs(&f64.t[2 * (size_t)j]), tb = __ldcs(&f64.t[2 * (size_t)j + 1]);
                    const double t[4] = {ta.x, ta.y, tb.x, tb.y};
                    Corners<double> K;
                    load_corners<double, G, S, REDUCED, kPer>(g, Vin, cl, vj, K);   // membership checked when stored
                    D = K.blend(t);
                    if constexpr (kDiag) ws = self_weight<G, kPer>(g, i, cl, t);
                } else {
                    NodeEval<G, S, REDUCED, DYN> ev;
                    decode_node(g, j, ev.i);
                    setup_node<G, S, DYN>(ev, g, Vin, vj);
                    const int c0 = code[j];
                    typename NodeEval<G, S, REDUCED, DYN>::R wr = 0;
                    if (kPer && g.off && c0 == kCodeOff)
                        D = kDiag ? ev.at_sc_w((G)0, (G)0, wr) : ev.at_sc((G)0, (G)0);
                    else
                        D = kDiag ? ev.at_code_w(c0, wr) : ev.at_code(c0);
                    ws = wr;
                }
                double q = cj + g.beta64 * ((double)vj + D);
                if constexpr (kDiag) q = diag_step(g, (double)vj, q, ws);
                vnew = (S)q;
            }
            Vout[j] = vnew;
            resid = fmax(resid, (S)fabs(vnew - vj));
            bad = bad || !isfinite(vnew);
        }
    } else if constexpr (MODE == kEvalFeet || MODE == kEvalFeet8 || MODE == kIncr || MODE == kEvalFeetDiag ||
                         MODE == kIncrDiag) {
        constexpr bool kDiag = MODE == kEvalFeetDiag || MODE == kIncrDiag;
        // frozen feet: gather-bound.  With PREFETCH the next node's foot and
        // value are fetched while this node's corners are in flight; without
        // it the loop needs fewer registers (more resident blocks instead).
        // The feet are read once per sweep: evict-first loads keep L1 and L2
        // for the gathered V.
        constexpr bool kPrefetch = PREFETCH;
        // kEvalFeet8 reads one 8-byte word per node, the other modes the
        // 24-bit word pair
        constexpr bool kF8 = MODE == kEvalFeet8;
        typedef typename std::conditional<kF8, unsigned long long, FootWord>::type FW;
        auto load_foot = [&](int k) -> FW {
            if constexpr (kF8) return __ldcs(&feet_lo[k]);
            else return FootWord{__ldcs(&feet_lo[k]), __ldcs(&feet_hi[k])};
        };
        const bool first = incr_flags & 1, last = incr_flags & 2;
        int j = j0;
        FW w_next{};
        S v_next = (S)0;
        if (kPrefetch && j < end) {
            w_next = load_foot(j);
            v_next = Vin[j];
        }
        for (; j < end; j += stride) {
            FW w;
            S vj;
            if constexpr (kPrefetch) {
                w = w_next;
                vj = v_next;
                if (j + stride < end) {
                    w_next = load_foot(j + stride);
                    v_next = Vin[j + stride];
                }
            } else {
                w = load_foot(j);
                vj = Vin[j];
            }
            const int kind = foot_kind(w);
            S vnew = (S)0;
            if constexpr (MODE == kEvalFeet || MODE == kEvalFeet8 || MODE == kEvalFeetDiag) {
                float ws = 0.0f;
                if (kind == kFootInside) {
                    if constexpr (kDiag) ws = foot_self_weight(g, w);
                    vnew = bellman_value<G, S>(g, vj, eval_foot<REDUCED>(g, Vin, j, w, vj));
                } else if (kind == kFootOut) {
                    vnew = bellman_value<G, S>(g, vj, (G)((S)g.M64 - vj));
                } else if (kind == kFootRecompute) {
                    const float2 r = feet_recompute<REDUCED, DYN, kDiag>(g, Vin, j, code[j], vj);
                    vnew = r.x;
                    ws = r.y;
                }
                if constexpr (kDiag) {
                    if (kind != kFootTarget) vnew = diag_step(g, vj, vnew, ws);
                }
                Vout[j] = vnew;
                resid = fmax(resid, (S)fabs(vnew - vj));
            } else {
                // increment: d' = beta W d at the frozen policy (no running cost,
                // no penalty: both cancel between consecutive sweeps).  Diagonal
                // solved: the first increment after the improvement's plain step
                // is beta W d scaled by 1 / (1 - beta w_jj), later ones use the
                // off-diagonal weights only, d' = beta (W d - w_jj d_j) / (1 - beta w_jj)
                float D = 0.0f, ws = 0.0f;
                if (kind == kFootInside) {
                    D = eval_foot<REDUCED>(g, Vin, j, w, 0.0f);
                    if constexpr (kDiag) ws = foot_self_weight(g, w);
                } else if (kind == kFootRecompute) {
                    D = incr_recompute<REDUCED, DYN>(g, Vin, j, code[j], kDiag ? &ws : nullptr);
                }
                if constexpr (kDiag) {
                    const float Dx = first ? D : D - ws * vj;
                    vnew = __fdividef(fmaf(g.beta_hi, Dx, g.beta_lo * Dx), 1.0f - (g.beta_hi + g.beta_lo) * ws);
                } else {
                    vnew = fmaf(g.beta_hi, D, g.beta_lo * D);
                }
                Vout[j] = vnew;
                const float sum = (first ? 0.0f : acc[j]) + vnew;
                if (last) V64[j] += (double)sum;
                else acc[j] = sum;
                resid = fmax(resid, (S)fabs(vnew));
            }
            bad = bad || !isfinite(vnew);
        }
    } else {
        // evaluation sweeps interpolate once per node; searches keep the cell's
        // corners in registers across angles
        // FP64 values: the search blends FP32-rounded FP64 differences (about
        // 1e-9 of a cell's value spread, far below the FP32 geometry's own
        // noise), and the chosen code is then re-evaluated in FP64
        typedef typename std::conditional<kPolish, float, typename BlendType<G, S>::type>::type SearchR;
        typedef typename std::conditional<kSearch, CachedEval<G, S, REDUCED, DYN, SearchR, false, MODE == kVIDiag>,
                                          NodeEval<G, S, REDUCED, DYN>>::type Eval;
        for (int j = j0; j < end; j += stride) {
            const S vj = Vin[j];
            S vnew = (S)0;
            double vnew64 = 0.0;
            (void)vnew64;
            Eval ev;
            decode_node(g, j, ev.i);
            if constexpr (DYN == kDynPolar) {
                // the paper's Example 1: running cost of Eq. (11) and the
                // thrust-off control, which wins a tie (FP64 grids only)
                if (!in_target(g, ev.i)) {
                    setup_node<G, S, DYN>(ev, g, Vin, vj);
                    const double lrun = __dmul_rn(g.dt64, state_cost(g, ev.i));   // rounded on its own: no contraction with the sums below
                    double q;
                    if constexpr (MODE == kEval) {
                        const int c0 = code[j];
                        if (g.off && c0 == kCodeOff) q = lrun + g.beta64 * ((double)vj + (double)ev.at_sc((G)0, (G)0));
                        else q = lrun + g.thrust_cost + g.beta64 * ((double)vj + (double)ev.at_code(c0));
                    } else if constexpr (MODE == kEvalDiag) {
                        const int c0 = code[j];
                        typename Eval::R ws;
                        if (g.off && c0 == kCodeOff)
                            q = lrun + g.beta64 * ((double)vj + (double)ev.at_sc_w((G)0, (G)0, ws));
                        else
                            q = lrun + g.thrust_cost + g.beta64 * ((double)vj + (double)ev.at_code_w(c0, ws));
                        q = diag_step(g, (double)vj, q, (double)ws);
                    } else {
                        ev.reset();
                        typename Eval::R D;
                        int k;
                        const int c_old = MODE == kImproveWalk ? (int)code[j] : 0;
                        // a node whose previous control was off has no angle to walk from
                        if (MODE == kImproveWalk && !(g.off && c_old == kCodeOff))
                            k = walk_table(ev, T, nearest_index(g.K, c_old), D);
                        else
                            k = enumerate_table(ev, T, D);
                        int c = T.code[k] & (kCodes - 1);
                        if (!kIsVI && g.refine) c = fibonacci_refine(ev, T, g.fib_n0, g.fib_stop, k, D, D);
                        q = lrun + g.thrust_cost + g.beta64 * ((double)vj + (double)D);
                        if (g.off) {
                            const double q_off = lrun + g.beta64 * ((double)vj + (double)ev.at_sc((G)0, (G)0));
                            if (q_off <= q) {
                                q = q_off;
                                c = kCodeOff;
                            }
                        }
                        if (!kIsVI) code[j] = (uint16_t)c;
                        if constexpr (!kGeo32 && kImprove) {
                            if (f64.w) {
                                const bool off = g.off && c == kCodeOff;
                                G sn = (G)0, cs = (G)0, t[4];
                                if (!off) code_sincos(g, c, sn, cs);
                                f64.w[j] = ev.foot64_of(sn, cs, t);
                                f64.t[2 * (size_t)j] = make_double2((double)t[0], (double)t[1]);
                                f64.t[2 * (size_t)j + 1] = make_double2((double)t[2], (double)t[3]);
                                f64.c[j] = off ? lrun : lrun + g.thrust_cost;
                            }
                        }
                    }
                    vnew = (S)q;
                } else if constexpr (!kGeo32 && kImprove) {
                    if (f64.w) f64.w[j] = (unsigned long long)kFootTarget << 32;
                }
            } else if (!in_target(g, ev.i)) {
                setup_node<G, S, DYN>(ev, g, Vin, vj);
                typename Eval::R D;
                typename Eval::R ws = 0;
                (void)ws;
                if constexpr (MODE == kEval) {
                    D = ev.at_code(code[j]);
                } else if constexpr (MODE == kEvalDiag) {
                    D = ev.at_code_w(code[j], ws);
                } else {
                    ev.reset();
                    int k;
                    const int c_old = (MODE == kImproveWalk || kPolish) ? (int)code[j] : 0;
                    if (MODE == kImproveWalk)
                        k = walk_table(ev, T, nearest_index(g.K, c_old), D);
                    else
                        k = enumerate_table(ev, T, D);
                    int c = T.code[k] & (kCodes - 1);
                    if (!kIsVI && g.refine) c = fibonacci_refine(ev, T, g.fib_n0, g.fib_stop, k, D, D);
                    if constexpr (kImprove && kPolish) {
                        // FP64 blend of the chosen code.  Both the walk and the
                        // full tabulation keep the node's current code unless the
                        // new one is strictly better in FP64 (policy iteration's
                        // rule for termination): otherwise the two searches, which
                        // can stop in different local minima, undo each other
                        // The FP64 blends interpolate V itself (reference value 0,
                        // so no corner differences): FP64 keeps its 1e-16 relative
                        // error on V, and the FP64 pipe does half the work.
                        NodeEval<G, S, REDUCED, DYN> e64;
                        e64.g = ev.g;
                        e64.V = ev.V;
                        e64.sp = ev.sp;
                        e64.vj = (S)0;
                        e64.nd = ev.nd;
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            e64.i[d] = ev.i[d];
                            e64.u0[d] = ev.u0[d];
                        }
                        double q_new = e64.at_code(c);   // I[V] at the foot, M outside
                        if (c != c_old) {
                            const double q_old = e64.at_code(c_old);
                            if (!(q_new < q_old)) {
                                c = c_old;
                                q_new = q_old;
                            }
                        }
                        vnew64 = g.dt64 + g.beta64 * q_new;
                    }
                    if (!kIsVI) code[j] = (uint16_t)c;
                    if constexpr (kGeo32 && kImprove) {
                        if (feet_lo) {
                            // 8-byte feet for the plain evaluation of FP32
                            // values (feet8), else the 24-bit word pair
                            int cl[4];
                            int kind;
                            if (!kPolish && feet8) {
                                const unsigned long long w = ev.foot8_of(c, cl);
                                feet_lo[j] = w;
                                kind = foot_kind(w);
                            } else {
                                const FootWord w = ev.foot_of(c, cl);
                                feet_lo[j] = w.lo;
                                feet_hi[j] = w.hi;
                                kind = foot_kind(w);
                            }
                            if (reach && kind != kFootOut) *reach = max(*reach, cell_reach<REDUCED>(g, j, cl));
                        }
                    }
                    if constexpr (!kGeo32 && kImprove) {
                        if (f64.w) {
                            G sn, cs, t[4];
                            code_sincos(g, c, sn, cs);
                            f64.w[j] = ev.foot64_of(sn, cs, t);
                            f64.t[2 * (size_t)j] = make_double2((double)t[0], (double)t[1]);
                            f64.t[2 * (size_t)j + 1] = make_double2((double)t[2], (double)t[3]);
                            f64.c[j] = g.dt64;
                        }
                    }
                }
                if constexpr (kPolish) vnew = (S)bellman_value(g, (double)vj, (double)D);
                else vnew = bellman_value<G, S>(g, vj, D);
                if constexpr (kImprove && kPolish) vnew = (S)vnew64;
                if constexpr (MODE == kEvalDiag) vnew = (S)diag_step(g, vj, vnew, ws);
            } else if constexpr (kGeo32 && kImprove) {
                if (feet_lo) {
                    if (!kPolish && feet8) {
                        feet_lo[j] = foot8_kind(kFootTarget);
                    } else {
                        const FootWord w = foot_word_kind(kFootTarget);
                        feet_lo[j] = w.lo;
                        feet_hi[j] = w.hi;
                    }
                }
            } else if constexpr (!kGeo32 && kImprove) {
                if (f64.w) f64.w[j] = (unsigned long long)kFootTarget << 32;
            }
            if constexpr (kImprove) {
                if (inc) inc[j] = (float)(vnew - vj);   // first increment of the evaluation sweeps
            }
            Vout[j] = vnew;
            resid = fmax(resid, (S)fabs(vnew - vj));
            bad = bad || !isfinite(vnew);
        }
    }

}

// Block-wide max of resid folded into *slot (FP64 bits) and the non-finite
// flag into *nonfinite.  Every thread of the block calls it.
template <typename S, int BLOCK = kBlock>
__device__ __forceinline__ void block_fold(S resid, bool bad, unsigned long long* slot, int* nonfinite)
{
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block of whole warps, at most 32");
    __shared__ S red[BLOCK / 32];
    resid = warp_max(resid);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = resid;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
    if (threadIdx.x < 32) {
        S r = threadIdx.x < BLOCK / 32 ? red[threadIdx.x] : (S)0;
        r = warp_max(r);
        if (threadIdx.x == 0) atomicMax(slot, (unsigned long long)__double_as_longlong((double)r));
    }
}

// Frozen-feet sweeps are bound by the bytes and gathers each thread keeps in
// flight.  The plain evaluation prefetches the next node's foot and value
// (40 registers, 768-thread blocks): on the full box 76.7 against 79.0 us per
// 61^4 sweep without it at 32 registers.  The diagonal-solved evaluation of
// the full box fits 32 registers without the prefetch (64 warps per SM); on
// the reduced grid it keeps the prefetch, as do the increment forms (they
// spill at 32 registers).
template <int MODE, bool REDUCED>
__host__ __device__ constexpr bool eval_prefetch()
{
    return !(MODE == kEvalFeetDiag && !REDUCED);
}

// Block size of the frozen-feet sweeps.  A grid-stride iteration of a block
// covers that many consecutive nodes, whose corner lines overlap (a node's
// v_t neighbours lie 61 nodes on, on the 61^4 grid), so larger blocks take
// more of their gathers from L1: 768 threads (2 blocks per SM at 40
// registers) for the plain evaluation, the increment sweeps and the
// diagonal-solved evaluation of the reduced grid (the prefetching loop needs
// the 40 registers: 0.346 against 0.376 ms per plain sweep of the 121^4 band
// in 1024-thread blocks, 0.387 without the prefetch; 640-, 384x4- and
// 512x4-thread blocks 0.354-0.381), 1024 (2 per SM, 32 registers) for the
// diagonal-solved evaluation of the full box, 1024 (one per SM at 64
// registers) for the FP64 evaluation from FP64 feet.
// Same-box A/B against 256-thread blocks: 78.9 against 83.0 us per evaluation
// sweep on 61^4, 88.0 against 90.8 us diagonal-solved; 0.40 against 0.45 ms
// for the diagonal-solved sweep of the 121^4 band grid.  A grid too small to give
// every SM a large block (the 17^4 box has 83,521 nodes) runs 256-thread
// blocks instead (BIG = false).
template <int MODE, bool REDUCED>
__host__ __device__ constexpr int big_block()
{
    return (MODE == kIncr || MODE == kIncrDiag || MODE == kEvalFeet || MODE == kEvalFeet8 ||
            (MODE == kEvalFeetDiag && REDUCED))
               ? 768
           : (MODE == kEvalFeetDiag || MODE == kEvalFeet64 || MODE == kEvalFeet64Diag) ? 1024
                                                                                        : kBlock;
}

template <int MODE, bool REDUCED, bool BIG>
__host__ __device__ constexpr int sweep_block()
{
    return BIG ? big_block<MODE, REDUCED>() : kBlock;
}

template <typename G, typename S, int MODE, bool REDUCED, bool BIG>
constexpr int min_blocks()
{
    constexpr bool feet64 = MODE == kEvalFeet64 || MODE == kEvalFeet64Diag;
    if (BIG) return feet64 ? 1 : 2;
    // FP32 angle searches: 3 blocks of 256 per SM (80 registers).  Left to
    // itself the compiler gives the reduced-grid walk 96 registers (2 blocks):
    // 4.84 against 4.36 ms per sweep on the 121^4 band
    if (std::is_same<G, float>::value && std::is_same<S, float>::value &&
        (MODE == kImproveWalk || MODE == kImproveFull))
        return 3;
    return ((MODE == kEvalFeet || MODE == kEvalFeet8 || MODE == kEvalFeetDiag) && !REDUCED) ? 8
           : (MODE == kIncr || MODE == kIncrDiag || MODE == kEvalFeetDiag) ? 6
           : feet64                                                      ? 4
                                                                         : 1;
}

template <typename G, typename S, int MODE, bool REDUCED, int DYN, bool BIG>
__global__ void __launch_bounds__(sweep_block<MODE, REDUCED, BIG>(), min_blocks<G, S, MODE, REDUCED, BIG>())
sweep_kernel(const __grid_constant__ Geo<G> g, const S* __restrict__ Vin, S* __restrict__ Vout,
             uint16_t* __restrict__ code, unsigned long long* __restrict__ feet_lo, unsigned* __restrict__ feet_hi,
             float* __restrict__ inc, float* __restrict__ acc, double* __restrict__ V64, int incr_flags,
             Ctl* __restrict__ ctl, unsigned long long* __restrict__ ring, int ring_mask, long long sweep,
             int check_prev, double tol, const Feet64 f64, int feet8)
{
    constexpr bool kSearch = MODE == kVI || MODE == kVIDiag || MODE == kImproveFull || MODE == kImproveWalk;
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

    // angle searches read the tabulated codes and (sin, cos) from shared memory
    __shared__ int s_code[kSearch ? kMaxAngles + 1 : 1];
    __shared__ typename V2<G>::type s_sc[kSearch ? kMaxAngles : 1];
    if constexpr (kSearch) {
        build_table(g, s_code, s_sc);
        __syncthreads();
    }
    const Table<G> T{s_code, s_sc, g.K, g.off};

    S resid = (S)0;
    bool bad = false;
    constexpr int B = sweep_block<MODE, REDUCED, BIG>();
    const int j0 = blockIdx.x * B + threadIdx.x, end = g.n_nodes, stride = gridDim.x * B;
    constexpr bool kReach = std::is_same<G, float>::value && (MODE == kImproveFull || MODE == kImproveWalk);
    int reach = 0;
    sweep_nodes<G, S, MODE, REDUCED, DYN, eval_prefetch<MODE, REDUCED>()>(
        g, T, Vin, Vout, code, feet_lo, feet_hi, inc, acc, V64, incr_flags, j0, end, stride, resid, bad, f64,
        kReach ? &reach : nullptr, feet8 != 0);
    if constexpr (kReach) {
        // the stored feet's reach, for the multi-level evaluation that follows
        reach = __reduce_max_sync(0xffffffffu, (unsigned)reach);
        if ((threadIdx.x & 31) == 0 && reach > 0) atomicMax(&ctl->reach, reach);
    }
    block_fold<S, B>(resid, bad, &ring[sweep & ring_mask], &ctl->nonfinite);
}

template <typename G, typename S, int MODE, bool REDUCED, int DYN, bool BIG>
cudaError_t launch_sized(const SweepLaunch<G, S>& L)
{
    auto kern = sweep_kernel<G, S, MODE, REDUCED, DYN, BIG>;
    constexpr int B = sweep_block<MODE, REDUCED, BIG>();
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    long long need = ((long long)L.g.n_nodes + B - 1) / B;
    long long cap = (long long)per_sm * L.sm_count;
    int blocks = (int)(need < cap ? need : cap);
    if (blocks < 1) blocks = 1;
    kern<<<blocks, B, 0, L.stream>>>(L.g, L.Vin, L.Vout, L.code, L.feet_lo, L.feet_hi, L.inc, L.acc, L.V64,
                                      L.incr_flags, L.ctl, L.ring, L.ring_mask, L.sweep, L.check_prev, L.tol, L.f64,
                                      L.feet8);
    return cudaGetLastError();
}

template <typename G, typename S, int MODE, bool REDUCED, int DYN>
cudaError_t launch_one(const SweepLaunch<G, S>& L)
{
    constexpr int Bbig = big_block<MODE, REDUCED>();
    if constexpr (Bbig != kBlock) {
        // large blocks only where every SM gets one
        if ((long long)L.g.n_nodes >= (long long)Bbig * L.sm_count)
            return launch_sized<G, S, MODE, REDUCED, DYN, true>(L);
    }
    return launch_sized<G, S, MODE, REDUCED, DYN, false>(L);
}

template <typename G, typename S, int DYN, bool REDUCED>
cudaError_t launch_mode(const SweepLaunch<G, S>& L)
{
    constexpr bool f32 = std::is_same<G, float>::value && std::is_same<S, float>::value;
    switch (L.mode) {
    case kVI: return launch_one<G, S, kVI, REDUCED, DYN>(L);
    case kImproveFull: return launch_one<G, S, kImproveFull, REDUCED, DYN>(L);
    case kImproveWalk: return launch_one<G, S, kImproveWalk, REDUCED, DYN>(L);
    case kEval: return launch_one<G, S, kEval, REDUCED, DYN>(L);
    case kEvalFeet:
        if constexpr (f32) return L.feet_lo ? launch_one<G, S, kEvalFeet, REDUCED, DYN>(L) : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    case kEvalFeet8:
        if constexpr (f32) return L.feet_lo ? launch_one<G, S, kEvalFeet8, REDUCED, DYN>(L) : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    case kIncr:
        if constexpr (f32)
            return (L.feet_lo && L.acc && L.V64) ? launch_one<G, S, kIncr, REDUCED, DYN>(L) : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    case kEvalDiag: return launch_one<G, S, kEvalDiag, REDUCED, DYN>(L);
    case kVIDiag:
        if constexpr (DYN != kDynPolar) return launch_one<G, S, kVIDiag, REDUCED, DYN>(L);
        return cudaErrorInvalidValue;
    case kEvalFeet64:
        if constexpr (std::is_same<G, double>::value && std::is_same<S, double>::value)
            return L.f64.w ? launch_one<G, S, kEvalFeet64, REDUCED, DYN>(L) : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    case kEvalFeet64Diag:
        if constexpr (std::is_same<G, double>::value && std::is_same<S, double>::value)
            return L.f64.w ? launch_one<G, S, kEvalFeet64Diag, REDUCED, DYN>(L) : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    case kEvalFeetDiag:
        if constexpr (f32) return L.feet_lo ? launch_one<G, S, kEvalFeetDiag, REDUCED, DYN>(L) : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    case kIncrDiag:
        if constexpr (f32)
            return (L.feet_lo && L.acc && L.V64) ? launch_one<G, S, kIncrDiag, REDUCED, DYN>(L)
                                                 : cudaErrorInvalidValue;
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

}  // namespace dpk
