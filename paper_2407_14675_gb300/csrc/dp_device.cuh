// dp_device.cuh -- device-side pieces of the semi-Lagrangian Bellman sweep.
//
// One thread owns one stored grid node.  For a control angle it takes the
// Heun (second-order Runge-Kutta) step of the polar dynamics (§3 "Grid and
// polar coordinates", angle coordinate dropped, mass added), expresses the
// displacement in cells, and interpolates V multilinearly (Q1) over the 16
// corners of the foot's cell (§3 after Eq. (10)).  A foot outside the box, or
// in a cell with a corner outside the reduced node set, is charged M.
//
// Values are compared and blended as D = I[V](z) - V_j, the difference to the
// node's own value, so that FP32 keeps the few significant digits that
// separate one thrust angle from the next (V ~ 20 while the control changes
// I[V] by ~1e-4).  The Bellman value is then dt + beta (V_j + D).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace dpk {

constexpr int kCodes = 65536;       // 16-bit angle lattice, alpha = 2 pi c / 65536
constexpr int kBlock = 256;         // threads per block of the sweep kernels
constexpr int kMaxFib = 30;

enum { kVI = 0, kImproveFull = 1, kImproveWalk = 2, kEval = 3 };
enum { kDynOrbit = 0, kDynUnitSpeed = 1 };

// Fibonacci numbers F[1] = F[2] = 1 (index 0 unused).
__constant__ int kFib[kMaxFib] = {0, 1, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377, 610, 987,
                                  1597, 2584, 4181, 6765, 10946, 17711, 28657, 46368, 75025,
                                  121393, 196418, 317811, 514229};

template <typename G> struct V2;
template <> struct V2<float>  { typedef float2 type; };
template <> struct V2<double> { typedef double2 type; };

// Device control block of one solve.
struct Ctl {
    int stop;         // 1 once a stopping test has passed
    int stop_sweep;   // sweeps completed when it passed
    int nonfinite;    // a sweep produced a non-finite value
    int pad;
};

// Everything a sweep kernel needs about the grid, in geometry precision G.
template <typename G>
struct Geo {
    int n[4];
    int stride[4];             // box strides, mass fastest (full-box addressing)
    G lo[4], h[4], ih[4];      // box origin, spacing, 1 / spacing
    G mu, accel, mdot, dt, hdt, beta, M;
    G beta_hi, beta_lo;        // beta = beta_hi + beta_lo (FP32 value update)
    double dt64, beta64, M64;  // exact parameters for FP64 value updates
    G um;                      // mass displacement in cells, identical at every node
    int dyn;
    int K, refine, fib_stop;   // refinement stops once the bracket is <= fib_stop codes
    int tlo[4], thi[4];        // target index box, inclusive (tlo > thi: no target)
    int n_m;
    unsigned long long magic_m;    // ceil(2^40 / n_m): j / n_m for j < 2^40 / (n_m - 1)
    int n_nodes;               // stored nodes
    const int4* rows;          // per (i_r, i_vr): {first compact index, lo_vt, len, 0}
    const unsigned* lines;     // per compact (r, v_r, v_t) line: i_r | i_vr<<10 | i_vt<<20
    const typename V2<G>::type* tab_hi;   // (sin, cos) of 2 pi (c >> 8) 256 / 65536
    const typename V2<G>::type* tab_lo;   // (sin, cos) of 2 pi (c & 255) / 65536
};

template <typename G> __device__ __forceinline__ G ginf();
template <> __device__ __forceinline__ float ginf<float>() { return CUDART_INF_F; }
template <> __device__ __forceinline__ double ginf<double>() { return CUDART_INF; }

__device__ __forceinline__ float grcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double grcp(double x) { return __drcp_rn(x); }

// Code of the k-th tabulated angle 2 pi k / K on the lattice (round half up).
__device__ __forceinline__ int table_code(int K, int k) { return (k * kCodes + K / 2) / K; }

// Nearest tabulated index to a code (start of the local walk).
__device__ __forceinline__ int nearest_table_index(int K, int code)
{
    return (int)((((long long)code * K + kCodes / 2) / kCodes) % K);
}

__device__ __forceinline__ int wrap_code(int c) { return c & (kCodes - 1); }

// (sin, cos) of a lattice code from two 256-entry tables:
// alpha = a_hi + a_lo, sin = s_h c_l + c_h s_l, cos = c_h c_l - s_h s_l.
template <typename G>
__device__ __forceinline__ void code_sincos(const Geo<G>& g, int code, G& s, G& c)
{
    code = wrap_code(code);
    typename V2<G>::type hi = __ldg(&g.tab_hi[code >> 8]);
    typename V2<G>::type lo = __ldg(&g.tab_lo[code & 255]);
    s = hi.x * lo.y + hi.y * lo.x;
    c = hi.y * lo.y - hi.x * lo.x;
}

// Node decode: compact index -> (i_r, i_vr, i_vt, i_m).
template <typename G>
__device__ __forceinline__ void decode_node(const Geo<G>& g, int j, int i[4])
{
    unsigned line = (unsigned)(((unsigned long long)(unsigned)j * g.magic_m) >> 40);
    i[3] = j - (int)line * g.n_m;
    unsigned L = __ldg(&g.lines[line]);
    i[0] = (int)(L & 1023u);
    i[1] = (int)((L >> 10) & 1023u);
    i[2] = (int)((L >> 20) & 1023u);
}

template <typename G>
__device__ __forceinline__ bool in_target(const Geo<G>& g, const int i[4])
{
    bool t = true;
#pragma unroll
    for (int d = 0; d < 4; ++d) t = t && i[d] >= g.tlo[d] && i[d] <= g.thi[d];
    return t;
}

// Step of the one-step map: dt for the sweeps, tau for the feedback.
template <typename G>
struct StepP {
    G dt, hdt;   // step and half step
    G um;        // mass displacement over the step, in cells
};

// Control-independent part of the Heun step at a state.
template <typename G>
struct NodeDyn {
    G vr, vt;
    G am, am2;       // a/m at x and at the predictor (m' does not depend on alpha)
    G d1vr, d1vt;    // drift of v_r, v_t at x
    G ir2, muir2sq;  // 1/r and mu/r^2 at the predictor (r' = v_r does not depend on alpha)
};

template <typename G, int DYN>
__device__ __forceinline__ NodeDyn<G> node_dyn(const Geo<G>& g, const StepP<G>& sp, const G x[4])
{
    NodeDyn<G> n;
    n.vr = x[1];
    n.vt = x[2];
    if (DYN == kDynOrbit) {
        G ir = grcp(x[0]);
        n.am = g.accel * grcp(x[3]);
        n.d1vr = n.vt * n.vt * ir - g.mu * ir * ir;
        n.d1vt = -n.vr * n.vt * ir;
        G r2 = x[0] + sp.dt * n.vr;
        G m2 = x[3] + sp.dt * g.mdot;
        n.ir2 = grcp(r2);
        n.muir2sq = g.mu * n.ir2 * n.ir2;
        n.am2 = g.accel * grcp(m2);
    }
    return n;
}

// Heun displacement in cells for control (s, c) = (sin alpha, cos alpha):
// k1 = b(x), k2 = b(x + dt k1), u = dt (k1 + k2) / 2 / h.
template <typename G, int DYN>
__device__ __forceinline__ void heun_cells(const Geo<G>& g, const StepP<G>& sp, const NodeDyn<G>& n,
                                           G s, G c, G u[4])
{
    if (DYN == kDynOrbit) {
        G k1vr = n.d1vr + n.am * s;
        G k1vt = n.d1vt + n.am * c;
        G vr2 = n.vr + sp.dt * k1vr;
        G vt2 = n.vt + sp.dt * k1vt;
        G k2vr = vt2 * vt2 * n.ir2 - n.muir2sq + n.am2 * s;
        G k2vt = -vr2 * vt2 * n.ir2 + n.am2 * c;
        u[0] = sp.hdt * (n.vr + vr2) * g.ih[0];
        u[1] = sp.hdt * (k1vr + k2vr) * g.ih[1];
        u[2] = sp.hdt * (k1vt + k2vt) * g.ih[2];
        u[3] = sp.um;
    } else {
        // test dynamics: unit speed in the (x0, x1) plane, tiny components zeroed
        G cc = fabs(c) < (G)1e-12 ? (G)0 : c;
        G ss = fabs(s) < (G)1e-12 ? (G)0 : s;
        u[0] = sp.dt * cc / g.h[0];   // division: dt = h lands exactly on a node
        u[1] = sp.dt * ss / g.h[1];
        u[2] = (G)0;
        u[3] = (G)0;
    }
}

// Q1 interpolation at the foot i + u (grid units), returned as the difference
// D = I[V] - vj; M - vj when the foot is outside the box or the node set.
template <typename G, typename S, bool REDUCED>
__device__ __forceinline__ G interp_delta(const Geo<G>& g, const S* __restrict__ V, const int i[4],
                                          const G u[4], S vj)
{
    int c[4];
    G t[4];
    bool out = false;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        G fl = floor(u[d]);
        t[d] = u[d] - fl;
        c[d] = i[d] + (int)fl;
        out = out || !(t[d] >= (G)0) || c[d] < 0 || c[d] > g.n[d] - 1;
        if (c[d] == g.n[d] - 1) {     // foot exactly on the upper face
            out = out || t[d] > (G)0;
            c[d] = g.n[d] - 2;
            t[d] = (G)1;
        }
    }
    if (out) return (G)((S)g.M64 - vj);

    S v[16];
    if (!REDUCED) {
        int base = c[0] * g.stride[0] + c[1] * g.stride[1] + c[2] * g.stride[2] + c[3];
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            int off = ((b >> 3) & 1) * g.stride[0] + ((b >> 2) & 1) * g.stride[1] +
                      ((b >> 1) & 1) * g.stride[2] + (b & 1);
            v[b] = __ldg(&V[base + off]);
        }
    } else {
        // the cell's four (r, v_r) rows must each hold both v_t corners
        int base[4];
#pragma unroll
        for (int rb = 0; rb < 4; ++rb) {
            int row = (c[0] + (rb >> 1)) * g.n[1] + c[1] + (rb & 1);
            int4 R = __ldg(&g.rows[row]);
            out = out || c[2] < R.y || c[2] + 1 > R.y + R.z - 1;
            base[rb] = R.x + (c[2] - R.y) * g.n_m + c[3];
        }
        if (out) return (G)((S)g.M64 - vj);
#pragma unroll
        for (int rb = 0; rb < 4; ++rb) {
            v[rb * 4 + 0] = __ldg(&V[base[rb]]);
            v[rb * 4 + 1] = __ldg(&V[base[rb] + 1]);
            v[rb * 4 + 2] = __ldg(&V[base[rb] + g.n_m]);
            v[rb * 4 + 3] = __ldg(&V[base[rb] + g.n_m + 1]);
        }
    }
    // differences to the node's own value, then 15 lerps: m, v_t, v_r, r
    G e[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) e[b] = (G)(v[b] - vj);
#pragma unroll
    for (int b = 0; b < 8; ++b) e[b] = e[2 * b] + t[3] * (e[2 * b + 1] - e[2 * b]);
#pragma unroll
    for (int b = 0; b < 4; ++b) e[b] = e[2 * b] + t[2] * (e[2 * b + 1] - e[2 * b]);
#pragma unroll
    for (int b = 0; b < 2; ++b) e[b] = e[2 * b] + t[1] * (e[2 * b + 1] - e[2 * b]);
    return e[0] + t[0] * (e[1] - e[0]);
}

// Control-dependent evaluation at one state: node i plus the offset u0 (both
// in grid units; u0 = 0 at a grid node).
template <typename G, typename S, bool REDUCED, int DYN>
struct NodeEval {
    const Geo<G>* g;
    const S* __restrict__ V;
    StepP<G> sp;
    int i[4];
    G u0[4];
    S vj;
    NodeDyn<G> nd;

    __device__ __forceinline__ G at_code(int code) const
    {
        G s, c, u[4];
        code_sincos(*g, code, s, c);
        heun_cells<G, DYN>(*g, sp, nd, s, c, u);
#pragma unroll
        for (int d = 0; d < 4; ++d) u[d] += u0[d];
        return interp_delta<G, S, REDUCED>(*g, V, i, u, vj);
    }
};

// Full tabulation; ties go to the lowest index.
template <class E>
__device__ __forceinline__ int enumerate_table(const E& ev, int K, decltype(ev.at_code(0))& Dbest)
{
    auto Db = ev.at_code(table_code(K, 0));
    int kb = 0;
    for (int k = 1; k < K; ++k) {
        auto D = ev.at_code(table_code(K, k));
        if (D < Db) { Db = D; kb = k; }
    }
    Dbest = Db;
    return kb;
}

// Local walk from k0 towards the strictly lower tabulated neighbour (left
// wins a tie between neighbours) until neither neighbour is lower.
template <class E>
__device__ __forceinline__ int walk_table(const E& ev, int K, int k0, decltype(ev.at_code(0))& Dbest)
{
    int k = k0;
    auto Dk = ev.at_code(table_code(K, k));
    auto Dl = ev.at_code(table_code(K, k == 0 ? K - 1 : k - 1));
    auto Dr = ev.at_code(table_code(K, k == K - 1 ? 0 : k + 1));
    for (int step = 0; step < K; ++step) {
        if (Dl < Dk && Dl <= Dr) {
            Dr = Dk; Dk = Dl; k = (k == 0) ? K - 1 : k - 1;
            Dl = ev.at_code(table_code(K, k == 0 ? K - 1 : k - 1));
        } else if (Dr < Dk) {
            Dl = Dk; Dk = Dr; k = (k == K - 1) ? 0 : k + 1;
            Dr = ev.at_code(table_code(K, k == K - 1 ? 0 : k + 1));
        } else {
            break;
        }
    }
    Dbest = Dk;
    return k;
}

// Golden-section refinement in its discrete (Fibonacci) form on the angle
// lattice inside the bracket of the two tabulated neighbours of k, extended
// to a Fibonacci length with +inf past the upper neighbour.  Returns the best
// evaluated code (the tabulated minimiser included).
template <class E>
__device__ __forceinline__ int fibonacci_refine(const E& ev, int K, int fib_stop, int k,
                                                decltype(ev.at_code(0)) Dk,
                                                decltype(ev.at_code(0))& Dbest)
{
    typedef decltype(ev.at_code(0)) G;
    const int ck = table_code(K, k);
    const int cl = (k == 0) ? table_code(K, K - 1) - kCodes : table_code(K, k - 1);
    const int cr = (k == K - 1) ? kCodes : table_code(K, k + 1);
    const int lo_off = cl - ck, hi_off = cr - ck, L = hi_off - lo_off;
    int n = 2;
    while (kFib[n] < L) ++n;
    int best = ck;
    G qb = Dk;
    int a = lo_off;
    int x1 = a + kFib[n - 2], x2 = a + kFib[n - 1];
    G f1 = (x1 >= hi_off) ? ginf<G>() : ev.at_code(ck + x1);
    G f2 = (x2 >= hi_off) ? ginf<G>() : ev.at_code(ck + x2);
    if (f1 < qb) { qb = f1; best = ck + x1; }
    if (f2 < qb) { qb = f2; best = ck + x2; }
    for (int kk = n; kk > 4 && kFib[kk] > fib_stop; --kk) {
        if (f1 <= f2) {
            x2 = x1; f2 = f1;
            x1 = a + kFib[kk - 3];
            f1 = (x1 >= hi_off) ? ginf<G>() : ev.at_code(ck + x1);
            if (f1 < qb) { qb = f1; best = ck + x1; }
        } else {
            a = x1;
            x1 = x2; f1 = f2;
            x2 = a + kFib[kk - 2];
            f2 = (x2 >= hi_off) ? ginf<G>() : ev.at_code(ck + x2);
            if (f2 < qb) { qb = f2; best = ck + x2; }
        }
    }
    Dbest = qb;
    return wrap_code(best);
}

}  // namespace dpk
