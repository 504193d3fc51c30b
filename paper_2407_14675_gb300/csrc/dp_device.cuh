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

#include <type_traits>

namespace dpk {

constexpr int kCodes = 65536;       // 16-bit angle lattice, alpha = 2 pi c / 65536
constexpr int kBlock = 256;         // threads per block of the sweep kernels
constexpr int kMaxFib = 30;
constexpr int kMaxAngles = 1024;   // tabulated angles per grid (shared-memory table)

enum { kVI = 0, kImproveFull = 1, kImproveWalk = 2, kEval = 3, kEvalFeet = 4, kIncr = 5,
       kEvalDiag = 6, kEvalFeetDiag = 7, kIncrDiag = 8, kVIDiag = 9, kEvalFeet64 = 10, kEvalFeet64Diag = 11,
       kEvalFeet8 = 12 };
// kEvalFeet8: kEvalFeet at 8-byte frozen feet (kEvalFeet: at the word pairs).
// kEval*Diag, kIncrDiag: the evaluation as a Jacobi iteration on the linear
// system of Eq. (13) with each node's own coefficient solved exactly (the
// weight w_jj of node j among the Q1 corners of its own foot):
//   V'_j = V_j + (T_f(V)_j - V_j) / (1 - beta w_jj),
// which has the fixed point of the plain evaluation sweep.  Where the foot
// stays in the node's own cell (w_jj near 1: the mass moves ~0.002 cells per
// step) the plain sweep contracts by beta w_jj ~ 0.997 there; this one does
// not.  kVIDiag: value iteration with the node's own coefficient solved
// inside the minimisation, min_a (c_a + beta R_a) / (1 - beta w_jj^a) (the
// fixed point of Eq. (12); minimum-time dynamics).
enum { kDynOrbit = 0, kDynUnitSpeed = 1, kDynPolar = 2 };
constexpr int kCodeOff = 65535;     // policy code of the thrust-off control

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
    int reach;        // largest |corner index - node index| of the stored frozen feet
                      //   (improvement sweeps fold it in; the multi-level
                      //   evaluation orders its chunks by it)
    int wave_err;     // a multi-level evaluation gave up a bounded wait
    int pad[3];
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
    int foot_dm;               // its cell offset floor(um) and fraction um - floor(um)
    float foot_tm;             //   (grid constants of every frozen foot)
    int dyn;
    int K, refine, fib_stop;   // refinement stops once the bracket is <= fib_stop codes
    int fib_n0;                // Fibonacci index of the shortest refinement bracket
    int tlo[4], thi[4];        // target index box, inclusive (tlo > thi: no target)
    int n_m;
    unsigned long long magic_m;    // ceil(2^40 / n_m): j / n_m for j < 2^40 / (n_m - 1)
    int n_nodes;               // stored nodes
    const int4* rows;          // per (i_r, i_vr): {first compact index, lo_vt, len, 0}
    const int* row_org;        // reduced grids, per (i_r, i_vr): first compact index - lo_vt * n_m, the
                               //   index (v_t = 0, m = 0) would have (4 bytes a row for the feet's lookups)
    const unsigned* lines;     // per compact (r, v_r, v_t) line: i_r | i_vr<<10 | i_vt<<20
    const typename V2<G>::type* tab_hi;   // (sin, cos) of 2 pi (c >> 8) 256 / 65536
    const typename V2<G>::type* tab_lo;   // (sin, cos) of 2 pi (c & 255) / 65536
    // polar dynamics (the paper's Example 1): running cost of Eq. (11)
    int off;                   // thrust off (kCodeOff) is a control
    double cost_b, cost_g;     // weights of (a - a_bar)^2 and of the eccentricity term
    double a_bar, ex_bar, ey_bar;
    double thrust_cost;        // dt alpha |u| of every thrust control
};

template <typename G> __device__ __forceinline__ G ginf();
template <> __device__ __forceinline__ float ginf<float>() { return CUDART_INF_F; }
template <> __device__ __forceinline__ double ginf<double>() { return CUDART_INF; }

// Reciprocal for the geometry: FP32 uses the hardware approximation (about
// 1 ulp); its error moves a foot by ~1e-9 cells, far below FP32 grid noise.
__device__ __forceinline__ float grcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double grcp(double x) { return __drcp_rn(x); }

// 1 / den for the diagonal factor den = 1 - beta w in [1 - beta, 1]: the FP32
// reciprocal refined by two Newton-Raphson steps for 1/x, r <- r + r (1 - den r),
// each of which squares the relative error (about 6e-8, then 4e-15, then the
// FP64 rounding level).  Four FP64 FMAs instead of an FP64 division, whose
// iterations the FP64 pipe would run for every node.
__device__ __forceinline__ double recip_newton(double den)
{
    double r = (double)__frcp_rn((float)den);
    double e = fma(-den, r, 1.0);
    r = fma(r, e, r);
    e = fma(-den, r, 1.0);
    return fma(r, e, r);
}

// Explicitly rounded operations: expressions written with them compile to
// the same instructions in every kernel (no context-dependent contraction).
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Code of the k-th tabulated angle 2 pi k / K on the lattice (round half up).
__device__ __forceinline__ int table_code(int K, int k) { return (k * kCodes + K / 2) / K; }

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
//
// Orbit dynamics: with the control held over the step, the predictor is
// v_r2 = R0 + R1 s, v_t2 = P0 + P1 c (s, c = sin, cos alpha; R1 = P1 = dt a/m),
// and r2, m2 do not depend on alpha.  So the Heun displacement in cells is a
// polynomial in (s, c), expanded once per state:
//   u_r  = a0 + b0 s
//   u_vr = a1 + b1 s + c (g1 + d1 c)      (from the v_t2^2 / r2 term)
//   u_vt = a2 + b2 s + c (g2 + e2 s)      (from the v_r2 v_t2 / r2 term)
// Seven FMAs per control instead of the two-stage step; the terms that do
// not depend on alpha are rounded once for all controls of the state.  The
// polar dynamics (Example 1) are the same with a fixed thrust acceleration
// (no mass), plus the orbital angle u_theta = a3 + g3 c from theta' = v_t / r.
template <typename G>
struct NodeDyn {
    G vr, vt;
    G a0, b0, a1, b1, g1, d1, a2, b2, g2, e2;   // the expanded displacement
    G a3, g3;                                   // polar: the orbital angle's
};

template <typename G, int DYN>
__device__ __forceinline__ NodeDyn<G> node_dyn(const Geo<G>& g, const StepP<G>& sp, const G x[4])
{
    NodeDyn<G> n;
    n.vr = x[1];
    n.vt = x[2];
    if (DYN == kDynOrbit || DYN == kDynPolar) {
        // every operation rounded explicitly: the searches, the stored feet and
        // the recomputing sweeps run this in different kernels and must agree
        const G ir = grcp(x[0]);
        const G d1vr = xfma(xmul(n.vt, n.vt), ir, -xmul(g.mu, xmul(ir, ir)));
        const G d1vt = -xmul(xmul(n.vr, n.vt), ir);
        const G ir2 = grcp(xfma(sp.dt, n.vr, x[0]));
        const G muir2sq = xmul(g.mu, xmul(ir2, ir2));
        G am = g.accel, am2 = g.accel;   // polar: no mass, the thrust acceleration is fixed
        if (DYN == kDynOrbit) {
            am = xmul(g.accel, grcp(x[3]));
            am2 = xmul(g.accel, grcp(xfma(sp.dt, g.mdot, x[3])));
        }
        const G R0 = xfma(sp.dt, d1vr, n.vr), P0 = xfma(sp.dt, d1vt, n.vt), R1 = xmul(sp.dt, am), P1 = R1;
        const G h0 = xmul(sp.hdt, g.ih[0]), h1 = xmul(sp.hdt, g.ih[1]), h2 = xmul(sp.hdt, g.ih[2]);
        const G amm = xadd(am, am2);
        const G q = xmul(P0, ir2), p1r = xmul(P1, ir2);   // P0 / r2, P1 / r2
        n.a0 = xmul(h0, xadd(n.vr, R0));
        n.b0 = xmul(h0, R1);
        n.a1 = xmul(h1, xadd(d1vr, xfma(P0, q, -muir2sq)));
        n.b1 = xmul(h1, amm);
        n.g1 = xmul(h1, xmul(xadd(P1, P1), q));
        n.d1 = xmul(h1, xmul(P1, p1r));
        n.a2 = xmul(h2, xfma(-R0, q, d1vt));
        n.b2 = -xmul(h2, xmul(R1, q));
        n.g2 = xmul(h2, xfma(-R0, p1r, amm));
        n.e2 = -xmul(h2, xmul(R1, p1r));
        if (DYN == kDynPolar) {
            // the orbital angle, theta' = v_t / r: u_theta = a3 + g3 c
            const G h3 = xmul(sp.hdt, g.ih[3]);
            n.a3 = xmul(h3, xfma(n.vt, ir, q));
            n.g3 = xmul(h3, p1r);
        }
    }
    return n;
}

// Heun displacement in cells for control (s, c) = (sin alpha, cos alpha):
// k1 = b(x), k2 = b(x + dt k1), u = dt (k1 + k2) / 2 / h.
template <typename G, int DYN>
__device__ __forceinline__ void heun_cells(const Geo<G>& g, const StepP<G>& sp, const NodeDyn<G>& n,
                                           G s, G c, G u[4])
{
    if (DYN == kDynOrbit || DYN == kDynPolar) {
        u[0] = xfma(n.b0, s, n.a0);
        u[1] = xfma(c, xfma(n.d1, c, n.g1), xfma(n.b1, s, n.a1));
        u[2] = xfma(c, xfma(n.e2, s, n.g2), xfma(n.b2, s, n.a2));
        u[3] = DYN == kDynOrbit ? sp.um : xfma(n.g3, c, n.a3);
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

// Cell of the foot i + u (grid units): c = i + floor(u), t = u - floor(u).
// A foot exactly on an upper face uses the last cell with t = 1.  Returns
// true when the foot is outside the box (strictly) or not finite.
template <typename G>
__device__ __forceinline__ bool foot_dim(int n, int i, G u, int& c, G& t)
{
    G fl = floor(u);
    t = u - fl;
    c = i + (int)fl;
    bool out = !(t >= (G)0);
    if ((unsigned)c > (unsigned)(n - 2)) {   // outside, or on the upper face
        out = out || c != n - 1 || t > (G)0;
        c = n - 2;
        t = (G)1;
    }
    return out;
}

// The periodic angle coordinate: the cell index wraps, nothing is outside.
template <typename G>
__device__ __forceinline__ bool foot_dim_periodic(int n, int i, G u, int& c, G& t)
{
    G fl = floor(u);
    t = u - fl;
    int cc = (i + (int)fl) % n;
    c = cc < 0 ? cc + n : cc;
    return !(t >= (G)0);
}

template <typename G, bool PER3 = false>
__device__ __forceinline__ bool foot_cell(const Geo<G>& g, const int i[4], const G u[4], int c[4], G t[4])
{
    bool out = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) out = foot_dim(g.n[d], i[d], u[d], c[d], t[d]) || out;
    if (PER3) out = foot_dim_periodic(g.n[3], i[3], u[3], c[3], t[3]) || out;
    else out = foot_dim(g.n[3], i[3], u[3], c[3], t[3]) || out;
    return out;
}

// Offset from the lower to the upper corner in the last coordinate (the
// periodic angle wraps from node n-1 to node 0).
template <typename G, bool PER3>
__device__ __forceinline__ int up3(const Geo<G>& g, int c3)
{
    return (PER3 && c3 == g.n[3] - 1) ? 1 - g.n[3] : 1;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// Paired FP32 arithmetic (two IEEE round-to-nearest results per instruction).
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The 16 corner values of a cell as differences to the node's value, ready
// for the blend.  Corner x = 4 r + 2 v_r + v_t (bits of the cell corner) has
// e0[x] at the lower mass node and de[x] = step to the upper mass node.
// blend(t) lerps along m, v_t, v_r, r in that order; the FP32 version does
// the same lerps two at a time (pairs x and x + 4), with identical rounding.
template <typename G> struct Corners;

template <> struct Corners<double> {
    double e0[8], de[8];
    __device__ __forceinline__ void set(const double a[8], const double d[8])
    {
#pragma unroll
        for (int x = 0; x < 8; ++x) { e0[x] = a[x]; de[x] = d[x]; }
    }
    __device__ __forceinline__ double blend(const double t[4]) const
    {
        double e[8], f[4];
#pragma unroll
        for (int x = 0; x < 8; ++x) e[x] = e0[x] + t[3] * de[x];
#pragma unroll
        for (int y = 0; y < 4; ++y) f[y] = e[2 * y] + t[2] * (e[2 * y + 1] - e[2 * y]);
        double h0 = f[0] + t[1] * (f[1] - f[0]);
        double h1 = f[2] + t[1] * (f[3] - f[2]);
        return h0 + t[0] * (h1 - h0);
    }
    // the lerp along m done once for a fixed mass fraction (e0 then holds
    // it); blend_m_folded(t) equals blend(t) for that fraction
    __device__ __forceinline__ void fold_m(double t3)
    {
#pragma unroll
        for (int x = 0; x < 8; ++x) e0[x] = e0[x] + t3 * de[x];
    }
    __device__ __forceinline__ double blend_m_folded(const double t[4]) const
    {
        double f[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) f[y] = e0[2 * y] + t[2] * (e0[2 * y + 1] - e0[2 * y]);
        double h0 = f[0] + t[1] * (f[1] - f[0]);
        double h1 = f[2] + t[1] * (f[3] - f[2]);
        return h0 + t[0] * (h1 - h0);
    }
};

template <> struct Corners<float> {
    unsigned long long q0[4], qd[4];   // (e0[x], e0[x + 4]), (de[x], de[x + 4])
    __device__ __forceinline__ void set(const float a[8], const float d[8])
    {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            q0[x] = pack2(a[x], a[x + 4]);
            qd[x] = pack2(d[x], d[x + 4]);
        }
    }
    __device__ __forceinline__ float blend(const float t[4]) const
    {
        const unsigned long long t3 = pack2(t[3], t[3]), t2 = pack2(t[2], t[2]), t1 = pack2(t[1], t[1]);
        unsigned long long Q[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) Q[x] = fma2(qd[x], t3, q0[x]);              // along m
        unsigned long long R0 = fma2(sub2(Q[1], Q[0]), t2, Q[0]);               // along v_t
        unsigned long long R1 = fma2(sub2(Q[3], Q[2]), t2, Q[2]);
        unsigned long long S = fma2(sub2(R1, R0), t1, R0);                      // along v_r
        float h0, h1;
        unpack2(S, h0, h1);
        return h0 + t[0] * (h1 - h0);                                            // along r
    }
    __device__ __forceinline__ void fold_m(float t3)
    {
        const unsigned long long tt = pack2(t3, t3);
#pragma unroll
        for (int x = 0; x < 4; ++x) q0[x] = fma2(qd[x], tt, q0[x]);
    }
    __device__ __forceinline__ float blend_m_folded(const float t[4]) const
    {
        const unsigned long long t2 = pack2(t[2], t[2]), t1 = pack2(t[1], t[1]);
        unsigned long long R0 = fma2(sub2(q0[1], q0[0]), t2, q0[0]);
        unsigned long long R1 = fma2(sub2(q0[3], q0[2]), t2, q0[2]);
        unsigned long long S = fma2(sub2(R1, R0), t1, R0);
        float h0, h1;
        unpack2(S, h0, h1);
        return h0 + t[0] * (h1 - h0);
    }
};

// Gathers the corners of cell c.  Returns true when a corner lies outside
// the node set (reduced grids: the cell's four (r, v_r) rows must each hold
// both v_t corners); the corners are then not loaded.
template <typename G, bool REDUCED>
__device__ __forceinline__ bool cell_rows(const Geo<G>& g, const int c[4], int base[4])
{
    // per (r, v_r) corner row rb = 2 r + v_r: index of corner (c_vt, c_m)
    if (!REDUCED) {
        const int b0 = c[0] * g.stride[0] + c[1] * g.stride[1] + c[2] * g.stride[2] + c[3];
        base[0] = b0;
        base[1] = b0 + g.stride[1];
        base[2] = b0 + g.stride[0];
        base[3] = b0 + g.stride[0] + g.stride[1];
        return false;
    }
    bool out = false;
#pragma unroll
    for (int rb = 0; rb < 4; ++rb) {
        int row = (c[0] + (rb >> 1)) * g.n[1] + c[1] + (rb & 1);
        int4 R = __ldg(&g.rows[row]);
        out = out || c[2] < R.y || c[2] + 1 > R.y + R.z - 1;
        base[rb] = R.x + (c[2] - R.y) * g.n_m + c[3];
    }
    return out;
}

// Loads the 16 corners given the index of corner (c_vt, c_m) in each of the
// four (r, v_r) rows (n_m: stride of v_t).  The lower mass corner enters as
// its difference to vj, the step to the upper one as v_upper - v_lower
// (one rounding, in the value type).
template <typename G, typename S>
__device__ __forceinline__ void load_rows(const S* __restrict__ V, const int base[4], int n_m, S vj, Corners<G>& K,
                                          int up = 1)
{
    G a[8], d[8];
#pragma unroll
    for (int rb = 0; rb < 4; ++rb) {
        const S* p = V + base[rb];
        S v00 = __ldg(p), v01 = __ldg(p + up), v10 = __ldg(p + n_m), v11 = __ldg(p + n_m + up);
        a[2 * rb] = (G)(v00 - vj);
        d[2 * rb] = (G)(v01 - v00);
        a[2 * rb + 1] = (G)(v10 - vj);
        d[2 * rb + 1] = (G)(v11 - v10);
    }
    K.set(a, d);
}

// Weak global load through L1 (ld.global): for values that other blocks of
// the same launch write (the multi-level evaluation), where the read-only
// path (ld.global.nc) may return stale data.  volatile keeps it after the
// acquire fence and block barrier that make those writes visible.
__device__ __forceinline__ float ld_coherent(const float* p)
{
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// FP32 values and blend: the same differences, two per paired instruction,
// written straight into the pairs (x, x + 4) of Corners<float>: row rb and
// row rb + 2 of the same v_t corner.  COH: coherent loads (ld_coherent).
template <bool COH>
__device__ __forceinline__ void load_rows_f32(const float* __restrict__ V, const int base[4], int n_m, float vj,
                                              Corners<float>& K, int up = 1)
{
    float v00[4], v01[4], v10[4], v11[4];
#pragma unroll
    for (int rb = 0; rb < 4; ++rb) {
        const float* p = V + base[rb];
        if constexpr (COH) {
            v00[rb] = ld_coherent(p);
            v01[rb] = ld_coherent(p + up);
            v10[rb] = ld_coherent(p + n_m);
            v11[rb] = ld_coherent(p + n_m + up);
        } else {
            v00[rb] = __ldg(p);
            v01[rb] = __ldg(p + up);
            v10[rb] = __ldg(p + n_m);
            v11[rb] = __ldg(p + n_m + up);
        }
    }
    const unsigned long long jj = pack2(vj, vj);
#pragma unroll
    for (int rb = 0; rb < 2; ++rb) {
        const unsigned long long lo0 = pack2(v00[rb], v00[rb + 2]), lo1 = pack2(v10[rb], v10[rb + 2]);
        K.q0[2 * rb] = sub2(lo0, jj);
        K.qd[2 * rb] = sub2(pack2(v01[rb], v01[rb + 2]), lo0);
        K.q0[2 * rb + 1] = sub2(lo1, jj);
        K.qd[2 * rb + 1] = sub2(pack2(v11[rb], v11[rb + 2]), lo1);
    }
}

template <>
__device__ __forceinline__ void load_rows<float, float>(const float* __restrict__ V, const int base[4], int n_m,
                                                        float vj, Corners<float>& K, int up)
{
    load_rows_f32<false>(V, base, n_m, vj, K, up);
}

// Type in which D = I[V] - V_j is blended and compared: FP64 when the values
// are FP64 (so that decisions resolve differences far below V), else the
// geometry type.
template <typename G, typename S>
struct BlendType {
    typedef typename std::conditional<std::is_same<S, double>::value, double, G>::type type;
};

template <typename R, typename G, typename S, bool REDUCED, bool PER3 = false>
__device__ __forceinline__ bool load_corners(const Geo<G>& g, const S* __restrict__ V, const int c[4], S vj,
                                             Corners<R>& K)
{
    int base[4];
    if (cell_rows<G, REDUCED>(g, c, base)) return true;
    load_rows<R, S>(V, base, g.n_m, vj, K, up3<G, PER3>(g, c[3]));
    return false;
}

// Frozen foot of a node under a fixed policy (FP32 geometry).  Policy
// evaluation sweeps repeat the same foot ~20 times, so the improvement sweep
// stores it and the evaluation sweep only gathers and blends.  With FP64
// values (12 bytes in two arrays):
//   lo (64 bits): t_r bits 0-23, t_vr bits 24-47, low 16 bits of t_vt 48-63
//   hi (32 bits): high 8 bits of t_vt 0-7, cell offset from the node in r
//                 (-2..1) bits 8-9, v_r (-8..7) bits 10-13, v_t (-2..1) bits
//                 14-15, kind bits 16-17 (inside, outside -> penalty M, target
//                 node, or "recompute from the policy code")
// Fractions are 24-bit fixed point q / (2^24 - 1), about FP32 resolution, so
// repeated evaluation does not drift from the recomputed operator.  The mass
// coordinate needs no storage: m' = -a/c is the same at every node, so its
// offset and fraction are grid constants (a node where they differ, at the
// upper mass face, is marked "recompute").
enum { kFootInside = 0, kFootOut = 1, kFootTarget = 2, kFootRecompute = 3 };
constexpr float kFootQ = 16777215.0f;   // 2^24 - 1

// The FP32-value phase stores the same foot in one 8-byte word (no second
// array to stream): fractions t_r bits 0-17, t_vr 18-35, t_vt 36-53 as 18-bit
// fixed point q / (2^18 - 1); cell offsets r (-2..1) bits 54-55, v_r (-8..7)
// 56-59, v_t (-2..1) 60-61; kind bits 62-63.  The quantisation step, 3.8e-6
// of a cell, is about the rounding of the FP32 one-step map itself for
// displacements of a few cells (v_r); the FP64-value phase, whose values
// converge far below FP32 resolution, keeps the 24-bit word pair.
constexpr float kFoot8Q = 262143.0f;    // 2^18 - 1

struct FootWord {
    unsigned long long lo;
    unsigned hi;
};

// Frozen feet of FP64 grids.  The FP64 evaluation sweep otherwise repeats the
// FP64 one-step map and, for the paper's Example 1, the running cost of
// Eq. (11) at every node in every sweep.  Per node: a word with the kind
// (bits 32-33) and the cell's offsets from the node as int8 (coordinate d in
// bits 8d..8d+7), the four fractions in FP64 (two double2), and the constant
// part c_j of the node's update under its control (dt l(x_j, control), the
// thrust cost included).  Evaluation from them gives the recomputing sweep's
// results bit for bit for the minimum-time dynamics; with the running cost of
// Eq. (11), computed in another kernel, to an ulp of the constant.
struct Feet64 {
    unsigned long long* w = nullptr;
    double2* t = nullptr;
    double* c = nullptr;
};

__device__ __forceinline__ FootWord foot_word_kind(int kind)
{
    return FootWord{0ull, (unsigned)kind << 16};
}

__device__ __forceinline__ unsigned long long foot8_kind(int kind) { return (unsigned long long)kind << 62; }
__device__ __forceinline__ int foot8_kind_of(unsigned long long w) { return (int)(w >> 62); }

// Encodes cell c and fractions t of a foot from node i in the 8-byte word.
__device__ __forceinline__ unsigned long long encode_foot8(const int i[4], const int c[4], const float t[4], int dm,
                                                           float tm)
{
    const int dr = c[0] - i[0], dv = c[1] - i[1], dt = c[2] - i[2];
    if (dr < -2 || dr > 1 || dv < -8 || dv > 7 || dt < -2 || dt > 1 || c[3] - i[3] != dm || t[3] != tm)
        return foot8_kind(kFootRecompute);
    const unsigned long long q0 = __float2uint_rn(t[0] * kFoot8Q);
    const unsigned long long q1 = __float2uint_rn(t[1] * kFoot8Q);
    const unsigned long long q2 = __float2uint_rn(t[2] * kFoot8Q);
    return q0 | (q1 << 18) | (q2 << 36) | ((unsigned long long)(dr + 2) << 54) |
           ((unsigned long long)(dv + 8) << 56) | ((unsigned long long)(dt + 2) << 60);
}

// Encodes cell c and fractions t of a foot from node i; dm, tm: the grid's
// mass offset and fraction.
__device__ __forceinline__ FootWord encode_foot(const int i[4], const int c[4], const float t[4], int dm, float tm)
{
    const int dr = c[0] - i[0], dv = c[1] - i[1], dt = c[2] - i[2];
    if (dr < -2 || dr > 1 || dv < -8 || dv > 7 || dt < -2 || dt > 1 || c[3] - i[3] != dm || t[3] != tm)
        return foot_word_kind(kFootRecompute);
    const unsigned q0 = __float2uint_rn(t[0] * kFootQ);
    const unsigned q1 = __float2uint_rn(t[1] * kFootQ);
    const unsigned q2 = __float2uint_rn(t[2] * kFootQ);
    FootWord w;
    w.lo = (unsigned long long)q0 | ((unsigned long long)q1 << 24) | ((unsigned long long)(q2 & 0xffffu) << 48);
    w.hi = (q2 >> 16) | ((unsigned)(dr + 2) << 8) | ((unsigned)(dv + 8) << 10) | ((unsigned)(dt + 2) << 14);
    return w;
}

// Weight of node i among the Q1 corners of cell c with fractions t (0 when i
// is not a corner of the cell).
template <typename G, bool PER3>
__device__ __forceinline__ G self_weight(const Geo<G>& g, const int i[4], const int c[4], const G t[4])
{
    G w = (G)1;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        int hi = c[d] + 1;
        if (PER3 && d == 3 && hi == g.n[3]) hi = 0;
        w *= i[d] == c[d] ? (G)1 - t[d] : (i[d] == hi ? t[d] : (G)0);
    }
    return w;
}

// Q1 interpolation at the foot i + u (grid units), returned as the difference
// D = I[V] - vj; M - vj when the foot is outside the box or the node set.
template <typename G, typename S, bool REDUCED, bool PER3 = false>
__device__ __forceinline__ typename BlendType<G, S>::type interp_delta(const Geo<G>& g, const S* __restrict__ V,
                                                                       const int i[4], const G u[4], S vj)
{
    typedef typename BlendType<G, S>::type R;
    int c[4];
    G t[4];
    Corners<R> K;
    if (foot_cell<G, PER3>(g, i, u, c, t) || load_corners<R, G, S, REDUCED, PER3>(g, V, c, vj, K))
        return (R)((S)g.M64 - vj);
    const R tr[4] = {(R)t[0], (R)t[1], (R)t[2], (R)t[3]};
    return K.blend(tr);
}

// The same, also returning the node's own weight among the corners (0 when
// the foot is outside: that row of the system is empty).
template <typename G, typename S, bool REDUCED, bool PER3 = false>
__device__ __forceinline__ typename BlendType<G, S>::type interp_delta_w(const Geo<G>& g, const S* __restrict__ V,
                                                                         const int i[4], const G u[4], S vj,
                                                                         typename BlendType<G, S>::type& wself)
{
    typedef typename BlendType<G, S>::type R;
    int c[4];
    G t[4];
    Corners<R> K;
    wself = (R)0;
    if (foot_cell<G, PER3>(g, i, u, c, t) || load_corners<R, G, S, REDUCED, PER3>(g, V, c, vj, K))
        return (R)((S)g.M64 - vj);
    const R tr[4] = {(R)t[0], (R)t[1], (R)t[2], (R)t[3]};
    wself = (R)self_weight<G, PER3>(g, i, c, t);
    return K.blend(tr);
}

// Control-dependent evaluation at one state: node i plus the offset u0 (both
// in grid units; u0 = 0 at a grid node).  One interpolation per call.
template <typename G, typename S, bool REDUCED, int DYN>
struct NodeEval {
    typedef typename BlendType<G, S>::type R;
    static constexpr bool kMayOff = DYN == kDynPolar;   // only these dynamics have the thrust-off code
    const Geo<G>* g;
    const S* __restrict__ V;
    StepP<G> sp;
    int i[4];
    G u0[4];
    S vj;
    NodeDyn<G> nd;

    __device__ __forceinline__ R at_sc(G s, G c)
    {
        G u[4];
        heun_cells<G, DYN>(*g, sp, nd, s, c, u);
#pragma unroll
        for (int d = 0; d < 4; ++d) u[d] += u0[d];
        return interp_delta<G, S, REDUCED, DYN == kDynPolar>(*g, V, i, u, vj);
    }

    __device__ __forceinline__ R at_code(int code)
    {
        G s, c;
        code_sincos(*g, code, s, c);
        return at_sc(s, c);
    }

    // with the node's own weight among the corners
    __device__ __forceinline__ R at_sc_w(G s, G c, R& wself)
    {
        G u[4];
        heun_cells<G, DYN>(*g, sp, nd, s, c, u);
#pragma unroll
        for (int d = 0; d < 4; ++d) u[d] += u0[d];
        return interp_delta_w<G, S, REDUCED, DYN == kDynPolar>(*g, V, i, u, vj, wself);
    }

    __device__ __forceinline__ R at_code_w(int code, R& wself)
    {
        G s, c;
        code_sincos(*g, code, s, c);
        return at_sc_w(s, c, wself);
    }
};

// The same evaluation for searches over many angles at one state: the
// corners of the last cell used stay in registers.  Thrust moves the foot by
// about 1e-3 cells across all angles, so nearly every angle after the first
// costs the Heun step and the blend, with no memory access.  With the default
// blend type the results are bit-identical to NodeEval; BLEND = float with
// FP64 values blends the FP64 corner differences V_c - V_j rounded to FP32.
//
// The mass displacement does not depend on the control, so the mass
// coordinate of the foot is found once per state (reset(), after vj, u0 and
// the dynamics are set).  OFF = false: the state is a grid node (u0 = 0).
template <typename G, typename S, bool REDUCED, int DYN, typename BLEND = typename BlendType<G, S>::type,
          bool OFF = true, bool DIAG = false>
struct CachedEval {
    typedef BLEND R;
    static constexpr bool kMayOff = DYN == kDynPolar;   // only these dynamics have the thrust-off code
    const Geo<G>* g;
    const S* __restrict__ V;
    StepP<G> sp;
    int i[4];
    G u0[4];
    S vj;
    NodeDyn<G> nd;
    int cc[3];        // cached cell in (r, v_r, v_t); cc[0] = -1: none
    G co[3];          // its offset from the node, cc - i
    bool cout;        // the cached cell has a corner outside the node set
    Corners<R> K;
    R pen;            // M - vj
    int cm;           // mass cell and fraction of every foot of this state
    G tm;
    bool outm;

    __device__ __forceinline__ void reset()
    {
        cc[0] = -1;
        pen = (R)((S)g->M64 - vj);
        if (DYN != kDynPolar) outm = foot_dim(g->n[3], i[3], OFF ? sp.um + u0[3] : sp.um, cm, tm);
        else outm = false;
    }

    // 0 <= t < 1 (false for NaN and -0)
    static __device__ __forceinline__ bool unit_fraction(float t) { return __float_as_uint(t) < 0x3f800000u; }
    static __device__ __forceinline__ bool unit_fraction(double t)
    {
        return (unsigned long long)__double_as_longlong(t) < 0x3ff0000000000000ull;
    }

    __device__ __forceinline__ R at_code(int code)
    {
        G s, c;
        code_sincos(*g, code, s, c);
        return at_sc(s, c);
    }

    __device__ __forceinline__ R at_sc(G s, G c)
    {
        G u[4], t[4];
        int cl[4];
        heun_cells<G, DYN>(*g, sp, nd, s, c, u);
        if (OFF) {
#pragma unroll
            for (int d = 0; d < 3; ++d) u[d] += u0[d];
        }
        if constexpr (DYN != kDynPolar) {
            // the usual case: the foot lies in the cached cell, whose fractions
            // are u - (cell - node) in [0, 1), the same numbers foot_dim gives
            if (cc[0] >= 0) {
                bool in = true;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    t[d] = u[d] - co[d];
                    in = in && unit_fraction(t[d]);
                }
                if (in) {
                    if (cout) return pen;
#pragma unroll
                    for (int d = 0; d < 3; ++d) cl[d] = cc[d];
                    cl[3] = cm;
                    t[3] = tm;
                    return blend_at(cl, t);
                }
            }
        }
        bool out = outm;
#pragma unroll
        for (int d = 0; d < 3; ++d) out = foot_dim(g->n[d], i[d], u[d], cl[d], t[d]) || out;
        if (DYN == kDynPolar) {
            // the angle moves with the control: its cell is found every time
            out = foot_dim_periodic(g->n[3], i[3], OFF ? u[3] + u0[3] : u[3], cl[3], t[3]) || out;
        }
        if (out) return pen;
        if (DYN != kDynPolar) {
            cl[3] = cm;
            t[3] = tm;
        }
        if (cl[0] != cc[0] || cl[1] != cc[1] || cl[2] != cc[2] || (DYN == kDynPolar && cl[3] != cm)) {
            cout = load_corners<R, G, S, REDUCED, DYN == kDynPolar>(*g, V, cl, vj, K);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                cc[d] = cl[d];
                co[d] = (G)(cl[d] - i[d]);
            }
            if (DYN == kDynPolar) cm = cl[3];
            else K.fold_m((R)tm);   // every foot of this state has the same mass fraction
        }
        if (cout) return pen;
        return blend_at(cl, t);
    }

    // D at the cached corners for cell cl, fractions t
    __device__ __forceinline__ R blend_at(const int cl[4], const G t[4]) const
    {
        const R tr[4] = {(R)t[0], (R)t[1], (R)t[2], (R)t[3]};
        const R D = DYN == kDynPolar ? K.blend(tr) : K.blend_m_folded(tr);
        if constexpr (DIAG) {
            // the node's own coefficient solved (grid node, l = 1): return the
            // difference D~ with dt + beta (vj + D~) = vj + r / (1 - beta w),
            // r = dt + beta (vj + D) - vj the plain update's change and w the
            // node's own weight among the corners; D~ = D + w r / (1 - beta w)
            // orders the controls as the solved values do
            const R w = (R)self_weight<G, DYN == kDynPolar>(*g, i, cl, t);
            const R beta = std::is_same<R, double>::value ? (R)g->beta64 : (R)(g->beta_hi + g->beta_lo);
            const R dt = std::is_same<R, double>::value ? (R)g->dt64 : (R)g->dt;
            const R vr = (R)vj;
            const R r = dt + beta * (vr + D) - vr;
            if constexpr (std::is_same<R, double>::value) return D + w * r * recip_newton((R)1 - beta * w);
            else return D + w * r / ((R)1 - beta * w);
        }
        return D;
    }

    // FP64 frozen foot of this node for the control (s, c) (sine and cosine;
    // 0, 0 for thrust off): returns the word, fractions in t.
    __device__ __forceinline__ unsigned long long foot64_of(G s, G c, G t[4]) const
    {
        G u[4];
        int cl[4], base[4];
        heun_cells<G, DYN>(*g, sp, nd, s, c, u);
#pragma unroll
        for (int d = 0; d < 4; ++d) u[d] += u0[d];
        if (foot_cell<G, DYN == kDynPolar>(*g, i, u, cl, t)) return (unsigned long long)kFootOut << 32;
        if (REDUCED && cell_rows<G, REDUCED>(*g, cl, base)) return (unsigned long long)kFootOut << 32;
        unsigned long long w = (unsigned long long)kFootInside << 32;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int off = cl[d] - i[d];
            if (off < -128 || off > 127) return (unsigned long long)kFootRecompute << 32;
            w |= (unsigned long long)(unsigned char)(signed char)off << (8 * d);
        }
        return w;
    }

    // Cell cl and fractions t of this node's foot for a code (FP32 geometry
    // only); false when the foot is outside the box or the node set.
    __device__ __forceinline__ bool foot_at(int code, int cl[4], G t[4]) const
    {
        G s, c, u[4];
        int base[4];
        code_sincos(*g, code, s, c);
        heun_cells<G, DYN>(*g, sp, nd, s, c, u);
#pragma unroll
        for (int d = 0; d < 4; ++d) u[d] += u0[d];
        if (foot_cell(*g, i, u, cl, t)) return false;
        if (REDUCED && cell_rows<G, REDUCED>(*g, cl, base)) return false;
        return true;
    }

    // Frozen-foot word pair of this node for a code (FP32 geometry only).
    // cell (nullable) receives the foot's cell when it has corners (kinds
    // inside and recompute).
    __device__ __forceinline__ FootWord foot_of(int code, int* cell = nullptr) const
    {
        G t[4];
        int cl[4];
        if (!foot_at(code, cl, t)) return foot_word_kind(kFootOut);
        if (cell) {
#pragma unroll
            for (int d = 0; d < 4; ++d) cell[d] = cl[d];
        }
        return encode_foot(i, cl, t, g->foot_dm, g->foot_tm);
    }

    // The same foot as one 8-byte word.
    __device__ __forceinline__ unsigned long long foot8_of(int code, int* cell = nullptr) const
    {
        G t[4];
        int cl[4];
        if (!foot_at(code, cl, t)) return foot8_kind(kFootOut);
        if (cell) {
#pragma unroll
            for (int d = 0; d < 4; ++d) cell[d] = cl[d];
        }
        return encode_foot8(i, cl, t, g->foot_dm, g->foot_tm);
    }
};

// Tabulated angles: codes c_k of 2 pi k / K for k = 0..K (c_K = 65536) and
// (sin, cos) of c_k for k < K.  Kernels that search over angles build it
// once per block in shared memory (build_table), so the searches do no
// integer division and no trig lookup for tabulated angles.
template <typename G>
struct Table {
    const int* code;
    const typename V2<G>::type* sc;
    int K;
    int off = 0;     // the lattice code kCodeOff stands for thrust off
};

template <typename G>
__device__ __forceinline__ void build_table(const Geo<G>& g, int* code, typename V2<G>::type* sc)
{
    for (int k = threadIdx.x; k <= g.K; k += blockDim.x) {
        int c = table_code(g.K, k);
        code[k] = c;
        if (k < g.K) {
            G s, cs;
            code_sincos(g, c, s, cs);
            sc[k].x = s;
            sc[k].y = cs;
        }
    }
}

// Nearest tabulated index to a code (start of the local walk).
__device__ __forceinline__ int nearest_index(int K, int code)
{
    int k = (code * K + kCodes / 2) >> 16;
    return k >= K ? k - K : k;
}

// Full tabulation; ties go to the lowest index.
template <class E, typename G>
__device__ __forceinline__ int enumerate_table(E& ev, const Table<G>& T, typename E::R& Dbest)
{
    typedef typename E::R R;
    R Db = ev.at_sc(T.sc[0].x, T.sc[0].y);
    int kb = 0;
    for (int k = 1; k < T.K; ++k) {
        R D = ev.at_sc(T.sc[k].x, T.sc[k].y);
        if (D < Db) { Db = D; kb = k; }
    }
    Dbest = Db;
    return kb;
}

// Local walk from k0 towards the strictly lower tabulated neighbour (left
// wins a tie between neighbours) until neither neighbour is lower.
template <class E, typename G>
__device__ __forceinline__ int walk_table(E& ev, const Table<G>& T, int k0, typename E::R& Dbest)
{
    typedef typename E::R R;
    const int K = T.K;
    int k = k0;
    int kl = k == 0 ? K - 1 : k - 1, kr = k == K - 1 ? 0 : k + 1;
    R Dk = ev.at_sc(T.sc[k].x, T.sc[k].y);
    R Dl = ev.at_sc(T.sc[kl].x, T.sc[kl].y);
    R Dr = ev.at_sc(T.sc[kr].x, T.sc[kr].y);
    // one evaluation per step, outside the branch, so that lanes of a warp that
    // walk in different directions share it
    for (int step = 0; step < K; ++step) {
        const bool go_l = Dl < Dk && Dl <= Dr;
        if (!go_l && !(Dr < Dk)) break;
        int kn;
        if (go_l) {
            Dr = Dk; Dk = Dl; k = kl;
            kl = k == 0 ? K - 1 : k - 1;
            kn = kl;
        } else {
            Dl = Dk; Dk = Dr; k = kr;
            kr = k == K - 1 ? 0 : k + 1;
            kn = kr;
        }
        const R Dn = ev.at_sc(T.sc[kn].x, T.sc[kn].y);
        if (go_l) Dl = Dn;
        else Dr = Dn;
    }
    Dbest = Dk;
    return k;
}

// Golden-section refinement in its discrete (Fibonacci) form on the angle
// lattice inside the bracket of the two tabulated neighbours of k, extended
// to a Fibonacci length with +inf past the upper neighbour.  Returns the best
// evaluated code (the tabulated minimiser included).  n0 is a lower bound of
// the Fibonacci index of the bracket length.
template <class E, typename G>
__device__ __forceinline__ int fibonacci_refine(E& ev, const Table<G>& T, int n0, int fib_stop, int k,
                                                typename E::R Dk, typename E::R& Dbest)
{
    typedef typename E::R R;
    const int ck = T.code[k];
    const int cl = (k == 0) ? T.code[T.K - 1] - kCodes : T.code[k - 1];
    const int cr = T.code[k + 1];
    const int lo_off = cl - ck, hi_off = cr - ck, L = hi_off - lo_off;
    int n = n0;
    while (kFib[n] < L) ++n;
    int best = ck;
    R qb = Dk;
    int a = lo_off;
    int x1 = a + kFib[n - 2], x2 = a + kFib[n - 1];
    R f1 = (x1 >= hi_off || (E::kMayOff && T.off && wrap_code(ck + x1) == kCodeOff)) ? ginf<R>() : ev.at_code(ck + x1);
    R f2 = (x2 >= hi_off || (E::kMayOff && T.off && wrap_code(ck + x2) == kCodeOff)) ? ginf<R>() : ev.at_code(ck + x2);
    if (f1 < qb) { qb = f1; best = ck + x1; }
    if (f2 < qb) { qb = f2; best = ck + x2; }
    for (int kk = n; kk > 4 && kFib[kk] > fib_stop; --kk) {
        // keep [a, x2] (new point a + F[kk-3]) or [x1, a + F[kk]] (new point
        // x1 + F[kk-2]); one evaluation per step, outside the branch
        const bool left = f1 <= f2;
        int xn;
        if (left) {
            x2 = x1; f2 = f1;
            x1 = a + kFib[kk - 3];
            xn = x1;
        } else {
            a = x1;
            x1 = x2; f1 = f2;
            x2 = a + kFib[kk - 2];
            xn = x2;
        }
        const bool skip = xn >= hi_off || (E::kMayOff && T.off && wrap_code(ck + xn) == kCodeOff);
        const R fn = skip ? ginf<R>() : ev.at_code(ck + xn);
        if (left) f1 = fn;
        else f2 = fn;
        if (fn < qb) { qb = fn; best = ck + xn; }
    }
    Dbest = qb;
    return wrap_code(best);
}

}  // namespace dpk
