// dp_loop.cu -- approximate optimal feedback (§3 Eq. (15)) and its closed
// loop (§3 "Computation of the approximate optimal solution").
//
// One warp per state or trajectory.  The feedback at a state y minimises
// tau + beta_tau I[V](y + tau Phi(y, alpha)): the lanes split the tabulated
// angles, a warp argmin (lowest index on ties) picks the tabulated minimiser,
// and the whole warp then runs the same golden-section (Fibonacci) refinement
// as the improvement sweep.  The closed loop holds that angle over one
// classical RK4 step of the dynamics (FP64 state) and repeats until the state
// enters the target or the step budget ends.
#include "dp_host.h"
#include "dp_sweep.cuh"

namespace dpk {

template <int DYN>
__device__ __forceinline__ void dyn64(const double y[4], double s, double c, double mu, double accel,
                                      double mdot, double drag, double f[4])
{
    if (DYN == kDynOrbit) {
        double am = accel / y[3];
        f[0] = y[1];
        f[1] = y[2] * y[2] / y[0] - mu / (y[0] * y[0]) + am * s;
        f[2] = -y[1] * y[2] / y[0] + am * c;
        f[3] = mdot;
    } else if (DYN == kDynPolar) {
        // thrust off: s = c = 0; drag of the simulated system (Example 2 of
        // §4) with the printed components -C v_rho^2 and -C v_theta^2
        f[0] = y[1];
        f[1] = y[2] * y[2] / y[0] - mu / (y[0] * y[0]) + accel * s - drag * y[1] * y[1];
        f[2] = -y[1] * y[2] / y[0] + accel * c - drag * y[2] * y[2];
        f[3] = y[2] / y[0];
    } else {
        f[0] = fabs(c) < 1e-12 ? 0.0 : c;
        f[1] = fabs(s) < 1e-12 ? 0.0 : s;
        f[2] = 0.0;
        f[3] = 0.0;
    }
}

template <typename G, typename S>
__device__ __forceinline__ bool better(G a, int ka, G b, int kb)
{
    return a < b || (a == b && ka < kb);
}

template <typename G, typename S, bool REDUCED, int DYN>
__global__ void __launch_bounds__(128)
loop_kernel(const __grid_constant__ Geo<G> g, const __grid_constant__ LoopLaunch<G, S> a)
{
    __shared__ int s_code[kMaxAngles + 1];
    __shared__ typename V2<G>::type s_sc[kMaxAngles];
    build_table(g, s_code, s_sc);
    __syncthreads();
    const Table<G> T{s_code, s_sc, g.K, g.off};

    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= a.n) return;

    double y[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) y[d] = a.x0[4 * w + d];

    CachedEval<G, S, REDUCED, DYN> ev;
    ev.g = &g;
    ev.V = a.V;
    ev.sp.dt = (G)a.tau;
    ev.sp.hdt = (G)(0.5 * a.tau);
    ev.sp.um = (G)(a.tau * a.mdot / (double)g.h[3]);

    const long long steps = a.steps > 0 ? a.steps : 1;
    double t_arr = -1.0;
    for (long long step = 0; step < steps; ++step) {
        // --- feedback at y (Eq. (15)) ---
        G x[4];
        double yw[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            yw[d] = y[d];
            if (DYN == kDynPolar && d == 3) {
                // the orbital angle keeps growing along a trajectory: wrap it
                const double per = (double)g.h[3] * g.n[3], lo3 = (double)g.lo[3];
                yw[d] = lo3 + (y[d] - lo3) - per * floor((y[d] - lo3) / per);
            }
            x[d] = (G)yw[d];
            double sd = (yw[d] - (double)g.lo[d]) / (double)g.h[d];
            double fl = floor(sd);
            fl = fmin(fmax(fl, -4.0), (double)g.n[d] + 4.0);   // keep the index finite
            ev.i[d] = (int)fl;
            ev.u0[d] = (G)(sd - fl);
        }
        ev.nd = node_dyn<G, DYN>(g, ev.sp, x);
        // compensation reference: the plain interpolated value at angle 0
        ev.vj = (S)0;
        ev.reset();
        ev.vj = (S)ev.at_code(0);
        ev.reset();          // cached corners are differences to the old vj

        typedef typename CachedEval<G, S, REDUCED, DYN>::R R;
        R Db = ginf<R>();
        int kb = 0x7fffffff;
        for (int k = lane; k < g.K; k += 32) {
            R D = ev.at_sc(T.sc[k].x, T.sc[k].y);
            if (better<R, S>(D, k, Db, kb)) { Db = D; kb = k; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            R Do = __shfl_xor_sync(0xffffffffu, Db, o);
            int ko = __shfl_xor_sync(0xffffffffu, kb, o);
            if (better<R, S>(Do, ko, Db, kb)) { Db = Do; kb = ko; }
        }
        int code = T.code[kb] & (kCodes - 1);
        if (g.refine) code = fibonacci_refine(ev, T, g.fib_n0, g.fib_stop, kb, Db, Db);
        // running cost over tau (polar: Eq. (11); otherwise minimum time) and
        // the thrust-off control, which wins a tie
        double cost = a.tau, q = 0.0;
        if (DYN == kDynPolar) {
            const double lx = a.tau * state_cost_x(g, yw);
            cost = lx + a.tau * (g.thrust_cost / g.dt64);
            q = cost + a.beta_tau * ((double)ev.vj + (double)Db);
            if (g.off) {
                const double q_off = lx + a.beta_tau * ((double)ev.vj + (double)ev.at_sc((G)0, (G)0));
                if (q_off <= q) {
                    q = q_off;
                    code = kCodeOff;
                }
            }
        } else {
            q = cost + a.beta_tau * ((double)ev.vj + (double)Db);
        }
        const bool off = g.off && code == kCodeOff;

        double2 hi = a.tab_hi64[code >> 8], lo = a.tab_lo64[code & 255];
        double s = off ? 0.0 : hi.x * lo.y + hi.y * lo.x;
        double c = off ? 0.0 : hi.y * lo.y - hi.x * lo.x;

        if (a.steps == 0) {
            if (lane == 0) {
                a.alpha[w] = off ? CUDART_NAN : 6.283185307179586476925286766559 * (double)code / (double)kCodes;
                if (a.q) a.q[w] = q;
            }
            return;
        }

        // --- one RK4 step of the dynamics with the angle held ---
        double k1[4], k2[4], k3[4], k4[4], z[4];
        dyn64<DYN>(y, s, c, a.mu, a.accel, a.mdot, a.drag, k1);
#pragma unroll
        for (int d = 0; d < 4; ++d) z[d] = y[d] + 0.5 * a.h * k1[d];
        dyn64<DYN>(z, s, c, a.mu, a.accel, a.mdot, a.drag, k2);
#pragma unroll
        for (int d = 0; d < 4; ++d) z[d] = y[d] + 0.5 * a.h * k2[d];
        dyn64<DYN>(z, s, c, a.mu, a.accel, a.mdot, a.drag, k3);
#pragma unroll
        for (int d = 0; d < 4; ++d) z[d] = y[d] + a.h * k3[d];
        dyn64<DYN>(z, s, c, a.mu, a.accel, a.mdot, a.drag, k4);
#pragma unroll
        for (int d = 0; d < 4; ++d) y[d] = y[d] + a.h / 6.0 * (k1[d] + 2.0 * k2[d] + 2.0 * k3[d] + k4[d]);

        bool in = true;
#pragma unroll
        for (int d = 0; d < 4; ++d) in = in && (!(a.tgt_w[d] > 0.0) || fabs(y[d] - a.tgt_c[d]) < a.tgt_w[d]);
        if (in) { t_arr = (double)(step + 1) * a.h; break; }
    }
    if (lane == 0) {
        a.t_arrive[w] = t_arr;
#pragma unroll
        for (int d = 0; d < 4; ++d) a.x_final[4 * w + d] = y[d];
    }
}

template <typename G, typename S>
static cudaError_t launch_loop_t(const LoopLaunch<G, S>& L)
{
    int threads = 128;
    long long blocks = ((long long)L.n * 32 + threads - 1) / threads;
    if (blocks < 1) return cudaSuccess;
    if (L.dyn == kDynUnitSpeed) {
        if (L.reduced) return cudaErrorInvalidValue;
        loop_kernel<G, S, false, kDynUnitSpeed><<<(unsigned)blocks, threads, 0, L.stream>>>(L.g, L);
    } else if (L.dyn == kDynPolar) {
        if (L.reduced || !std::is_same<G, double>::value) return cudaErrorInvalidValue;
        loop_kernel<G, S, false, kDynPolar><<<(unsigned)blocks, threads, 0, L.stream>>>(L.g, L);
    } else if (L.reduced) {
        loop_kernel<G, S, true, kDynOrbit><<<(unsigned)blocks, threads, 0, L.stream>>>(L.g, L);
    } else {
        loop_kernel<G, S, false, kDynOrbit><<<(unsigned)blocks, threads, 0, L.stream>>>(L.g, L);
    }
    return cudaGetLastError();
}

cudaError_t launch_loop(const LoopLaunch<double, double>& L) { return launch_loop_t(L); }
cudaError_t launch_loop(const LoopLaunch<float, float>& L) { return launch_loop_t(L); }
cudaError_t launch_loop(const LoopLaunch<float, double>& L) { return launch_loop_t(L); }

}  // namespace dpk
