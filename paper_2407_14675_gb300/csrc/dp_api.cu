// dp_api.cu -- host side of the C ABI declared in include/dp.h.
//
// A dp_grid owns every device buffer of one problem: the row and line tables
// of the node set, double-buffered V in the grid's storage precision (plus
// FP64 buffers once a polish starts), the 16-bit policy, the angle tables, a
// control block and a ring of FP64 residual slots (one per sweep).  Solvers
// enqueue Jacobi sweeps in chunks on the grid's stream; each sweep can check
// the previous sweep's residual on the device and turn the rest of the queue
// into no-ops, so the host only synchronises once per chunk.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "dp.h"
#include "dp_host.h"

using namespace dpk;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail(DP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kRing = 8192;        // residual slots (power of two)
constexpr int kMaxChunk = 2048;    // sweeps enqueued between host checks (< kRing / 2)
constexpr double kStallZone = 64.0; // "near the FP32 floor": below this multiple of the switch tolerance
constexpr int kStallFar = 30;       // improvements without gain that switch anywhere
constexpr int kMaxConfirms = 3;     // full-table confirmations of an FP32 -> FP64 switch
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kGmDefaultRestart = 30;
constexpr double kGmDefaultRtol = 1e-3;
constexpr int kGmMaxCycles = 64;

// The end of GmCtl that the host reads back after a cycle.
struct GmTail {
    double beta0, rel;
    int k, done;
};
static_assert(offsetof(GmCtl, rel) == offsetof(GmCtl, beta0) + 8 && offsetof(GmCtl, k) == offsetof(GmCtl, beta0) + 16 &&
                  offsetof(GmCtl, done) == offsetof(GmCtl, beta0) + 20,
              "GmTail mirrors the tail of GmCtl");

}  // namespace

struct dp_grid {
    dp_grid_desc d;
    int device = 0;
    cudaStream_t st = nullptr;
    int sm_count = 0;
    int fp32 = 0;
    long long n_box = 0, n_active = 0, n_target = 0;
    int n_rows = 0;
    double h[4] = {0, 0, 0, 0};
    double M = 0;
    int tlo[4], thi[4];

    int4* rows = nullptr;
    int* row_org = nullptr;
    unsigned* lines = nullptr;
    double2 *hi64 = nullptr, *lo64 = nullptr;
    float2 *hi32 = nullptr, *lo32 = nullptr;
    void* V[2] = {nullptr, nullptr};     // storage precision
    int cur = 0;
    double* V64[2] = {nullptr, nullptr}; // FP64 values after a polish (FP32 grids)
    int cur64 = 0;
    bool fp64_values = false;
    uint16_t* code = nullptr;
    unsigned long long* feet_lo = nullptr;  // frozen feet of the current policy (FP32 grids)
    unsigned* feet_hi = nullptr;
    bool feet_valid = false;
    bool feet8 = false;                     // they are 8-byte words (stored with FP32 values)
    bool store_feet8 = true;                // what the next FP32-value improvements store
    int foot_format = DP_FOOT_AUTO;         // dp_set_foot_format
    Feet64 f64;                             // frozen feet of FP64 grids
    bool feet64_valid = false;
    float* acc = nullptr;                   // FP64-value polish: running sum of increments
    int* wave_sync = nullptr;               // FP32 grids: counters of the multi-level evaluation
    Ctl* ctl = nullptr;
    unsigned long long* ring = nullptr;
    double* staging = nullptr;           // n_active doubles
    long long* scratch64 = nullptr;      // n_active int64 (index export)
    Ctl* h_ctl = nullptr;                // pinned
    unsigned long long* h_ring = nullptr;// pinned, kRing
    long long device_bytes = 0;
    // GMRES policy evaluation (allocated on first use)
    unsigned char* gm_Q = nullptr;       // (gm_m + 1) x gm_ldq basis values
    long long gm_ldq = 0;
    int gm_m = 0;
    int gm_es = 0;                       // bytes per basis value
    long long gm_bytes = 0;
    double* gm_partial = nullptr;        // gm_blocks x kGmLd
    int gm_blocks = 0;
    GmCtl* gm_ctl = nullptr;
    GmTail* h_gm = nullptr;              // pinned, one per cycle of a round

    Geo<double> g64;
    Geo<float> g32;
};

namespace {

template <typename T>
int dalloc(dp_grid* g, T** p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? DP_ENOMEM : DP_ECUDA, "cudaMalloc(%zu bytes): %s",
                    count * sizeof(T), cudaGetErrorString(e));
    }
    g->device_bytes += (long long)(count * sizeof(T));
    return DP_OK;
}

void free_grid(dp_grid* g)
{
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->st) cudaStreamSynchronize(g->st);
    void* ps[] = {g->rows, g->row_org, g->lines, g->hi64, g->lo64, g->hi32, g->lo32, g->V[0], g->V[1], g->V64[0],
                  g->V64[1], g->code, g->feet_lo, g->feet_hi, g->acc, g->ctl, g->ring, g->staging,
                  g->scratch64, g->gm_Q, g->gm_partial, g->gm_ctl, g->f64.w, g->f64.t, g->f64.c,
                  g->wave_sync};
    for (void* p : ps)
        if (p) cudaFree(p);
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    if (g->h_ring) cudaFreeHost(g->h_ring);
    if (g->h_gm) cudaFreeHost(g->h_gm);
    delete g;
}

int validate(const dp_grid_desc* d)
{
    if (!d) return fail(DP_EINVAL, "desc is NULL");
    long long box = 1;
    for (int k = 0; k < 4; ++k) {
        if (d->n[k] < 2 || d->n[k] > 1024) return fail(DP_EINVAL, "n[%d] = %d outside [2, 1024]", k, d->n[k]);
        if (!(d->lo[k] < d->hi[k]) || !std::isfinite(d->lo[k]) || !std::isfinite(d->hi[k]))
            return fail(DP_EINVAL, "box dimension %d needs finite lo < hi", k);
        box *= d->n[k];
    }
    if (box > 2147483647LL) return fail(DP_EINVAL, "box of %lld nodes exceeds 2^31 - 1", box);
    if (d->dynamics != DP_DYN_ORBIT && d->dynamics != DP_DYN_UNIT_SPEED && d->dynamics != DP_DYN_POLAR)
        return fail(DP_EINVAL, "unknown dynamics %d", d->dynamics);
    if (d->dynamics == DP_DYN_POLAR) {
        if (d->precision != DP_FP64) return fail(DP_EINVAL, "polar dynamics need DP_FP64");
        if (d->reduced) return fail(DP_EINVAL, "polar dynamics take full-box grids");
        if (!(d->mu > 0) || !(d->accel >= 0) || !(d->lo[0] > 0))
            return fail(DP_EINVAL, "polar dynamics need mu > 0, accel >= 0 and rho > 0 on the box");
        double r2 = d->lo[0] + d->dt * std::fmin(d->lo[1], 0.0);
        if (!(r2 > 0)) return fail(DP_EINVAL, "Heun predictor leaves rho > 0");
        const double period = (d->hi[3] - d->lo[3]) * d->n[3] / (double)(d->n[3] - 1);
        if (!(std::fabs(period - kTwoPi) <= 1e-9 * kTwoPi))
            return fail(DP_EINVAL, "the angle axis must cover 2 pi: hi[3] = lo[3] + 2 pi (n[3] - 1) / n[3]");
        if (!(d->cost_alpha >= 0) || !(d->cost_beta >= 0) || !(d->cost_gamma >= 0) || !(d->a_bar > 0) ||
            !(d->e_bar >= 0) || !std::isfinite(d->omega_bar))
            return fail(DP_EINVAL, "cost weights must be >= 0, a_bar > 0, e_bar >= 0");
    }
    if (!(d->dt > 0) || !std::isfinite(d->dt)) return fail(DP_EINVAL, "dt must be > 0");
    if (!(d->beta > 0 && d->beta < 1)) return fail(DP_EINVAL, "beta must lie in (0, 1)");
    if (d->n_angles < 2 || d->n_angles > kMaxAngles) return fail(DP_EINVAL, "n_angles must lie in [2, 1024]");
    if (d->refine && !(d->refine_tol > 0)) return fail(DP_EINVAL, "refine_tol must be > 0");
    if (d->precision != DP_FP64 && d->precision != DP_FP32) return fail(DP_EINVAL, "unknown precision");
    if (!std::isfinite(d->penalty_M)) return fail(DP_EINVAL, "penalty_M must be finite");
    if (d->dynamics == DP_DYN_ORBIT) {
        if (!(d->mu > 0) || !(d->accel >= 0) || !(d->exhaust_c > 0))
            return fail(DP_EINVAL, "orbit dynamics need mu > 0, accel >= 0, exhaust_c > 0");
        if (!(d->lo[0] > 0) || !(d->lo[3] > 0)) return fail(DP_EINVAL, "orbit box needs r > 0 and m > 0");
        double r2 = d->lo[0] + d->dt * std::fmin(d->lo[1], 0.0);
        double m2 = d->lo[3] - d->dt * d->accel / d->exhaust_c;
        if (!(r2 > 0) || !(m2 > 0)) return fail(DP_EINVAL, "Heun predictor leaves r > 0 or m > 0 on the box");
    }
    if (d->reduced) {
        if (d->dynamics != DP_DYN_ORBIT) return fail(DP_EINVAL, "the energy-band grid needs orbit dynamics");
        if (!(d->lo[2] > 0)) return fail(DP_EINVAL, "the energy-band grid needs v_t > 0 on the box");
        if (!(d->energy_lo <= d->energy_hi)) return fail(DP_EINVAL, "energy_lo > energy_hi");
    }
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(d->target_c[k]) || !std::isfinite(d->target_w[k]))
            return fail(DP_EINVAL, "target box must be finite");
    return DP_OK;
}

template <typename G>
void fill_geo(const dp_grid* gr, Geo<G>& g)
{
    const dp_grid_desc& d = gr->d;
    for (int k = 0; k < 4; ++k) {
        g.n[k] = d.n[k];
        g.lo[k] = (G)d.lo[k];
        g.h[k] = (G)gr->h[k];
        g.ih[k] = (G)(1.0 / gr->h[k]);
        g.tlo[k] = gr->tlo[k];
        g.thi[k] = gr->thi[k];
    }
    g.stride[3] = 1;
    g.stride[2] = d.n[3];
    g.stride[1] = d.n[2] * d.n[3];
    g.stride[0] = d.n[1] * d.n[2] * d.n[3];
    double mdot = d.dynamics == DP_DYN_ORBIT ? -d.accel / d.exhaust_c : 0.0;
    g.mu = (G)d.mu;
    g.accel = (G)d.accel;
    g.mdot = (G)mdot;
    g.dt = (G)d.dt;
    g.hdt = (G)(0.5 * d.dt);
    g.beta = (G)d.beta;
    g.M = (G)gr->M;
    g.beta_hi = (G)d.beta;
    g.beta_lo = (G)(d.beta - (double)g.beta_hi);
    g.dt64 = d.dt;
    g.beta64 = d.beta;
    g.M64 = gr->M;
    g.um = (G)(d.dt * mdot / gr->h[3]);
    {
        float um = (float)(d.dt * mdot / gr->h[3]);
        float fl = std::floor(um);
        g.foot_dm = (int)fl;
        g.foot_tm = um - fl;
    }
    g.dyn = d.dynamics;
    const bool polar = d.dynamics == DP_DYN_POLAR;
    g.off = polar && d.off_control;
    g.cost_b = polar ? d.cost_beta : 0.0;
    g.cost_g = polar ? d.cost_gamma : 0.0;
    g.a_bar = d.a_bar;
    g.ex_bar = d.e_bar * std::cos(d.omega_bar);
    g.ey_bar = d.e_bar * std::sin(d.omega_bar);
    g.thrust_cost = polar ? d.dt * d.cost_alpha * d.accel : 0.0;   // dt alpha |u| of a thrust control
    g.K = d.n_angles;
    g.refine = d.refine;
    double tc = d.refine ? std::floor(d.refine_tol / (kTwoPi / kCodes)) : 0.0;
    g.fib_stop = (int)std::fmin(tc, 1e9);
    // shortest bracket between tabulated neighbours, and its Fibonacci index
    const int K = d.n_angles;
    long long Lmin = 1LL << 40;
    for (int k = 0; k < K; ++k) {
        long long prev = k == 0 ? (((long long)(K - 1) * kCodes + K / 2) / K) - kCodes
                                : (((long long)(k - 1) * kCodes + K / 2) / K);
        long long next = ((long long)(k + 1) * kCodes + K / 2) / K;
        Lmin = std::min(Lmin, next - prev);
    }
    long long F1 = 1, F2 = 1;
    int n = 2;
    while (F2 < Lmin) { long long F3 = F1 + F2; F1 = F2; F2 = F3; ++n; }
    g.fib_n0 = n;
    g.n_m = d.n[3];
    g.magic_m = ((1ULL << 40) + (unsigned long long)d.n[3] - 1) / (unsigned long long)d.n[3];
    g.n_nodes = (int)gr->n_active;
    g.rows = gr->rows;
    g.row_org = gr->row_org;
    g.lines = gr->lines;
}

template <typename G, typename S>
SweepLaunch<G, S> sweep_launch(dp_grid* g, const Geo<G>& geo, const S* Vin, S* Vout, int mode, long long sweep,
                               int check_prev, double tol)
{
    SweepLaunch<G, S> L;
    L.g = geo;
    L.Vin = Vin;
    L.Vout = Vout;
    L.code = g->code;
    L.feet_lo = g->feet_lo;
    L.feet_hi = g->feet_hi;
    L.inc = nullptr;
    L.acc = nullptr;
    L.V64 = nullptr;
    L.incr_flags = 0;
    if constexpr (std::is_same<G, double>::value && std::is_same<S, double>::value) L.f64 = g->f64;
    L.ctl = g->ctl;
    L.ring = g->ring;
    L.ring_mask = kRing - 1;
    L.sweep = sweep;
    L.check_prev = check_prev;
    L.tol = tol;
    L.mode = mode;
    L.feet8 = g->store_feet8 ? 1 : 0;
    L.dyn = g->d.dynamics;
    L.reduced = g->d.reduced;
    L.stream = g->st;
    L.sm_count = g->sm_count;
    return L;
}

// Value storage of the grid for the sweep kernels.
enum Store { kStoreF64, kStoreF32, kStoreMix };

Store store_of(const dp_grid* g)
{
    if (!g->fp32) return kStoreF64;
    return g->fp64_values ? kStoreMix : kStoreF32;
}

// Enqueue sweep number `t` (relative to the solve start, buffers alternate
// from the current one).
// Internal sweep mode of a public DP_SWEEP_* mode for the grid's storage
// (the two numberings overlap: every public mode is mapped exactly once).
int internal_mode(const dp_grid* g, int mode)
{
    // with FP32 values the plain evaluation reads either foot format, the
    // diagonal-solved one only the word pairs (8-byte feet are recomputed)
    const bool feet = store_of(g) == kStoreF32 && g->feet_valid;
    const bool feet64 = store_of(g) == kStoreF64 && g->feet64_valid;
    switch (mode) {
    case DP_SWEEP_VI: return kVI;
    case DP_SWEEP_IMPROVE_FULL: return kImproveFull;
    case DP_SWEEP_IMPROVE_WALK: return kImproveWalk;
    case DP_SWEEP_EVAL: return feet ? (g->feet8 ? kEvalFeet8 : kEvalFeet) : (feet64 ? kEvalFeet64 : kEval);
    case DP_SWEEP_EVAL_DIAG: return (feet && !g->feet8) ? kEvalFeetDiag : (feet64 ? kEvalFeet64Diag : kEvalDiag);
    case DP_SWEEP_VI_DIAG: return kVIDiag;
    }
    return -1;
}

// Enqueue sweep number `t` of public mode `pmode` (relative to the solve
// start, buffers alternate from the current one).
cudaError_t enqueue_sweep(dp_grid* g, int pmode, long long t, int check_prev, double tol)
{
    int a = (int)(t & 1);
    // improvement sweeps of FP32 grids store the frozen feet of the new
    // policy; the evaluation sweeps after them read those instead of
    // recomputing
    if (pmode == DP_SWEEP_IMPROVE_FULL || pmode == DP_SWEEP_IMPROVE_WALK) {
        if (store_of(g) == kStoreF32) {
            g->feet_valid = g->feet_lo != nullptr;
            g->feet8 = g->store_feet8;
        }
        if (store_of(g) == kStoreF64) g->feet64_valid = g->f64.w != nullptr;
    }
    const int mode = internal_mode(g, pmode);
    switch (store_of(g)) {
    case kStoreF64: {
        const double* in = (const double*)g->V[(g->cur + a) & 1];
        double* out = (double*)g->V[(g->cur + a + 1) & 1];
        return launch_sweep(sweep_launch<double, double>(g, g->g64, in, out, mode, t, check_prev, tol));
    }
    case kStoreF32: {
        const float* in = (const float*)g->V[(g->cur + a) & 1];
        float* out = (float*)g->V[(g->cur + a + 1) & 1];
        return launch_sweep(sweep_launch<float, float>(g, g->g32, in, out, mode, t, check_prev, tol));
    }
    default: {
        const double* in = g->V64[(g->cur64 + a) & 1];
        double* out = g->V64[(g->cur64 + a + 1) & 1];
        return launch_sweep(sweep_launch<float, double>(g, g->g32, in, out, mode, t, check_prev, tol));
    }
    }
}

// FP64-value policy iteration (FP32 grids after the switch).  The improvement
// maps V64[c] to V64[c ^ 1] with FP64 values and writes the first increment
// (float) and the frozen feet; the n evaluation sweeps then run on increments
// d' = beta W d in FP32 (scratch = the grid's FP32 value buffers) and the
// last one adds their sum to V64[c ^ 1].  Same iterates as n FP64 evaluation
// sweeps, to FP32 rounding of the increments.
cudaError_t enqueue_polish_improve(dp_grid* g, int mode, int c, long long t, int check_prev, double tol)
{
    SweepLaunch<float, double> L =
        sweep_launch<float, double>(g, g->g32, g->V64[c], g->V64[c ^ 1], mode, t, check_prev, tol);
    L.inc = (float*)g->V[0];
    g->feet_valid = g->feet_lo != nullptr;
    g->feet8 = false;   // the FP64-value phase stores the 24-bit word pair
    return launch_sweep(L);
}

cudaError_t enqueue_increment(dp_grid* g, int c, int e, int n, long long t, int check_prev, double tol, bool diag)
{
    // the increments read the word pairs of the FP64-value improvement
    if (!g->feet_valid || g->feet8) return cudaErrorInvalidValue;
    SweepLaunch<float, float> L = sweep_launch<float, float>(g, g->g32, (const float*)g->V[e & 1],
                                                             (float*)g->V[(e + 1) & 1], diag ? kIncrDiag : kIncr, t,
                                                             check_prev, tol);
    L.acc = g->acc;
    L.V64 = g->V64[c];
    L.incr_flags = (e == 0 ? 1 : 0) | (e == n - 1 ? 2 : 0);
    return launch_sweep(L);
}

// Evaluation sweeps per launch in policy iteration (the multi-level
// evaluation of dp_wave.cuh) for an FP32 grid whose frozen feet are stored:
// opts->eval_levels, or automatic.  Automatic is one sweep per launch: the
// multi-level launch cuts DRAM traffic per sweep but, measured on 61^4 and the
// 121^4 band, takes longer per sweep than single sweeps (the evaluation is
// bound by gather latency, and the chunk hand-offs add waits).
int wave_levels(const dp_grid* g, const dp_solve_opts* o)
{
    (void)g;
    if (o->eval_levels > 0) return std::min(o->eval_levels, kWaveMaxLevels);
    return 1;
}

// Limit of each bounded wait of the multi-level evaluation (test hook).
unsigned long long g_wave_timeout_ns = kWaveTimeoutNs;

// Levels e0 .. e0 + k - 1 of the n evaluation sweeps after an improvement as
// one launch; t = sweep index of level 0.  FP32 values: plain or
// diagonal-solved evaluation at the frozen feet.  FP64 values (mix): the
// increment chain into V64[c].
cudaError_t enqueue_wave(dp_grid* g, bool mix, bool diag, int c, int e0, int n, int k, long long t, int check_prev,
                         double tol)
{
    // diagonal-solved and increment levels read the word pairs
    if (!g->feet_valid || (g->feet8 && (mix || diag))) return cudaErrorInvalidValue;
    WaveArgs a;
    a.g = g->g32;
    a.V[0] = (float*)g->V[0];
    a.V[1] = (float*)g->V[1];
    a.code = g->code;
    a.feet_lo = g->feet_lo;
    a.feet_hi = g->feet_hi;
    a.acc = mix ? g->acc : nullptr;
    a.V64 = mix ? g->V64[c] : nullptr;
    a.e0 = e0;
    a.ne = n;
    a.levels = k;
    a.sync = g->wave_sync;
    a.ctl = g->ctl;
    a.ring = g->ring;
    a.ring_mask = kRing - 1;
    a.sweep = t;
    a.check_prev = check_prev;
    a.tol = tol;
    a.timeout_ns = g_wave_timeout_ns;
    // buffers as enqueue_sweep / enqueue_increment alternate them
    a.in0 = mix ? (e0 & 1) : (int)((g->cur + t) & 1);
    const int mode = mix ? (diag ? kIncrDiag : kIncr) : (diag ? kEvalFeetDiag : (g->feet8 ? kEvalFeet8 : kEvalFeet));
    return launch_wave(a, mode, g->d.dynamics, g->d.reduced, g->st, g->sm_count);
}

void advance(dp_grid* g, long long done)
{
    if (store_of(g) == kStoreMix) g->cur64 = (int)((g->cur64 + done) & 1);
    else g->cur = (int)((g->cur + done) & 1);
}

double ring_value(const dp_grid* g, long long t)
{
    unsigned long long b = g->h_ring[t & (kRing - 1)];
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}

int reset_ctl(dp_grid* g)
{
    CK(cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), g->st));
    return DP_OK;
}

// Zero the ring slots of sweeps [t0, t0 + n).
int clear_ring(dp_grid* g, long long t0, long long n)
{
    long long a = t0 & (kRing - 1);
    long long first = n < kRing - a ? n : kRing - a;
    CK(cudaMemsetAsync(g->ring + a, 0, first * sizeof(unsigned long long), g->st));
    if (n > first) CK(cudaMemsetAsync(g->ring, 0, (n - first) * sizeof(unsigned long long), g->st));
    return DP_OK;
}

// Copy ring slots of sweeps [t0, t0 + n) and the control block to the host.
int fetch(dp_grid* g, long long t0, long long n)
{
    long long a = t0 & (kRing - 1);
    long long first = n < kRing - a ? n : kRing - a;
    CK(cudaMemcpyAsync(g->h_ring + a, g->ring + a, first * sizeof(unsigned long long), cudaMemcpyDeviceToHost, g->st));
    if (n > first)
        CK(cudaMemcpyAsync(g->h_ring, g->ring, (n - first) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    return DP_OK;
}

// Optional per-sweep CUDA-event timing.
struct SweepTimer {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    int used = 0;
    double ms[5] = {0, 0, 0, 0, 0};

    ~SweepTimer()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
    cudaError_t begin(int k)
    {
        if (!on) return cudaSuccess;
        if (used + 2 > (int)ev.size()) {
            for (int i = 0; i < 2; ++i) {
                cudaEvent_t e;
                cudaError_t r = cudaEventCreate(&e);
                if (r != cudaSuccess) return r;
                ev.push_back(e);
            }
            kind.resize(ev.size() / 2);
        }
        kind[used / 2] = k;
        return cudaEventRecord(ev[used], st);
    }
    cudaError_t end()
    {
        if (!on) return cudaSuccess;
        cudaError_t r = cudaEventRecord(ev[used + 1], st);
        used += 2;
        return r;
    }
    // after a stream synchronisation: accumulate and recycle
    cudaError_t collect()
    {
        if (!on) return cudaSuccess;
        for (int i = 0; i + 1 < used; i += 2) {
            float m = 0;
            cudaError_t r = cudaEventElapsedTime(&m, ev[i], ev[i + 1]);
            if (r != cudaSuccess) return r;
            ms[kind[i / 2]] += m;
        }
        used = 0;
        return cudaSuccess;
    }
};

enum { kTVI = 0, kTImp = 1, kTEval = 2, kTImp64 = 3, kTEval64 = 4 };

int finish_nonfinite(dp_grid* g)
{
    if (g->h_ctl->nonfinite) return fail(DP_ENONFINITE, "a sweep produced a non-finite value");
    return DP_OK;
}

long long updates_per_sweep(const dp_grid* g) { return g->n_active - g->n_target; }

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int ensure_fp64(dp_grid* g)
{
    int rc;
    if (!g->V64[0] && (rc = dalloc(g, &g->V64[0], g->n_active))) return rc;
    if (!g->V64[1] && (rc = dalloc(g, &g->V64[1], g->n_active))) return rc;
    if (g->fp32 && !g->acc && (rc = dalloc(g, &g->acc, g->n_active))) return rc;
    return DP_OK;
}

// GMRES options with their defaults filled in.
struct GmOpts {
    int m, cycles, reorth;
    double rtol;
};

int gm_options(const dp_solve_opts* o, GmOpts& go)
{
    if (o->gmres_restart < 0 || o->gmres_restart > kGmMaxRestart)
        return fail(DP_EINVAL, "gmres_restart %d outside 0..%d", o->gmres_restart, kGmMaxRestart);
    if (o->gmres_cycles < 0 || o->gmres_cycles > kGmMaxCycles)
        return fail(DP_EINVAL, "gmres_cycles %d outside 0..%d", o->gmres_cycles, kGmMaxCycles);
    if (!(o->gmres_rtol >= 0) || !(o->gmres_rtol < 1)) return fail(DP_EINVAL, "gmres_rtol must be in [0, 1)");
    if (o->gmres_reorth != 0 && o->gmres_reorth != 1) return fail(DP_EINVAL, "gmres_reorth must be 0 or 1");
    go.m = o->gmres_restart > 0 ? o->gmres_restart : kGmDefaultRestart;
    go.cycles = o->gmres_cycles > 0 ? o->gmres_cycles : 1;
    go.reorth = o->gmres_reorth;
    go.rtol = o->gmres_rtol > 0 ? o->gmres_rtol : kGmDefaultRtol;
    return DP_OK;
}

// Basis of m + 1 vectors in the grid's storage precision (FP32 grids keep an
// FP32 basis after the switch to FP64 values), partial sums and control.
int ensure_gmres(dp_grid* g, int m)
{
    const int es = g->fp32 ? (int)sizeof(float) : (int)sizeof(double);
    const long long ldq = (g->n_active + 63) / 64 * 64;   // 256-byte aligned vectors
    if (g->gm_Q && (g->gm_m < m || g->gm_es != es)) {
        CK(cudaStreamSynchronize(g->st));
        cudaFree(g->gm_Q);
        g->device_bytes -= g->gm_bytes;
        g->gm_Q = nullptr;
    }
    int rc;
    if (!g->gm_Q) {
        if ((rc = dalloc(g, &g->gm_Q, (size_t)(m + 1) * ldq * es))) return rc;
        g->gm_m = m;
        g->gm_es = es;
        g->gm_ldq = ldq;
        g->gm_bytes = (long long)(m + 1) * ldq * es;
    }
    if (!g->gm_partial) {
        g->gm_blocks = 8 * g->sm_count;
        if ((rc = dalloc(g, &g->gm_partial, (size_t)g->gm_blocks * kGmLd))) return rc;
    }
    if (!g->gm_ctl) {
        if ((rc = dalloc(g, &g->gm_ctl, 1))) return rc;
        CK(cudaMemsetAsync(g->gm_ctl, 0, sizeof(GmCtl), g->st));   // the block counter starts at 0
    }
    if (!g->h_gm) CK(cudaMallocHost((void**)&g->h_gm, kGmMaxCycles * sizeof(GmTail)));
    return DP_OK;
}

template <typename G, typename VT>
GmArgs<G, VT> gm_args(const dp_grid* g, const Geo<G>& geo, const GmOpts& go)
{
    GmArgs<G, VT> a;
    a.g = geo;
    a.g.M = (G)0;           // the products carry no penalty: a foot outside blends to 0
    a.g.M64 = 0.0;
    a.Q = (VT*)g->gm_Q;
    a.ldq = g->gm_ldq;
    a.m = go.m;
    a.reorth = go.reorth;
    a.rtol = go.rtol;
    a.code = g->code;
    a.feet_lo = g->feet_lo;
    a.feet_hi = g->feet8 ? nullptr : g->feet_hi;   // nullptr: 8-byte feet
    if (g->feet64_valid) a.f64 = g->f64;
    a.partial = g->gm_partial;
    a.max_blocks = g->gm_blocks;
    a.gctl = g->gm_ctl;
    a.ctl = g->ctl;
    a.dyn = g->d.dynamics;
    a.reduced = g->d.reduced;
    a.sm_count = g->sm_count;
    a.stream = g->st;
    return a;
}

// One GMRES cycle on the current value: the previous buffer holds V, the
// current one T_f(V) (an improvement or evaluation sweep just ran); the
// current one receives V + e.  The cycle's tail is copied to h_gm[slot].
cudaError_t enqueue_gmres(dp_grid* g, const GmOpts& go, int slot)
{
    cudaError_t e;
    switch (store_of(g)) {
    case kStoreF64:
        e = gm_cycle(gm_args<double, double>(g, g->g64, go), (const double*)g->V[g->cur ^ 1], (double*)g->V[g->cur]);
        break;
    case kStoreF32:
        if (!g->feet_valid) return cudaErrorInvalidValue;
        e = gm_cycle(gm_args<float, float>(g, g->g32, go), (const float*)g->V[g->cur ^ 1], (float*)g->V[g->cur]);
        break;
    default:
        if (!g->feet_valid) return cudaErrorInvalidValue;
        e = gm_cycle(gm_args<float, float>(g, g->g32, go), (const double*)g->V64[g->cur64 ^ 1], g->V64[g->cur64]);
        break;
    }
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(&g->h_gm[slot], &g->gm_ctl->beta0, sizeof(GmTail), cudaMemcpyDeviceToHost, g->st);
}

// Launches of one cycle (some exit at once after an early stop).
long long gmres_launches(const GmOpts& go) { return 2 + (long long)go.m * (go.reorth ? 4 : 3); }

int zero_value(dp_grid* g)
{
    size_t es = g->fp32 ? sizeof(float) : sizeof(double);
    CK(cudaMemsetAsync(g->V[g->cur], 0, es * g->n_active, g->st));
    g->fp64_values = false;
    return DP_OK;
}

}  // namespace

namespace {

template <typename G, typename S>
int run_loop(dp_grid* g, const Geo<G>& geo, const S* V, const double* x0, int n, double tau, double h,
                    long long steps, double drag, double* alpha, double* q, double* t_arrive, double* x_final)
{
    LoopLaunch<G, S> L;
    L.drag = drag;
    L.g = geo;
    L.V = V;
    L.x0 = x0;
    L.n = n;
    L.tau = tau;
    L.beta_tau = std::pow(g->d.beta, tau / g->d.dt);
    L.h = h;
    L.steps = steps;
    for (int k = 0; k < 4; ++k) {
        L.tgt_c[k] = g->d.target_c[k];
        L.tgt_w[k] = g->d.target_w[k];
    }
    L.mu = g->d.mu;
    L.accel = g->d.accel;
    L.mdot = g->d.dynamics == DP_DYN_ORBIT ? -g->d.accel / g->d.exhaust_c : 0.0;
    L.lo_m = g->d.lo[3];
    L.tab_hi64 = g->hi64;
    L.tab_lo64 = g->lo64;
    L.alpha = alpha;
    L.q = q;
    L.t_arrive = t_arrive;
    L.x_final = x_final;
    L.dyn = g->d.dynamics;
    L.reduced = g->d.reduced;
    L.stream = g->st;
    CK(launch_loop(L));
    return DP_OK;
}

int loop_common(const dp_grid* cg, const double* states, int n, double tau, double h, double t_max, double drag,
                       double* alpha_out, double* q_out, double* t_arrive, double* x_final)
{
    dp_grid* g = const_cast<dp_grid*>(cg);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    for (long long k = 0; k < 4LL * n; ++k)
        if (!std::isfinite(states[k])) return fail(DP_ENONFINITE, "state %lld is not finite", k / 4);
    long long steps = 0;
    if (t_arrive) steps = (long long)std::ceil(t_max / h - 1e-9);
    if (t_arrive && steps < 1) steps = 1;
    double* d_buf = nullptr;
    size_t nb = (size_t)n * (4 + 1 + 1 + 4);
    CK(cudaMallocAsync(&d_buf, nb * sizeof(double), g->st));
    double* d_x0 = d_buf;
    double* d_a = d_buf + 4 * (size_t)n;
    double* d_q = d_a + n;
    double* d_xf = d_q + n;
    int rc = DP_OK;
    cudaError_t e = cudaMemcpyAsync(d_x0, states, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) {
        switch (store_of(g)) {
        case kStoreF64:
            rc = run_loop<double, double>(g, g->g64, (const double*)g->V[g->cur], d_x0, n, tau, h, steps, drag,
                                          d_a, d_q, d_a, d_xf);
            break;
        case kStoreF32:
            rc = run_loop<float, float>(g, g->g32, (const float*)g->V[g->cur], d_x0, n, tau, h, steps, drag, d_a,
                                        d_q, d_a, d_xf);
            break;
        default:
            rc = run_loop<float, double>(g, g->g32, g->V64[g->cur64], d_x0, n, tau, h, steps, drag, d_a, d_q, d_a,
                                         d_xf);
        }
        if (rc == DP_OK) {
            if (t_arrive) {
                e = cudaMemcpyAsync(t_arrive, d_a, sizeof(double) * n, cudaMemcpyDeviceToHost, g->st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(x_final, d_xf, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, g->st);
            } else {
                e = cudaMemcpyAsync(alpha_out, d_a, sizeof(double) * n, cudaMemcpyDeviceToHost, g->st);
                if (e == cudaSuccess && q_out)
                    e = cudaMemcpyAsync(q_out, d_q, sizeof(double) * n, cudaMemcpyDeviceToHost, g->st);
            }
        }
    }
    cudaError_t e2 = cudaFreeAsync(d_buf, g->st);
    cudaError_t e3 = cudaStreamSynchronize(g->st);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(DP_ECUDA, "closed loop: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess || e3 != cudaSuccess)
        return fail(DP_ECUDA, "closed loop: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
    return DP_OK;
}

}  // namespace

namespace dpk {

// Records an error message for dp_last_error() and returns code (used by the
// allocation-free entry point in dp_noalloc.cu and the network in dp_mlp.cu).
int record_error(int code, const char* msg) { return fail(code, "%s", msg); }

// Resident state of a grid for the warm-start network (dp_mlp.cu).
struct GridView {
    Geo<double> g64;
    int fp32;
    const void* V;
    double* V64;
    uint16_t* code;
    long long n;
    double M;
    double lo[4], hi[4];
    cudaStream_t st;
    const double2* tab_hi64;
    const double2* tab_lo64;
};

int grid_view(dp_grid* g, GridView* v)
{
    if (!g || !v) return fail(DP_EINVAL, "NULL argument");
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    v->g64 = g->g64;
    v->fp32 = g->fp32;
    v->V = g->V[g->cur];
    v->V64 = g->fp32 ? (g->fp64_values ? g->V64[g->cur64] : nullptr) : (double*)g->V[g->cur];
    v->code = g->code;
    v->n = g->n_active;
    v->M = g->M;
    for (int k = 0; k < 4; ++k) {
        v->lo[k] = g->d.lo[k];
        v->hi[k] = g->d.hi[k];
    }
    v->st = g->st;
    v->tab_hi64 = g->hi64;
    v->tab_lo64 = g->lo64;
    return DP_OK;
}

// After a warm start wrote V (storage precision) and the policy.
void grid_after_warm_start(dp_grid* g)
{
    g->fp64_values = false;
    g->feet_valid = false;
    g->feet64_valid = false;
}

// Validation and sweep geometry of a full-box grid described by desc, without
// building a grid: the same checks and target box as dp_grid_create, the
// same Geo fields as a grid's.  Table pointers are left NULL for the caller.
int describe_full_grid(const dp_grid_desc* desc, Geo<double>* g64, Geo<float>* g32, long long* n_nodes)
{
    int rc = validate(desc);
    if (rc) return rc;
    if (desc->reduced) return fail(DP_EINVAL, "this call takes full-box grids only (reduced = 0)");
    dp_grid g;
    g.d = *desc;
    g.M = desc->penalty_M > 0 ? desc->penalty_M : desc->dt / (1.0 - desc->beta);
    g.n_box = (long long)desc->n[0] * desc->n[1] * desc->n[2] * desc->n[3];
    g.n_active = g.n_box;
    for (int k = 0; k < 4; ++k) {
        g.h[k] = (desc->hi[k] - desc->lo[k]) / (double)(desc->n[k] - 1);
        int a = -1, b = -2;
        for (int i = 0; i < desc->n[k]; ++i) {
            volatile double x = desc->lo[k] + (double)i * g.h[k];
            bool in = !(desc->target_w[k] > 0) || std::fabs(x - desc->target_c[k]) < desc->target_w[k];
            if (in) {
                if (a < 0) a = i;
                b = i;
            }
        }
        if (a < 0) { a = 1; b = 0; }
        g.tlo[k] = a;
        g.thi[k] = b;
    }
    fill_geo(&g, *g64);
    fill_geo(&g, *g32);
    *n_nodes = g.n_box;
    return DP_OK;
}

}  // namespace dpk


namespace {

// FP32 -> FP64 switch rule of policy iteration, shared by both evaluation
// solvers: switch once the FP32 improvement residual is small, or stalls: 3
// improvements without gain near the FP32 floor, 30 far above it (a short
// stall there is the transient of a warm start, which FP64 values would not
// shorten).  A switch decided after a walk is first confirmed by a full-table
// FP32 improvement: walks that settled in local minima of the table are
// caught while sweeps are still cheap.
struct SwitchRule {
    double tol;
    double best = INFINITY;
    int stall = 0, confirms = 0;
    bool confirming = false;

    // Returns 1 to switch, 2 to run a confirming full tabulation next, 0 to go on.
    int step(double res, bool last_was_walk)
    {
        if (res < best * 0.999) { best = res; stall = 0; } else ++stall;
        bool want = res < tol || (stall >= 3 && res < kStallZone * tol) || stall >= kStallFar;
        if (confirming) {
            // the confirming full table moved V: stay in FP32, stall count anew
            confirming = false;
            if (!want) { best = res; stall = 0; }
        } else if (want && last_was_walk && confirms < kMaxConfirms) {
            ++confirms;
            confirming = true;
            return 2;
        }
        return want ? 1 : 0;
    }
};

int switch_to_fp64(dp_grid* g)
{
    int rc;
    if ((rc = ensure_fp64(g))) return rc;
    CK(launch_widen((const float*)g->V[g->cur], g->V64[g->cur64], (int)g->n_active, g->st));
    g->fp64_values = true;
    return reset_ctl(g);
}

// Policy iteration with GMRES evaluation (§3, Eq. (13)-(14) with the linear
// system of the evaluation step solved by GMRES).  Every improvement sweep is
// checked on the host before the evaluation is enqueued: the solve stops at
// the first improvement that moves V by less than tol (after a walk, a
// full-table improvement confirms it).
int pi_gmres(dp_grid* g, const dp_solve_opts* o, const GmOpts& go, dp_solve_stats& S, SweepTimer& T, double& res,
             bool& conv, long long& hist_n)
{
    int rc;
    SwitchRule rule;
    rule.tol = o->switch_tol > 0 ? o->switch_tol : 16.0 * 1.1920928955078125e-07 * g->M;
    bool first_full = !o->warm;
    int pending = 0;   // cycles whose tails wait for the next synchronisation
    auto collect = [&]() {
        for (int c = 0; c < pending; ++c) {
            S.gmres_cycles += 1;
            S.gmres_matvecs += g->h_gm[c].k;
        }
        pending = 0;
    };
    long long outer = 0;
    while (outer < o->max_sweeps) {
        const bool mix = store_of(g) == kStoreMix;
        const bool full = first_full || !o->walk;
        first_full = false;
        if ((rc = clear_ring(g, 0, 1))) return rc;
        CK(T.begin(mix ? kTImp64 : kTImp));
        const int mode = full ? DP_SWEEP_IMPROVE_FULL : DP_SWEEP_IMPROVE_WALK;
        if (mix) CK(enqueue_polish_improve(g, mode, g->cur64, 0, 0, o->tol));
        else CK(enqueue_sweep(g, mode, 0, 0, o->tol));
        CK(T.end());
        S.launches += 1;
        if ((rc = fetch(g, 0, 1))) return rc;
        CK(T.collect());
        collect();
        res = ring_value(g, 0);
        if (o->history && hist_n < o->history_capacity) o->history[hist_n] = res;
        ++hist_n;
        if (mix) ++S.sweeps_improve_fp64;
        else ++S.sweeps_improve;
        ++outer;
        advance(g, 1);
        if (g->h_ctl->nonfinite) break;
        if (res < o->tol) {
            if (!full) {
                first_full = true;   // a converged walk is confirmed by a full tabulation
                continue;
            }
            conv = true;
            break;
        }
        if (g->fp32 && !mix && o->polish) {
            const int act = rule.step(res, !full);
            if (act == 1) {
                if ((rc = switch_to_fp64(g))) return rc;
                S.switch_outer = outer;
                continue;            // the FP64 phase starts with an improvement
            }
            if (act == 2) first_full = true;
        }
        for (int c = 0; c < go.cycles; ++c) {
            CK(T.begin(mix ? kTEval64 : kTEval));
            if (c > 0) {
                // the residual of the corrected value needs its image T_f(V)
                CK(enqueue_sweep(g, DP_SWEEP_EVAL, 0, 0, o->tol));
                advance(g, 1);
                if (mix) ++S.sweeps_eval_fp64;
                else ++S.sweeps_eval;
                S.launches += 1;
            }
            CK(enqueue_gmres(g, go, pending));
            CK(T.end());
            ++pending;
            S.launches += gmres_launches(go);
        }
    }
    CK(cudaStreamSynchronize(g->st));
    CK(T.collect());
    collect();
    return DP_OK;
}

}  // namespace

extern "C" {

const char* dp_last_error(void) { return g_err; }

int dp_grid_create(const dp_grid_desc* desc, dp_grid** out)
{
    if (!out) return fail(DP_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(desc);
    if (rc) return rc;
    dp_grid* g = new (std::nothrow) dp_grid();
    if (!g) return fail(DP_ENOMEM, "host allocation failed");
    g->d = *desc;
    const dp_grid_desc& d = g->d;
    g->st = (cudaStream_t)d.stream;
    g->fp32 = d.precision == DP_FP32;
    g->M = d.penalty_M > 0 ? d.penalty_M : d.dt / (1.0 - d.beta);
    g->n_box = (long long)d.n[0] * d.n[1] * d.n[2] * d.n[3];
    g->n_rows = d.n[0] * d.n[1];
    auto bail = [&](int code) {
        free_grid(g);
        return code;
    };
    if (cudaGetDevice(&g->device) != cudaSuccess) return bail(fail(DP_ECUDA, "no CUDA device"));
    if (cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
        return bail(fail(DP_ECUDA, "cannot query the device"));

    // target index box (FP64, node coordinates lo + i h)
    for (int k = 0; k < 4; ++k) {
        g->h[k] = (d.hi[k] - d.lo[k]) / (double)(d.n[k] - 1);
        int a = -1, b = -2;
        for (int i = 0; i < d.n[k]; ++i) {
            volatile double x = d.lo[k] + (double)i * g->h[k];
            bool in = !(d.target_w[k] > 0) || std::fabs(x - d.target_c[k]) < d.target_w[k];
            if (in) {
                if (a < 0) a = i;
                b = i;
            }
        }
        if (a < 0) { a = 1; b = 0; }
        g->tlo[k] = a;
        g->thi[k] = b;
    }

    // node set
    if ((rc = dalloc(g, &g->rows, g->n_rows)) || (rc = dalloc(g, &g->row_org, g->n_rows))) return bail(rc);
    int* d_err = nullptr;
    long long* d_total = nullptr;
    if ((rc = dalloc(g, &d_err, 1))) return bail(rc);
    if ((rc = dalloc(g, &d_total, 1))) { cudaFree(d_err); return bail(rc); }
    auto tidy = [&]() {
        cudaFree(d_err);
        cudaFree(d_total);
        g->device_bytes -= sizeof(int) + sizeof(long long);
    };
    int h_err = 0;
    long long h_total = 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(int), g->st)) != cudaSuccess ||
        (e = launch_rows(g->rows, d_err, d.n[0], d.n[1], d.n[2], d.n[3], d.lo, g->h, d.mu, d.reduced, d.energy_lo,
                         d.energy_hi, g->st)) != cudaSuccess ||
        (e = launch_row_offsets(g->rows, g->n_rows, d.n[3], d_total, g->st, g->row_org)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, g->st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&h_total, d_total, sizeof(long long), cudaMemcpyDeviceToHost, g->st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(g->st)) != cudaSuccess) {
        tidy();
        return bail(fail(DP_ECUDA, "node-set construction: %s", cudaGetErrorString(e)));
    }
    tidy();
    if (h_err) return bail(fail(DP_EINVAL, "energy band is not one v_t interval per (r, v_r) row"));
    if (h_total <= 0) return bail(fail(DP_EINVAL, "empty node set"));
    if (h_total > 2147483647LL || (unsigned long long)h_total * (unsigned long long)(d.n[3] - 1) >= (1ULL << 40))
        return bail(fail(DP_EINVAL, "too many stored nodes"));
    g->n_active = h_total;

    // target count from the row table
    {
        std::vector<int4> rows(g->n_rows);
        if (cudaMemcpy(rows.data(), g->rows, sizeof(int4) * g->n_rows, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(fail(DP_ECUDA, "row table copy failed"));
        long long nt = 0;
        for (int ir = g->tlo[0]; ir <= g->thi[0]; ++ir)
            for (int iv = g->tlo[1]; iv <= g->thi[1]; ++iv) {
                const int4& R = rows[ir * d.n[1] + iv];
                int a = std::max(R.y, g->tlo[2]), b = std::min(R.y + R.z - 1, g->thi[2]);
                if (b >= a) nt += (long long)(b - a + 1) * (g->thi[3] - g->tlo[3] + 1);
            }
        g->n_target = nt;
    }

    long long n_lines = g->n_active / d.n[3];
    if ((rc = dalloc(g, &g->lines, n_lines))) return bail(rc);
    if ((e = launch_lines(g->rows, g->lines, d.n[0], d.n[1], d.n[2], d.n[3], g->st)) != cudaSuccess)
        return bail(fail(DP_ECUDA, "line table: %s", cudaGetErrorString(e)));

    if ((rc = dalloc(g, &g->hi64, 256)) || (rc = dalloc(g, &g->lo64, 256)) || (rc = dalloc(g, &g->hi32, 256)) ||
        (rc = dalloc(g, &g->lo32, 256)))
        return bail(rc);
    if ((e = launch_trig_tables(g->hi64, g->lo64, g->hi32, g->lo32, g->st)) != cudaSuccess)
        return bail(fail(DP_ECUDA, "angle tables: %s", cudaGetErrorString(e)));

    size_t es = g->fp32 ? sizeof(float) : sizeof(double);
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaMalloc(&g->V[b], es * g->n_active)) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(e == cudaErrorMemoryAllocation ? DP_ENOMEM : DP_ECUDA, "value buffer: %s",
                             cudaGetErrorString(e)));
        }
        g->device_bytes += (long long)(es * g->n_active);
        if (cudaMemsetAsync(g->V[b], 0, es * g->n_active, g->st) != cudaSuccess)
            return bail(fail(DP_ECUDA, "memset failed"));
    }
    if ((rc = dalloc(g, &g->code, g->n_active))) return bail(rc);
    if (g->fp32 && ((rc = dalloc(g, &g->feet_lo, g->n_active)) || (rc = dalloc(g, &g->feet_hi, g->n_active)) ||
                    (rc = dalloc(g, &g->wave_sync, wave_sync_ints(kWaveMaxLevels, g->n_active)))))
        return bail(rc);
    if (!g->fp32 && ((rc = dalloc(g, &g->f64.w, g->n_active)) || (rc = dalloc(g, &g->f64.t, 2 * g->n_active)) ||
                     (rc = dalloc(g, &g->f64.c, g->n_active))))
        return bail(rc);
    if ((rc = dalloc(g, &g->ctl, 1))) return bail(rc);
    if ((rc = dalloc(g, &g->ring, kRing))) return bail(rc);
    if (cudaMemsetAsync(g->code, 0, sizeof(uint16_t) * g->n_active, g->st) != cudaSuccess ||
        cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), g->st) != cudaSuccess)
        return bail(fail(DP_ECUDA, "memset failed"));
    if (cudaMallocHost(&g->h_ctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost(&g->h_ring, sizeof(unsigned long long) * kRing) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(DP_ENOMEM, "pinned host allocation failed"));
    }

    fill_geo(g, g->g64);
    fill_geo(g, g->g32);
    g->g64.tab_hi = g->hi64;
    g->g64.tab_lo = g->lo64;
    g->g32.tab_hi = g->hi32;
    g->g32.tab_lo = g->lo32;
    if ((e = cudaStreamSynchronize(g->st)) != cudaSuccess)
        return bail(fail(DP_ECUDA, "grid setup: %s", cudaGetErrorString(e)));
    *out = g;
    return DP_OK;
}

int dp_grid_destroy(dp_grid* grid)
{
    free_grid(grid);
    return DP_OK;
}

int dp_grid_get_info(const dp_grid* g, dp_grid_info* info)
{
    if (!g || !info) return fail(DP_EINVAL, "NULL argument");
    info->n_box = g->n_box;
    info->n_active = g->n_active;
    info->n_target = g->n_target;
    info->penalty_M = g->M;
    info->fp64_values = (g->fp32 && g->fp64_values) || !g->fp32;
    info->device_bytes = g->device_bytes;
    return DP_OK;
}

int dp_get_active_index(const dp_grid* cg, int64_t* box_index, int64_t count)
{
    dp_grid* g = const_cast<dp_grid*>(cg);
    if (!g || !box_index) return fail(DP_EINVAL, "NULL argument");
    if (count != g->n_active) return fail(DP_EINVAL, "count %lld != stored nodes %lld", (long long)count, g->n_active);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    if (!g->scratch64) {
        int rc = dalloc(g, &g->scratch64, g->n_active);
        if (rc) return rc;
    }
    CK(launch_box_index(g->g64, g->scratch64, g->st));
    CK(cudaMemcpyAsync(box_index, g->scratch64, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    return DP_OK;
}

static int ensure_staging(dp_grid* g)
{
    if (g->staging) return DP_OK;
    return dalloc(g, &g->staging, g->n_active);
}

int dp_set_value(dp_grid* g, const double* host_V, int64_t count)
{
    if (!g || !host_V) return fail(DP_EINVAL, "NULL argument");
    if (count != g->n_active) return fail(DP_EINVAL, "count %lld != stored nodes %lld", (long long)count, g->n_active);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    int rc = ensure_staging(g);
    if (rc) return rc;
    CK(cudaMemcpyAsync(g->staging, host_V, sizeof(double) * count, cudaMemcpyHostToDevice, g->st));
    CK(launch_store_value(g->staging, g->V[g->cur], g->fp32, (int)count, g->g64, &g->ctl->nonfinite, g->st));
    CK(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (g->h_ctl->nonfinite) return fail(DP_ENONFINITE, "V holds a non-finite value; the resident V is unchanged");
    g->fp64_values = false;
    return DP_OK;
}

int dp_get_value(const dp_grid* cg, double* host_V, int64_t count)
{
    dp_grid* g = const_cast<dp_grid*>(cg);
    if (!g || !host_V) return fail(DP_EINVAL, "NULL argument");
    if (count != g->n_active) return fail(DP_EINVAL, "count %lld != stored nodes %lld", (long long)count, g->n_active);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    if (!g->fp32 || g->fp64_values) {
        const double* src = g->fp32 ? g->V64[g->cur64] : (const double*)g->V[g->cur];
        CK(cudaMemcpyAsync(host_V, src, sizeof(double) * count, cudaMemcpyDeviceToHost, g->st));
    } else {
        int rc = ensure_staging(g);
        if (rc) return rc;
        CK(launch_load_value(g->V[g->cur], g->staging, 1, (int)count, g->st));
        CK(cudaMemcpyAsync(host_V, g->staging, sizeof(double) * count, cudaMemcpyDeviceToHost, g->st));
    }
    CK(cudaStreamSynchronize(g->st));
    return DP_OK;
}

int dp_set_value_f32(dp_grid* g, const float* host_V, int64_t count)
{
    if (!g || !host_V) return fail(DP_EINVAL, "NULL argument");
    if (count != g->n_active) return fail(DP_EINVAL, "count %lld != stored nodes %lld", (long long)count, g->n_active);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    int rc = ensure_staging(g);   // room for count doubles, so for count floats
    if (rc) return rc;
    float* staging = (float*)g->staging;
    CK(cudaMemcpyAsync(staging, host_V, sizeof(float) * count, cudaMemcpyHostToDevice, g->st));
    CK(launch_store_value(staging, g->V[g->cur], g->fp32, (int)count, g->g64, &g->ctl->nonfinite, g->st));
    CK(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (g->h_ctl->nonfinite) return fail(DP_ENONFINITE, "V holds a non-finite value; the resident V is unchanged");
    g->fp64_values = false;
    return DP_OK;
}

int dp_get_value_f32(const dp_grid* cg, float* host_V, int64_t count)
{
    dp_grid* g = const_cast<dp_grid*>(cg);
    if (!g || !host_V) return fail(DP_EINVAL, "NULL argument");
    if (count != g->n_active) return fail(DP_EINVAL, "count %lld != stored nodes %lld", (long long)count, g->n_active);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    if (g->fp32 && !g->fp64_values) {
        // the stored values themselves
        CK(cudaMemcpyAsync(host_V, g->V[g->cur], sizeof(float) * count, cudaMemcpyDeviceToHost, g->st));
    } else {
        int rc = ensure_staging(g);
        if (rc) return rc;
        const void* src = g->fp32 ? (const void*)g->V64[g->cur64] : (const void*)g->V[g->cur];
        CK(launch_load_value(src, (float*)g->staging, 0, (int)count, g->st));   // FP64 rounded to FP32
        CK(cudaMemcpyAsync(host_V, g->staging, sizeof(float) * count, cudaMemcpyDeviceToHost, g->st));
    }
    CK(cudaStreamSynchronize(g->st));
    return DP_OK;
}

int dp_set_policy(dp_grid* g, const uint16_t* host_codes, int64_t count)
{
    if (!g || !host_codes) return fail(DP_EINVAL, "NULL argument");
    if (count != g->n_active) return fail(DP_EINVAL, "count %lld != stored nodes %lld", (long long)count, g->n_active);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    CK(cudaMemcpyAsync(g->code, host_codes, sizeof(uint16_t) * count, cudaMemcpyHostToDevice, g->st));
    g->feet_valid = false;   // the stored feet belong to the previous policy
    g->feet64_valid = false;
    CK(cudaStreamSynchronize(g->st));
    return DP_OK;
}

int dp_get_policy(const dp_grid* g, uint16_t* host_codes, int64_t count)
{
    if (!g || !host_codes) return fail(DP_EINVAL, "NULL argument");
    if (count != g->n_active) return fail(DP_EINVAL, "count %lld != stored nodes %lld", (long long)count, g->n_active);
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    CK(cudaMemcpyAsync(host_codes, g->code, sizeof(uint16_t) * count, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    return DP_OK;
}

int dp_bellman_sweep(dp_grid* g, int32_t mode, double* residual)
{
    if (!g) return fail(DP_EINVAL, "grid is NULL");
    if (mode < DP_SWEEP_VI || mode > DP_SWEEP_VI_DIAG) return fail(DP_EINVAL, "unknown sweep mode %d", mode);
    if (mode == DP_SWEEP_VI_DIAG && g->d.dynamics == DP_DYN_POLAR)
        return fail(DP_EINVAL, "DP_SWEEP_VI_DIAG needs the minimum-time dynamics");
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    int rc;
    if ((rc = reset_ctl(g)) || (rc = clear_ring(g, 0, 1))) return rc;
    g->store_feet8 = g->foot_format != DP_FOOT_PAIR;
    CK(enqueue_sweep(g, mode, 0, 0, 0.0));
    if ((rc = fetch(g, 0, 1))) return rc;
    advance(g, 1);
    if (residual) *residual = ring_value(g, 0);
    return finish_nonfinite(g);
}

int dp_value_iterate(dp_grid* g, const dp_solve_opts* o, dp_solve_stats* stats)
{
    if (!g || !o) return fail(DP_EINVAL, "NULL argument");
    if (o->max_sweeps < 0 || !(o->tol >= 0)) return fail(DP_EINVAL, "bad tol or max_sweeps");
    if (o->eval_solver != DP_EVAL_JACOBI && o->eval_solver != DP_EVAL_DIAG)
        return fail(DP_EINVAL, "value iteration: eval_solver must be DP_EVAL_JACOBI or DP_EVAL_DIAG");
    if (o->eval_solver == DP_EVAL_DIAG && g->d.dynamics == DP_DYN_POLAR)
        return fail(DP_EINVAL, "the diagonal-solved value iteration needs the minimum-time dynamics");
    const int vi_mode = o->eval_solver == DP_EVAL_DIAG ? DP_SWEEP_VI_DIAG : DP_SWEEP_VI;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    double t0 = now_ms();
    dp_solve_stats S;
    memset(&S, 0, sizeof S);
    SweepTimer T;
    T.on = o->time_kernels != 0;
    T.st = g->st;
    int rc;
    if (!o->warm && (rc = zero_value(g))) return rc;
    if ((rc = reset_ctl(g))) return rc;
    const int tk = store_of(g) == kStoreMix ? kTImp64 : kTVI;
    long long s = 0, done = -1, chunk = 8;
    double res = INFINITY;
    while (s < o->max_sweeps) {
        long long c = std::min<long long>(chunk, o->max_sweeps - s);
        if ((rc = clear_ring(g, s, c))) return rc;
        for (long long k = 0; k < c; ++k) {
            CK(T.begin(tk));
            CK(enqueue_sweep(g, vi_mode, s + k, s + k > 0, o->tol));
            CK(T.end());
            S.launches++;
        }
        if ((rc = fetch(g, s, c))) return rc;
        CK(T.collect());
        if (g->h_ctl->stop) {
            done = g->h_ctl->stop_sweep;
            res = ring_value(g, done - 1);
            break;
        }
        res = ring_value(g, s + c - 1);
        s += c;
        if (g->h_ctl->nonfinite) { done = s; break; }
        if (res < o->tol) { done = s; break; }
        chunk = std::min<long long>(chunk * 2, kMaxChunk);
    }
    bool conv = done >= 0 && !g->h_ctl->nonfinite;
    if (done < 0) done = s;
    advance(g, done);
    S.sweeps_vi = done;
    S.residual = res;
    S.converged = conv;
    S.node_updates = done * updates_per_sweep(g);
    S.ms_vi = T.ms[kTVI] + T.ms[kTImp64];
    S.ms_wall = now_ms() - t0;
    if (stats) *stats = S;
    if ((rc = finish_nonfinite(g))) return rc;
    if (!conv) return fail(DP_ENOCONV, "no convergence within %lld sweeps (residual %g)", (long long)o->max_sweeps, res);
    return DP_OK;
}

// Evaluation sweeps per improvement once the values are FP64.  An FP64-value
// improvement costs about as much as 30 evaluation sweeps (its blends run on
// the FP64 pipe), and the FP64 phase starts near the fixed point, where the
// policy changes little: evaluating each policy further pays.  Measured on
// the 61^4 and 121^4 band grids: at least 80 diagonal-solved iterations
// (from 40) and at least 160 plain sweeps (from 20), which contract far less
// per sweep, beat the FP32 phase's counts by 4-10 % and 5-25 %.
constexpr int kFp64PhaseMinDiag = 80;
constexpr int kFp64PhaseMinSweeps = 160;

static int fp64_phase_evals(const dp_solve_opts* o)
{
    if (o->n_eval_fp64 > 0) return o->n_eval_fp64;
    const int lo = o->eval_solver == DP_EVAL_DIAG ? kFp64PhaseMinDiag : kFp64PhaseMinSweeps;
    return o->n_eval > 0 ? std::max(o->n_eval, lo) : 0;
}

int dp_policy_iterate(dp_grid* g, const dp_solve_opts* o, dp_solve_stats* stats)
{
    if (!g || !o) return fail(DP_EINVAL, "NULL argument");
    if (o->max_sweeps < 0 || o->n_eval < 0 || o->n_eval_fp64 < 0 || !(o->tol >= 0))
        return fail(DP_EINVAL, "bad options");
    if (o->eval_solver != DP_EVAL_JACOBI && o->eval_solver != DP_EVAL_GMRES && o->eval_solver != DP_EVAL_DIAG)
        return fail(DP_EINVAL, "unknown eval_solver %d", o->eval_solver);
    const bool diag = o->eval_solver == DP_EVAL_DIAG;
    // the feet its FP32-value improvements store: 8-byte words where the
    // plain evaluation (or GMRES) reads them, word pairs for the
    // diagonal-solved evaluation
    g->store_feet8 = g->foot_format == DP_FOOT_AUTO ? !diag : g->foot_format == DP_FOOT_WORD8;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    double t0 = now_ms();
    dp_solve_stats S;
    memset(&S, 0, sizeof S);
    SweepTimer T;
    T.on = o->time_kernels != 0;
    T.st = g->st;
    int rc;
    GmOpts go{};
    const bool gmres = o->eval_solver == DP_EVAL_GMRES;
    if (gmres && ((rc = gm_options(o, go)) || (rc = ensure_gmres(g, go.m)))) return rc;
    if (!o->warm && (rc = zero_value(g))) return rc;
    if ((rc = reset_ctl(g))) return rc;

    SwitchRule rule;
    rule.tol = o->switch_tol > 0 ? o->switch_tol : 16.0 * 1.1920928955078125e-07 * g->M;
    long long outer = 0, t = 0;    // outer iterations and sweeps of the current phase
    double res = INFINITY;
    bool conv = false, first_full = !o->warm;
    long long hist_n = 0;
    S.switch_outer = -1;
    if (gmres && (rc = pi_gmres(g, o, go, S, T, res, conv, hist_n))) return rc;
    auto record = [&](long long t0, long long n_imp, long long per) {
        for (long long q = 0; q < n_imp; ++q, ++hist_n)
            if (o->history && hist_n < o->history_capacity) o->history[hist_n] = ring_value(g, t0 + q * per);
    };
    while (!gmres && outer < o->max_sweeps) {
        const bool mix = store_of(g) == kStoreMix;
        // the FP32 phase of a polished solve stores the word pairs once its
        // residual nears the switch: the FP64 phase then starts from the
        // evaluation fixed point of the 24-bit fractions
        if (g->foot_format == DP_FOOT_AUTO && !diag && g->fp32 && !mix && o->polish)
            g->store_feet8 = !(res < kFoot8Zone * rule.tol);
        // evaluation sweeps per improvement in this phase, sweeps per outer iteration
        const int ne = mix ? fp64_phase_evals(o) : o->n_eval;
        const long long per = 1 + ne;
        const long long per_chunk = std::max<long long>(1, kMaxChunk / per / 4);
        long long n_out = std::min<long long>(per_chunk, o->max_sweeps - outer);
        if (g->fp32 && !mix && o->polish) n_out = 1;     // watch for the FP32 stall each step
        if ((rc = clear_ring(g, t, n_out * per))) return rc;
        int c64 = g->cur64;
        const bool first_full_chunk = first_full;
        bool confirm_next = false;
        for (long long q = 0; q < n_out; ++q) {
            long long ti = t + q * per;
            int mode = (first_full && q == 0) || !o->walk ? DP_SWEEP_IMPROVE_FULL : DP_SWEEP_IMPROVE_WALK;
            CK(T.begin(mix ? kTImp64 : kTImp));
            // without evaluation sweeps each improvement checks the previous one
            if (mix) CK(enqueue_polish_improve(g, mode, c64, ti, ne == 0 && ti > 0, o->tol));
            else CK(enqueue_sweep(g, mode, ti, ne == 0 && ti > 0, o->tol));
            CK(T.end());
            // the evaluation sweeps, `levels` per launch where the frozen feet
            // are stored (mix: the improvement stores them too)
            // (the multi-level diagonal-solved evaluation reads word pairs:
            // 8-byte feet are evaluated one sweep per launch, recomputed)
            const int levels =
                (mix || g->feet_valid) && g->fp32 && !(g->feet8 && diag && !mix) ? wave_levels(g, o) : 1;
            for (int e = 0; e < ne;) {
                const int k = std::min(levels, ne - e);
                CK(T.begin(mix ? kTEval64 : kTEval));
                if (k > 1) CK(enqueue_wave(g, mix, diag, c64 ^ 1, e, ne, k, ti + 1 + e, e == 0, o->tol));
                else if (mix) CK(enqueue_increment(g, c64 ^ 1, e, ne, ti + 1 + e, e == 0, o->tol, diag));
                else CK(enqueue_sweep(g, diag ? DP_SWEEP_EVAL_DIAG : DP_SWEEP_EVAL, ti + 1 + e, e == 0, o->tol));
                CK(T.end());
                e += k;
                S.launches += 1;
            }
            c64 ^= 1;
            S.launches += 1;
        }
        first_full = false;
        if ((rc = fetch(g, t, n_out * per))) return rc;
        CK(T.collect());
        long long ran = n_out * per;
        long long imp_done = n_out;
        if (g->h_ctl->stop) {
            // stop_sweep is the first evaluation sweep after the converged improvement
            ran = g->h_ctl->stop_sweep - t;
            imp_done = (ran + per - 1) / per;
            res = ring_value(g, g->h_ctl->stop_sweep - 1);
            conv = true;
        } else {
            res = ring_value(g, t + (n_out - 1) * per);
            // an evaluation sweep checks its improvement on the device; only a
            // chunk-final improvement without evaluations is checked here
            if (ne == 0 && res < o->tol) conv = true;
        }
        // The local walk stops at a local minimum of the tabulated angles, so a
        // converged walk is confirmed by one full-tabulation improvement: the
        // solve ends only when that sweep also moves V by less than tol.
        const bool last_was_walk = !(first_full_chunk && imp_done == 1) && o->walk;
        if (conv && last_was_walk) {
            conv = false;
            confirm_next = true;
        }
        record(t, imp_done, per);
        long long evals = ran - imp_done;
        if (mix) { S.sweeps_improve_fp64 += imp_done; S.sweeps_eval_fp64 += evals; }
        else { S.sweeps_improve += imp_done; S.sweeps_eval += evals; }
        outer += imp_done;
        if (mix) {
            // the FP64 value moves once per improvement; the increments alternate
            // the scratch buffers but always land in that value
            g->cur64 = (int)((g->cur64 + imp_done) & 1);
            t += ran;
        } else {
            t += ran;
        }
        if (g->h_ctl->nonfinite || g->h_ctl->wave_err) break;
        if (conv) break;
        if (confirm_next) {
            first_full = true;
            if ((rc = reset_ctl(g))) return rc;
            continue;
        }
        // FP32 -> FP64 switch (SwitchRule)
        if (g->fp32 && !mix && o->polish) {
            const int act = rule.step(res, last_was_walk);
            if (act == 2) first_full = true;
            if (act == 1) {
                advance(g, t);
                t = 0;
                if ((rc = switch_to_fp64(g))) return rc;
                S.switch_outer = outer;
            }
        }
    }
    if (store_of(g) != kStoreMix) advance(g, t);
    S.history_count = std::min<long long>(hist_n, o->history ? o->history_capacity : 0);
    S.residual = res;
    S.converged = conv && !g->h_ctl->nonfinite;
    S.node_updates = (S.sweeps_improve + S.sweeps_eval + S.sweeps_improve_fp64 + S.sweeps_eval_fp64 +
                      S.gmres_matvecs) * updates_per_sweep(g);
    S.ms_improve = T.ms[kTImp];
    S.ms_eval = T.ms[kTEval];
    S.ms_improve_fp64 = T.ms[kTImp64];
    S.ms_eval_fp64 = T.ms[kTEval64];
    S.ms_wall = now_ms() - t0;
    if (g->h_ctl->wave_err) S.converged = 0;
    if (stats) *stats = S;
    if (g->h_ctl->wave_err)
        return fail(DP_ETIMEOUT, "a multi-level evaluation launch gave up a bounded wait; the value is not valid");
    if ((rc = finish_nonfinite(g))) return rc;
    if (!S.converged)
        return fail(DP_ENOCONV, "no convergence within %lld improvement sweeps (residual %g)",
                    (long long)o->max_sweeps, res);
    return DP_OK;
}

int dp_set_foot_format(dp_grid* g, int32_t format)
{
    if (!g) return fail(DP_EINVAL, "grid is NULL");
    if (format != DP_FOOT_AUTO && format != DP_FOOT_WORD8 && format != DP_FOOT_PAIR)
        return fail(DP_EINVAL, "unknown foot format %d", format);
    g->foot_format = format;
    g->store_feet8 = format != DP_FOOT_PAIR;
    return DP_OK;
}

int dp_set_wave_wait_limit(int64_t ns)
{
    if (ns < -1) return fail(DP_EINVAL, "bad wait limit");
    g_wave_timeout_ns = ns >= 0 ? (unsigned long long)ns : kWaveTimeoutNs;
    return DP_OK;
}

int dp_policy_evaluate(dp_grid* g, const dp_solve_opts* o, dp_solve_stats* stats)
{
    if (!g || !o) return fail(DP_EINVAL, "NULL argument");
    if (o->max_sweeps < 0 || !(o->tol >= 0)) return fail(DP_EINVAL, "bad options");
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    const double t0 = now_ms();
    int rc;
    GmOpts go{};
    if ((rc = gm_options(o, go)) || (rc = ensure_gmres(g, go.m))) return rc;
    dp_solve_stats S;
    memset(&S, 0, sizeof S);
    S.switch_outer = -1;
    SweepTimer T;
    T.on = o->time_kernels != 0;
    T.st = g->st;
    if ((rc = reset_ctl(g))) return rc;
    const bool mix = store_of(g) == kStoreMix;
    if (g->fp32 && !g->feet_valid) {
        // 8-byte feet with FP32 values (the evaluation kernels read them too),
        // word pairs with FP64 values
        CK(launch_feet(g->g32, g->code, g->feet_lo, mix ? g->feet_hi : nullptr, g->d.dynamics, g->d.reduced,
                       g->sm_count, g->st));
        g->feet_valid = true;
        g->feet8 = !mix;
        S.launches += 1;
    }
    double res = INFINITY;
    bool conv = false;
    for (long long c = 0;; ++c) {
        // V <- T_f(V): its change is the stopping test, and the new pair
        // (V, T_f(V)) starts the next cycle
        if ((rc = clear_ring(g, 0, 1))) return rc;
        CK(T.begin(mix ? kTEval64 : kTEval));
        CK(enqueue_sweep(g, DP_SWEEP_EVAL, 0, 0, o->tol));
        CK(T.end());
        S.launches += 1;
        if ((rc = fetch(g, 0, 1))) return rc;
        if (c > 0) {
            S.gmres_cycles += 1;
            S.gmres_matvecs += g->h_gm[0].k;
        }
        advance(g, 1);
        if (mix) ++S.sweeps_eval_fp64;
        else ++S.sweeps_eval;
        res = ring_value(g, 0);
        if (g->h_ctl->nonfinite) break;
        if (res < o->tol) {
            conv = true;
            break;
        }
        if (c >= o->max_sweeps) break;
        CK(T.begin(mix ? kTEval64 : kTEval));
        CK(enqueue_gmres(g, go, 0));
        CK(T.end());
        S.launches += gmres_launches(go);
    }
    CK(T.collect());
    S.residual = res;
    S.converged = conv && !g->h_ctl->nonfinite;
    S.node_updates = (S.sweeps_eval + S.sweeps_eval_fp64 + S.gmres_matvecs) * updates_per_sweep(g);
    S.ms_eval = T.ms[kTEval];
    S.ms_eval_fp64 = T.ms[kTEval64];
    S.ms_wall = now_ms() - t0;
    if (stats) *stats = S;
    if ((rc = finish_nonfinite(g))) return rc;
    if (!S.converged)
        return fail(DP_ENOCONV, "policy evaluation: no convergence within %lld GMRES cycles (residual %g)",
                    (long long)o->max_sweeps, res);
    return DP_OK;
}

int dp_warm_start_from_grid(const dp_grid* src, dp_grid* dst, double* ms_out)
{
    if (!src || !dst) return fail(DP_EINVAL, "NULL argument");
    if (src == dst) return fail(DP_EINVAL, "source and destination must differ");
    if (src->d.dynamics != dst->d.dynamics) return fail(DP_EINVAL, "source and destination need the same dynamics");
    if (src->device != dst->device) return fail(DP_EINVAL, "source and destination must be on one device");
    if (cudaSetDevice(dst->device) != cudaSuccess) return fail(DP_ECUDA, "cudaSetDevice failed");
    // the source's work must be finished before the destination's stream reads it
    CK(cudaStreamSynchronize(src->st));
    const bool src64 = !src->fp32 || src->fp64_values;
    const void* Vs = (src->fp32 && src->fp64_values) ? (const void*)src->V64[src->cur64] : src->V[src->cur];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, dst->st));
    cudaError_t e = launch_prolong(src->g64, Vs, src64 ? 0 : 1, src->code, src->d.reduced,
                                   src->d.dynamics == DP_DYN_POLAR, dst->g64, dst->V[dst->cur], dst->fp32, dst->code,
                                   dst->M, dst->st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, dst->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(e);
    if (ms_out) *ms_out = ms;
    dst->fp64_values = false;
    dst->feet_valid = false;
    dst->feet64_valid = false;
    return DP_OK;
}

int dp_feedback_control(const dp_grid* g, const double* states, int32_t n, double tau, double* alpha_out,
                        double* q_out)
{
    if (!g || (n > 0 && (!states || !alpha_out))) return fail(DP_EINVAL, "NULL argument");
    if (n < 0 || !(tau > 0) || !std::isfinite(tau)) return fail(DP_EINVAL, "bad n or tau");
    if (n == 0) return DP_OK;
    return loop_common(g, states, n, tau, tau, 0.0, 0.0, alpha_out, q_out, nullptr, nullptr);
}

int dp_simulate_closed_loop(const dp_grid* g, const double* x0, int32_t n, double tau, double h_rk4, double t_max,
                            double* t_arrive, double* x_final)
{
    if (!g || (n > 0 && (!x0 || !t_arrive || !x_final))) return fail(DP_EINVAL, "NULL argument");
    if (n < 0 || !(tau > 0) || !(h_rk4 > 0) || !(t_max > 0) || !std::isfinite(t_max))
        return fail(DP_EINVAL, "bad n, tau, h_rk4 or t_max");
    if (n == 0) return DP_OK;
    return loop_common(g, x0, n, tau, h_rk4, t_max, 0.0, nullptr, nullptr, t_arrive, x_final);
}

int dp_simulate_closed_loop_drag(const dp_grid* g, const double* x0, int32_t n, double tau, double h_rk4,
                                 double t_max, double drag_c, double* t_arrive, double* x_final)
{
    if (!g || (n > 0 && (!x0 || !t_arrive || !x_final))) return fail(DP_EINVAL, "NULL argument");
    if (n < 0 || !(tau > 0) || !(h_rk4 > 0) || !(t_max > 0) || !std::isfinite(t_max))
        return fail(DP_EINVAL, "bad n, tau, h_rk4 or t_max");
    if (!(drag_c >= 0) || !std::isfinite(drag_c)) return fail(DP_EINVAL, "drag_c must be finite and >= 0");
    if (drag_c > 0 && g->d.dynamics != DP_DYN_POLAR) return fail(DP_EINVAL, "drag needs DP_DYN_POLAR grids");
    if (n == 0) return DP_OK;
    return loop_common(g, x0, n, tau, h_rk4, t_max, drag_c, nullptr, nullptr, t_arrive, x_final);
}

}  // extern "C"
