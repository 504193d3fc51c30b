// dp_host.h -- launch descriptors shared by the host driver and the kernel
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dp_device.cuh"

namespace dpk {

template <typename G, typename S>
struct SweepLaunch {
    Geo<G> g;
    const S* Vin;
    S* Vout;
    uint16_t* code;
    unsigned long long* feet_lo;   // frozen feet (FP32 geometry) or NULL
    unsigned* feet_hi;
    float* inc;                    // improvement: V_out - V_in (FP64-value polish) or NULL
    float* acc;                    // kIncr: running sum of increments
    double* V64;                   // kIncr: FP64 value that receives the sum
    int incr_flags;                // kIncr: 1 = first sweep of the chain, 2 = last
    Ctl* ctl;
    unsigned long long* ring;   // FP64 residual bits, one slot per sweep
    int ring_mask;
    long long sweep;            // sweep index within the solve (ring slot)
    int check_prev;             // 1: stop if the previous sweep's residual < tol
    double tol;
    Feet64 f64;                 // FP64 grids: frozen feet (written by improvements, read by kEvalFeet64*)
    int feet8 = 1;              // improvements with FP32 values: 1 stores 8-byte feet, 0 the word pair
    int mode;                   // kVI, kImproveFull, kImproveWalk, kEval
    int dyn;
    int reduced;
    cudaStream_t stream;
    int sm_count;
};

cudaError_t launch_sweep(const SweepLaunch<double, double>& L);
cudaError_t launch_sweep(const SweepLaunch<float, float>& L);
cudaError_t launch_sweep(const SweepLaunch<float, double>& L);

// Several evaluation sweeps of policy iteration in one launch (FP32 grids with
// frozen feet; dp_wave.cuh): levels 0 .. levels-1 run sweeps sweep ..
// sweep + levels - 1, level s reading V[(in0 + s) & 1] and writing
// V[(in0 + s + 1) & 1].
constexpr int kWaveBlock = 512;
constexpr int kWaveNodesPerThread = 4;
constexpr int kWaveChunk = kWaveBlock * kWaveNodesPerThread;   // nodes per work item
constexpr int kWaveMaxLevels = 32;
constexpr unsigned long long kWaveTimeoutNs = 2000000000ull;   // 2 s per wait

// Counters of one launch: [0] ticket, then levels x n_chunks completion counts.
__host__ __device__ constexpr long long wave_sync_ints(int levels, long long n_nodes)
{
    return 1 + (long long)levels * ((n_nodes + kWaveChunk - 1) / kWaveChunk);
}

struct WaveArgs {
    Geo<float> g;
    float* V[2];                           // the value buffers (kEval*) or increment buffers (kIncr*)
    int in0;                               // buffer that level 0 reads
    const uint16_t* code;
    const unsigned long long* feet_lo;
    const unsigned* feet_hi;
    float* acc;                            // kIncr*: running sum of increments
    double* V64;                           // kIncr*: FP64 value that receives the sum
    int e0, ne;                            // kIncr*: chain index of level 0, chain length
    int levels;
    int* sync;                             // wave_sync_ints(levels, n_nodes), zeroed
    Ctl* ctl;
    unsigned long long* ring;
    int ring_mask;
    long long sweep;                       // ring slot of level 0
    int check_prev;
    double tol;
    unsigned long long timeout_ns;         // limit of each wait (kWaveTimeoutNs unless a test sets it)
};

// mode: kEvalFeet, kEvalFeet8, kEvalFeetDiag, kIncr or kIncrDiag.  Zeroes a.sync first.
cudaError_t launch_wave(const WaveArgs& a, int mode, int dyn, int reduced, cudaStream_t st, int sm_count);

// Feedback (steps == 0) or closed loop (steps > 0) over n states.
template <typename G, typename S>
struct LoopLaunch {
    Geo<G> g;
    const S* V;
    const double* x0;        // n x 4 (device)
    int n;
    double tau, beta_tau;    // feedback step and its discount beta^(tau/dt)
    double h;                // RK4 step
    long long steps;
    double tgt_c[4], tgt_w[4];
    double mu, accel, mdot, lo_m;
    double drag;             // closed loop: drag coefficient C of the simulated system (polar)
    const double2* tab_hi64;
    const double2* tab_lo64;
    double* alpha;           // n (feedback)
    double* q;               // n (feedback)
    double* t_arrive;        // n (closed loop)
    double* x_final;         // n x 4 (closed loop)
    int dyn;
    int reduced;
    cudaStream_t stream;
};

cudaError_t launch_loop(const LoopLaunch<double, double>& L);
cudaError_t launch_loop(const LoopLaunch<float, float>& L);
cudaError_t launch_loop(const LoopLaunch<float, double>& L);

// Grid construction (node set, tables) and value conversions.
cudaError_t launch_trig_tables(double2* hi64, double2* lo64, float2* hi32, float2* lo32, cudaStream_t st);
cudaError_t launch_rows(int4* rows, int* err, int n0, int n1, int n2, int n3, const double* lo,
                        const double* h, double mu, int reduced, double e_lo, double e_hi,
                        cudaStream_t st);
cudaError_t launch_row_offsets(int4* rows, int n_rows, int n_m, long long* total, cudaStream_t st,
                               int* org = nullptr);
cudaError_t launch_lines(const int4* rows, unsigned* lines, int n0, int n1, int n2, int n_m,
                         cudaStream_t st);
cudaError_t launch_store_value(const double* src, void* dst, int fp32, int n, const Geo<double>& g, int* bad,
                               cudaStream_t st);
cudaError_t launch_store_value(const float* src, void* dst, int fp32, int n, const Geo<double>& g, int* bad,
                               cudaStream_t st);
cudaError_t launch_load_value(const void* src, double* dst, int fp32, int n, cudaStream_t st);
cudaError_t launch_load_value(const void* src, float* dst, int fp32, int n, cudaStream_t st);
cudaError_t launch_widen(const float* src, double* dst, int n, cudaStream_t st);
cudaError_t launch_box_index(const Geo<double>& g, long long* out, cudaStream_t st);
cudaError_t launch_prolong(const Geo<double>& gs, const void* Vs, int src_fp32, const uint16_t* Cs, int src_reduced,
                           int periodic, const Geo<double>& gd, void* Vd, int fp32_dst, uint16_t* Cd, double Md,
                           cudaStream_t st);

// Policy evaluation by restarted GMRES (§3: with the control frozen, Eq. (13)
// is the sparse linear system (I - beta W_f) V = b).  One cycle starts from
// the residual r0 = T_f(V) - V of the current value, builds an m-step Arnoldi
// basis of A = I - beta W_f (classical Gram-Schmidt, optionally twice), and
// adds the minimal-residual correction to V.  Basis vectors are stored
// unnormalised with their scales; the small Hessenberg problem lives on the
// device and is updated by the last block of each launch.
constexpr int kGmMaxRestart = 64;
constexpr int kGmLd = kGmMaxRestart + 2;     // columns of the per-block partial sums

struct GmCtl {
    double H[kGmMaxRestart + 1][kGmMaxRestart];   // Hessenberg, rotated in place
    double cs[kGmMaxRestart], sn[kGmMaxRestart];  // Givens rotations
    double gv[kGmMaxRestart + 1];                 // rotated right-hand side
    double scale[kGmMaxRestart + 1];              // 1 / ||Q_i|| of the stored vectors
    double coef[kGmMaxRestart + 1];               // coefficients of raw Q_i for the next update
    double beta0;                                 // ||r0||_2
    double rel;                                   // residual estimate / beta0
    int k;                                        // Arnoldi steps taken in this cycle
    int done;                                     // the cycle has its correction in coef
    unsigned counter;                             // blocks finished (last-block reductions)
    int pad;
};

template <typename G, typename VT>
struct GmArgs {
    Geo<G> g;                        // grid geometry with M = 0 (the linear part has no penalty)
    VT* Q;                           // (m + 1) vectors of ldq entries
    long long ldq;
    int m;                           // Arnoldi steps per cycle (1..kGmMaxRestart)
    int reorth;                      // 1: Gram-Schmidt twice
    double rtol;                     // a cycle ends once ||r|| <= rtol ||r0||
    const uint16_t* code;            // frozen policy
    const unsigned long long* feet_lo;   // frozen feet (FP32 geometry)
    const unsigned* feet_hi;         // nullptr: 8-byte feet (FP32-value phase)
    Feet64 f64;                      // FP64 frozen feet (FP64 grids; w == nullptr: recompute)
    double* partial;                 // max_blocks x kGmLd
    int max_blocks;
    GmCtl* gctl;
    Ctl* ctl;                        // the grid's control block (non-finite flag)
    int dyn;
    int reduced;
    int sm_count;
    cudaStream_t stream;
};

// One GMRES cycle: reads V_in and V_next = T_f(V_in), writes V_next = V_in + e.
cudaError_t gm_cycle(const GmArgs<float, float>& a, const float* Vin, float* Vnext);
cudaError_t gm_cycle(const GmArgs<float, float>& a, const double* Vin, double* Vnext);
cudaError_t gm_cycle(const GmArgs<double, double>& a, const double* Vin, double* Vnext);
// Residuals, in units of the FP32 -> FP64 switch tolerance, below which the
// FP32 phase of a polished solve (plain evaluation) stores word pairs instead
// of 8-byte feet, so that the FP64 phase starts from the evaluation fixed
// point of the 24-bit fractions.
constexpr double kFoot8Zone = 16.0;

// Frozen feet of the resident policy (FP32 geometry), as an improvement sweep
// stores them: the word pair, or the 8-byte word when feet_hi is nullptr.
cudaError_t launch_feet(const Geo<float>& g, const uint16_t* code, unsigned long long* feet_lo, unsigned* feet_hi,
                        int dyn, int reduced, int sm_count, cudaStream_t st);

}  // namespace dpk
