// dp_batch.cu -- many independent transfers solved together.
//
// Each transfer is a full-box FP32 grid of its own size, thrust, target and
// box (§3, Eq. (10)); they share nothing but the angle lattice.  Their values,
// policies and frozen feet sit back to back in one set of buffers (each
// transfer's slice starts on a 128-node boundary), and each sweep kind is ONE
// persistent launch over all transfers: a block walks a list of work items
// (a transfer and a run of `item` consecutive nodes), loads that transfer's
// geometry and angle table into shared memory when the transfer changes, and
// runs the same per-node code as a single grid's sweep.  Item sizes are
// picked by timing the candidates on the batch itself (dp_batch_autotune).
//
// Modified policy iteration (§3, Eq. (13)/(14), 1 improvement + n_eval
// evaluation sweeps per outer step) runs per transfer as a small state
// machine kept on the device: a one-block control kernel after the
// improvement reads each transfer's FP64 residual, decides convergence, the
// confirming full-table improvement after a converged local walk, and the
// switch from FP32 values to FP64 values (FP64 improvements + FP32
// increment sweeps) once FP32 stalls; a second one at the end of the step
// flips the transfer's buffers and rebuilds the work lists (a block scan
// over transfers), so finished transfers drop out of every later launch.
// The launches of a few outer steps are captured once in a CUDA graph and
// replayed; the host reads one counter per replay.  Every transfer goes
// through exactly the sweep sequence a single grid's dp_policy_iterate
// would run, with the same per-node arithmetic.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "dp.h"
#include "dp_host.h"
#include "dp_sweep.cuh"

namespace dpk {
int record_error(int code, const char* msg);
int describe_full_grid(const dp_grid_desc* desc, Geo<double>* g64, Geo<float>* g32, long long* n_nodes);
}  // namespace dpk

using namespace dpk;

namespace {

// work lists: widen, improvements by (values, full table or walk), evaluations
enum { kLWiden = 0, kLImp32Full = 1, kLImp32Walk = 2, kLImp64Full = 3, kLImp64Walk = 4, kLEval = 5, kLists = 6 };
enum { kPh32 = 0, kPh64 = 1, kPhDone = 2 };
enum {
    kStBegin = 0,      // start of a solve
    kStAfterImp = 1,   // after the improvement sweeps of an outer step
    kStEnd = 2,        // after its evaluation sweeps
    kStManImpFull = 3, // one stand-alone sweep (dp_batch_sweep) ...
    kStManImpWalk = 4,
    kStManEval = 5,
    kStManEnd = 6      // ... and its end
};
constexpr int kCtlThreads = 256;
constexpr long long kAlignNodes = 128;
constexpr int kChunksPerGraph = 4;
constexpr int kMaxBatch = 65536;
const int kItemCandidates[] = {512, 1024, 2048, 4096, 8192, 16384, 32768};

// Solver state of one transfer (device).
struct BState {
    unsigned long long res_bits;   // max |TV - V| of the current sweep (FP64 bits, atomicMax)
    double res, best;              // last improvement residual; best FP32-phase residual
    long long imp32, eval32, imp64, eval64;   // sweeps run
    long long switch_outer;        // improvements before the FP64 switch (-1: none)
    int phase;                     // kPh32, kPh64, kPhDone
    int full_next;                 // the next improvement enumerates the whole table
    int cur, cur64;                // current FP32 / FP64 value buffer
    int evals;                     // this step's evaluation sweeps run
    int finish;                    // the transfer ends with this step
    int switch_pending;            // switch to FP64 values after this step
    int widen;                     // the next step starts by widening V into FP64
    int stall, nonfinite, converged;
    int confirms;                  // full-table confirmations of the FP64 switch so far
    int confirming;                // this step's improvement confirms a switch
    int feet8;                     // FP32-value improvements store, and plain evaluations
                                   //   read, 8-byte feet (1) or word pairs (0)
};

struct BParams {
    double tol, switch_tol;
    long long max_outer;
    int n_eval, polish, walk, warm;
    int active;                    // transfers not finished (written by the control kernel)
    int feet8;                     // 1: plain evaluation (8-byte feet until the residual nears
                                   //   the switch, as dp_policy_iterate), 0: word pairs
};

struct BArgs {
    const Geo<float>* geo;
    const long long* off;          // first node of each transfer in the shared buffers
    BState* st;
    int* prefix;                   // kLists lists of count + 1 item offsets
    float* V32[2];                 // indexed by a runtime bit only through pick()
    double* V64[2];
    uint16_t* code;
    unsigned long long* feet_lo;
    unsigned* feet_hi;
    float* acc;
    int count;
    int item_eval, item_imp;       // nodes per work item
};

// One of two buffers by a runtime bit, without indexing the parameter array
// (a dynamic index would copy the arguments to local memory).
template <typename T>
__device__ __forceinline__ T* pick(T* const (&p)[2], int bit)
{
    return (bit & 1) ? p[1] : p[0];
}

__device__ __forceinline__ void load_geo(Geo<float>& dst, const Geo<float>* src)
{
    static_assert(sizeof(Geo<float>) % 4 == 0, "Geo size");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(Geo<float>) / 4); k += blockDim.x) d[k] = s[k];
}

// The transfer of work item `it` in list `pre`: pre[t] <= it < pre[t + 1].
__device__ __forceinline__ int item_transfer(const int* pre, int count, int it)
{
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&pre[mid]) <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

// FP32 values -> FP64 values at the switch.
__global__ void __launch_bounds__(kBlock) batch_widen_kernel(const BArgs a)
{
    const int* pre = a.prefix + kLWiden * (a.count + 1);
    const int total = pre[a.count];
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int t = item_transfer(pre, a.count, it);
        const int first = (it - pre[t]) * a.item_eval;
        const int end = min(first + a.item_eval, a.geo[t].n_nodes);
        const BState& S = a.st[t];
        const float* src = pick(a.V32, S.cur) + a.off[t];
        double* dst = pick(a.V64, S.cur64) + a.off[t];
        for (int j = first + threadIdx.x; j < end; j += kBlock) dst[j] = (double)src[j];
    }
}

// Improvement sweeps (§3, Eq. (14)): S = float for FP32 values, double for
// the FP64-value polish (which also writes the first increment); full table
// or walk as MODE (one kernel each, so each keeps its own register budget).
// The geometry sits in shared memory here, not in the parameter bank, so the
// compiler holds more of it in registers: the bound keeps 3 blocks per SM for
// the FP32 kernels (80 registers, no spills) and 2 for the FP64-value ones.
template <typename S, int DYN, int MODE>
__global__ void __launch_bounds__(kBlock, std::is_same<S, double>::value ? 2 : 3) batch_improve_kernel(const BArgs a)
{
    constexpr bool k64 = std::is_same<S, double>::value;
    __shared__ Geo<float> s_g;
    __shared__ int s_code[kMaxAngles + 1];
    __shared__ float2 s_sc[kMaxAngles];
    const int list = k64 ? (MODE == kImproveFull ? kLImp64Full : kLImp64Walk)
                         : (MODE == kImproveFull ? kLImp32Full : kLImp32Walk);
    const int* pre = a.prefix + list * (a.count + 1);
    const int total = pre[a.count];
    int cur_t = -1;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int t = item_transfer(pre, a.count, it);
        __syncthreads();   // the previous item is done with the shared state
        if (t != cur_t) {
            load_geo(s_g, &a.geo[t]);
            __syncthreads();
            build_table(s_g, s_code, s_sc);
            __syncthreads();
            cur_t = t;
        }
        BState& st = a.st[t];
        const long long o = a.off[t];
        const int first = (it - pre[t]) * a.item_imp;
        const int end = min(first + a.item_imp, s_g.n_nodes);
        const Table<float> T{s_code, s_sc, s_g.K};
        S resid = (S)0;
        bool bad = false;
        const S* Vin;
        S* Vout;
        float* inc = nullptr;
        if constexpr (k64) {
            Vin = pick(a.V64, st.cur64) + o;
            Vout = pick(a.V64, st.cur64 ^ 1) + o;
            inc = a.V32[0] + o;
        } else {
            Vin = pick(a.V32, st.cur) + o;
            Vout = pick(a.V32, st.cur ^ 1) + o;
        }
        sweep_nodes<float, S, MODE, false, DYN>(s_g, T, Vin, Vout, a.code + o, a.feet_lo + o, a.feet_hi + o, inc,
                                                nullptr, nullptr, 0, first + threadIdx.x, end, kBlock, resid, bad,
                                                Feet64(), nullptr, st.feet8 != 0);
        block_fold(resid, bad, &st.res_bits, &st.nonfinite);
    }
}

// Evaluation sweep e of an outer step (§3, Eq. (13)) at the frozen policy:
// FP32 transfers blend at their frozen feet (FEET) or recompute them; FP64
// transfers sweep increments.  e = -1 is a stand-alone sweep of V[cur].
// DIAG: each node's own coefficient solved (the Jacobi method proper).
// Evaluation and increment sweeps of a batch run 640-thread blocks (2 per SM
// at up to 51 registers, the resident warps of 5 blocks of 256): a block's
// iteration then covers more neighbouring corner lines of its work item.
constexpr int kBatchEvalBlock = 640;

template <int DYN, bool FEET, bool DIAG>
__global__ void __launch_bounds__(kBatchEvalBlock, 2) batch_eval_kernel(const BArgs a, int e, int n_eval)
{
    __shared__ Geo<float> s_g;
    const int* pre = a.prefix + kLEval * (a.count + 1);
    const int total = pre[a.count];
    const Table<float> T{nullptr, nullptr, 0};
    int cur_t = -1;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int t = item_transfer(pre, a.count, it);
        __syncthreads();
        if (t != cur_t) {
            load_geo(s_g, &a.geo[t]);
            __syncthreads();
            cur_t = t;
        }
        BState& st = a.st[t];
        const long long o = a.off[t];
        const int first = (it - pre[t]) * a.item_eval;
        const int end = min(first + a.item_eval, s_g.n_nodes);
        float resid = 0.0f;
        bool bad = false;
        if (st.phase == kPh32 || !FEET) {
            const float* Vin = pick(a.V32, st.cur + 1 + e) + o;
            float* Vout = pick(a.V32, st.cur + 2 + e) + o;
            if constexpr (FEET && DIAG)
                sweep_nodes<float, float, kEvalFeetDiag, false, DYN>(
                    s_g, T, Vin, Vout, a.code + o, a.feet_lo + o, a.feet_hi + o, nullptr, nullptr, nullptr, 0,
                    first + threadIdx.x, end, kBatchEvalBlock, resid, bad);
            else if constexpr (FEET)
                if (st.feet8)
                    sweep_nodes<float, float, kEvalFeet8, false, DYN>(
                        s_g, T, Vin, Vout, a.code + o, a.feet_lo + o, nullptr, nullptr, nullptr, nullptr, 0,
                        first + threadIdx.x, end, kBatchEvalBlock, resid, bad);
                else
                    sweep_nodes<float, float, kEvalFeet, false, DYN>(
                        s_g, T, Vin, Vout, a.code + o, a.feet_lo + o, a.feet_hi + o, nullptr, nullptr, nullptr, 0,
                        first + threadIdx.x, end, kBatchEvalBlock, resid, bad);
            else
                sweep_nodes<float, float, DIAG ? kEvalDiag : kEval, false, DYN>(
                    s_g, T, Vin, Vout, a.code + o, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                    first + threadIdx.x, end, kBatchEvalBlock, resid, bad);
        } else if constexpr (FEET) {
            const int flags = (e == 0 ? 1 : 0) | (e == n_eval - 1 ? 2 : 0);
            sweep_nodes<float, float, DIAG ? kIncrDiag : kIncr, false, DYN>(s_g, T, pick(a.V32, e) + o, pick(a.V32, e + 1) + o,
                                                         a.code + o, a.feet_lo + o, a.feet_hi + o, nullptr,
                                                         a.acc + o, pick(a.V64, st.cur64 ^ 1) + o, flags,
                                                         first + threadIdx.x, end, kBatchEvalBlock, resid, bad);
        }
        block_fold<float, kBatchEvalBlock>(resid, bad, &st.res_bits, &st.nonfinite);
    }
}

// One transfer's step of the solver state machine (the decisions a single
// grid's dp_policy_iterate takes on the host).
__device__ void ctl_update(BState& s, const BParams& p, double M, int stage)
{
    switch (stage) {
    case kStBegin:
        if (!p.warm) s.cur = 0;
        s.cur64 = 0;
        s.phase = kPh32;
        s.full_next = !p.warm || !p.walk;
        s.evals = s.finish = s.switch_pending = s.widen = 0;
        s.stall = s.nonfinite = s.converged = 0;
        s.confirms = s.confirming = 0;
        s.res = s.best = CUDART_INF;
        s.res_bits = 0;
        s.imp32 = s.eval32 = s.imp64 = s.eval64 = 0;
        s.switch_outer = -1;
        s.feet8 = p.feet8;
        break;
    case kStAfterImp: {
        if (s.phase == kPhDone) break;
        const double res = __longlong_as_double((long long)s.res_bits);
        s.res = res;
        if (s.phase == kPh32) ++s.imp32;
        else ++s.imp64;
        const bool full = s.full_next;
        s.widen = 0;
        s.evals = 0;
        if (s.nonfinite) {
            s.finish = 1;
        } else if (res < p.tol) {
            // the local walk stops at local minima of the table: a converged
            // walk is confirmed by one full-table improvement
            if (p.walk && !full) s.full_next = 1;
            else {
                s.finish = 1;
                s.converged = 1;
            }
        } else {
            s.evals = p.n_eval > 0;
            s.full_next = !p.walk;
            if (s.phase == kPh32 && p.polish) {
                // the switch rule of dp_policy_iterate
                const double sw = p.switch_tol > 0 ? p.switch_tol : 16.0 * 1.1920928955078125e-07 * M;
                if (res < s.best * 0.999) {
                    s.best = res;
                    s.stall = 0;
                } else {
                    ++s.stall;
                }
                bool want = res < sw || (s.stall >= 3 && res < 64.0 * sw) || s.stall >= 30;
                if (s.confirming) {
                    s.confirming = 0;
                    if (!want) {
                        s.best = res;
                        s.stall = 0;
                    }
                } else if (want && p.walk && !full && s.confirms < 3) {
                    ++s.confirms;            // confirm by a full table first
                    s.confirming = 1;
                    s.full_next = 1;
                    want = false;
                }
                if (want) s.switch_pending = 1;
            }
            if (s.imp32 + s.imp64 >= p.max_outer) s.finish = 1;
        }
        break;
    }
    case kStEnd: {
        if (s.phase == kPhDone) break;
        const int ev = s.evals ? p.n_eval : 0;
        if (s.phase == kPh32) {
            s.cur = (s.cur + 1 + ev) & 1;
            s.eval32 += ev;
        } else {
            s.cur64 ^= 1;
            s.eval64 += ev;
        }
        s.evals = 0;
        s.res_bits = 0;
        if (s.finish) {
            s.phase = kPhDone;
        } else if (s.switch_pending) {
            s.switch_pending = 0;
            s.widen = 1;
            s.phase = kPh64;
            s.switch_outer = s.imp32;
        } else if (s.phase == kPh32 && p.polish) {
            // the foot format of dp_policy_iterate's next step
            const double sw = p.switch_tol > 0 ? p.switch_tol : 16.0 * 1.1920928955078125e-07 * M;
            s.feet8 = p.feet8 && !(s.res < kFoot8Zone * sw);
        }
        break;
    }
    case kStManImpFull:
    case kStManImpWalk:
    case kStManEval:
        // a stand-alone improvement stores 8-byte feet; a stand-alone
        // evaluation reads the format stored last
        if (stage != kStManEval) s.feet8 = 1;
        s.phase = kPh32;
        s.full_next = stage == kStManImpFull;
        s.evals = stage == kStManEval;
        s.widen = 0;
        s.res_bits = 0;
        s.nonfinite = 0;
        break;
    case kStManEnd:
        s.res = __longlong_as_double((long long)s.res_bits);
        s.res_bits = 0;
        s.cur ^= 1;
        s.evals = 0;
        s.phase = kPhDone;
        break;
    }
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Updates every transfer's state for `stage`, then rebuilds the work lists
// (exclusive scans of items per transfer) and the count of live transfers.
__global__ void __launch_bounds__(kCtlThreads) batch_ctl_kernel(const BArgs a, BParams* p, int stage)
{
    constexpr int kW = kCtlThreads / 32;
    __shared__ int s_w[kLists + 1][kW];
    __shared__ int s_carry[kLists + 1];
    if (threadIdx.x <= kLists) s_carry[threadIdx.x] = 0;
    __syncthreads();
    const BParams P = *p;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < a.count; base += kCtlThreads) {
        const int t = base + threadIdx.x;
        int c[kLists + 1] = {0, 0, 0, 0, 0, 0, 0};
        if (t < a.count) {
            BState s = a.st[t];
            ctl_update(s, P, a.geo[t].M64, stage);
            a.st[t] = s;
            const int n = a.geo[t].n_nodes;
            const int ne = (n + a.item_eval - 1) / a.item_eval, ni = (n + a.item_imp - 1) / a.item_imp;
            c[kLWiden] = (s.phase == kPh64 && s.widen) ? ne : 0;
            c[kLImp32Full] = (s.phase == kPh32 && s.full_next) ? ni : 0;
            c[kLImp32Walk] = (s.phase == kPh32 && !s.full_next) ? ni : 0;
            c[kLImp64Full] = (s.phase == kPh64 && s.full_next) ? ni : 0;
            c[kLImp64Walk] = (s.phase == kPh64 && !s.full_next) ? ni : 0;
            c[kLEval] = (s.phase != kPhDone && s.evals) ? ne : 0;
            c[kLists] = s.phase != kPhDone;
        }
        int inc[kLists + 1];
#pragma unroll
        for (int k = 0; k <= kLists; ++k) {
            inc[k] = warp_incl_scan(c[k]);
            if (lane == 31) s_w[k][w] = inc[k];
        }
        __syncthreads();
        if (w == 0) {
#pragma unroll
            for (int k = 0; k <= kLists; ++k) {
                int v = lane < kW ? s_w[k][lane] : 0;
                v = warp_incl_scan(v);
                if (lane < kW) s_w[k][lane] = v;
            }
        }
        __syncthreads();
        if (t < a.count) {
#pragma unroll
            for (int k = 0; k < kLists; ++k)
                a.prefix[k * (a.count + 1) + t] = s_carry[k] + (w ? s_w[k][w - 1] : 0) + inc[k] - c[k];
        }
        __syncthreads();
        if (threadIdx.x <= kLists) s_carry[threadIdx.x] += s_w[threadIdx.x][kW - 1];
        __syncthreads();
    }
    if (threadIdx.x < kLists) a.prefix[threadIdx.x * (a.count + 1) + a.count] = s_carry[threadIdx.x];
    if (threadIdx.x == 0) p->active = s_carry[kLists];
}

__global__ void narrow_kernel(const double* src, float* dst, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = (float)src[j];
}

thread_local char g_berr[512];

int bfail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_berr, sizeof g_berr, fmt, ap);
    va_end(ap);
    return record_error(code, g_berr);
}

#define BCK(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return bfail(DP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

template <typename K>
int occupancy_blocks(K kern, int sm_count, int* out, int block = kBlock)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0) != cudaSuccess) return 1;
    *out = std::max(1, per_sm) * sm_count;
    return 0;
}

}  // namespace

struct dp_batch {
    int count = 0, device = 0, sm_count = 0, dyn = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<dp_grid_desc> d;
    std::vector<Geo<float>> g32;
    std::vector<Geo<double>> g64;
    std::vector<long long> off, nodes, targets;
    long long total = 0, max_nodes = 0;
    Geo<float>* d_geo = nullptr;
    long long* d_off = nullptr;
    BState* d_st = nullptr;
    BParams* d_par = nullptr;
    int* d_prefix = nullptr;
    float* V32[2] = {nullptr, nullptr};
    double* V64[2] = {nullptr, nullptr};
    uint16_t* code = nullptr;
    unsigned long long* feet_lo = nullptr;
    unsigned* feet_hi = nullptr;
    float* acc = nullptr;
    unsigned* lines = nullptr;
    double2 *hi64 = nullptr, *lo64 = nullptr;
    float2 *hi32 = nullptr, *lo32 = nullptr;
    double* staging = nullptr;
    int* d_bad = nullptr;
    BState* h_st = nullptr;        // pinned mirror of d_st
    BParams* h_par = nullptr;      // pinned
    int item_eval = 8192, item_imp = 8192;
    int blocks_widen = 0, blocks_imp32f = 0, blocks_imp32w = 0, blocks_imp64f = 0, blocks_imp64w = 0;
    int blocks_eval = 0, blocks_eval_nf = 0;
    cudaGraphExec_t exec = nullptr;
    int graph_n_eval = -1, graph_item_eval = 0, graph_item_imp = 0;
    bool graph_diag = false;
    long long graph_launches = 0;
    bool feet_valid = false;
    long long device_bytes = 0;
};

namespace {

void free_batch(dp_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    void* ps[] = {b->d_geo, b->d_off, b->d_st, b->d_par, b->d_prefix, b->V32[0], b->V32[1], b->V64[0], b->V64[1],
                  b->code, b->feet_lo, b->feet_hi, b->acc, b->lines, b->hi64, b->lo64, b->hi32, b->lo32,
                  b->staging, b->d_bad};
    for (void* p : ps)
        if (p) cudaFree(p);
    if (b->h_st) cudaFreeHost(b->h_st);
    if (b->h_par) cudaFreeHost(b->h_par);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

template <typename T>
int balloc(dp_batch* b, T** p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return bfail(e == cudaErrorMemoryAllocation ? DP_ENOMEM : DP_ECUDA, "cudaMalloc(%zu bytes): %s",
                     count * sizeof(T), cudaGetErrorString(e));
    }
    b->device_bytes += (long long)(count * sizeof(T));
    return DP_OK;
}

BArgs args_of(const dp_batch* b)
{
    BArgs a;
    a.geo = b->d_geo;
    a.off = b->d_off;
    a.st = b->d_st;
    a.prefix = b->d_prefix;
    a.V32[0] = b->V32[0];
    a.V32[1] = b->V32[1];
    a.V64[0] = b->V64[0];
    a.V64[1] = b->V64[1];
    a.code = b->code;
    a.feet_lo = b->feet_lo;
    a.feet_hi = b->feet_hi;
    a.acc = b->acc;
    a.count = b->count;
    a.item_eval = b->item_eval;
    a.item_imp = b->item_imp;
    return a;
}

cudaError_t launch_ctl(const dp_batch* b, int stage)
{
    batch_ctl_kernel<<<1, kCtlThreads, 0, b->st>>>(args_of(b), b->d_par, stage);
    return cudaGetLastError();
}

template <int DYN>
cudaError_t launch_improve(const dp_batch* b, bool fp64, bool full)
{
    const BArgs a = args_of(b);
    if (fp64 && full) batch_improve_kernel<double, DYN, kImproveFull><<<b->blocks_imp64f, kBlock, 0, b->st>>>(a);
    else if (fp64) batch_improve_kernel<double, DYN, kImproveWalk><<<b->blocks_imp64w, kBlock, 0, b->st>>>(a);
    else if (full) batch_improve_kernel<float, DYN, kImproveFull><<<b->blocks_imp32f, kBlock, 0, b->st>>>(a);
    else batch_improve_kernel<float, DYN, kImproveWalk><<<b->blocks_imp32w, kBlock, 0, b->st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_improve(const dp_batch* b, bool fp64, bool full)
{
    return b->dyn == DP_DYN_ORBIT ? launch_improve<kDynOrbit>(b, fp64, full)
                                  : launch_improve<kDynUnitSpeed>(b, fp64, full);
}

template <int DYN>
cudaError_t launch_eval(const dp_batch* b, int e, int n_eval, bool feet, bool diag)
{
    const BArgs a = args_of(b);
    if (feet && diag) batch_eval_kernel<DYN, true, true><<<b->blocks_eval, kBatchEvalBlock, 0, b->st>>>(a, e, n_eval);
    else if (feet) batch_eval_kernel<DYN, true, false><<<b->blocks_eval, kBatchEvalBlock, 0, b->st>>>(a, e, n_eval);
    else if (diag) batch_eval_kernel<DYN, false, true><<<b->blocks_eval_nf, kBatchEvalBlock, 0, b->st>>>(a, e, n_eval);
    else batch_eval_kernel<DYN, false, false><<<b->blocks_eval_nf, kBatchEvalBlock, 0, b->st>>>(a, e, n_eval);
    return cudaGetLastError();
}

cudaError_t launch_eval(const dp_batch* b, int e, int n_eval, bool feet, bool diag = false)
{
    return b->dyn == DP_DYN_ORBIT ? launch_eval<kDynOrbit>(b, e, n_eval, feet, diag)
                                  : launch_eval<kDynUnitSpeed>(b, e, n_eval, feet, diag);
}

cudaError_t launch_widen(const dp_batch* b)
{
    batch_widen_kernel<<<b->blocks_widen, kBlock, 0, b->st>>>(args_of(b));
    return cudaGetLastError();
}

// One outer step of every live transfer: widen, improvements, decisions,
// evaluation sweeps, end-of-step bookkeeping.
cudaError_t enqueue_step(const dp_batch* b, int n_eval, bool diag, long long* launches)
{
    cudaError_t e;
    if ((e = launch_widen(b)) != cudaSuccess) return e;
    for (int k = 0; k < 4; ++k)
        if ((e = launch_improve(b, k >= 2, (k & 1) == 0)) != cudaSuccess) return e;
    if ((e = launch_ctl(b, kStAfterImp)) != cudaSuccess) return e;
    for (int k = 0; k < n_eval; ++k)
        if ((e = launch_eval(b, k, n_eval, true, diag)) != cudaSuccess) return e;
    if ((e = launch_ctl(b, kStEnd)) != cudaSuccess) return e;
    *launches += 7 + n_eval;
    return cudaSuccess;
}

int ensure_graph(dp_batch* b, int n_eval, bool diag)
{
    if (b->exec && b->graph_n_eval == n_eval && b->graph_diag == diag && b->graph_item_eval == b->item_eval &&
        b->graph_item_imp == b->item_imp)
        return DP_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    long long launches = 0;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < kChunksPerGraph && e == cudaSuccess; ++c) e = enqueue_step(b, n_eval, diag, &launches);
    cudaError_t e2 = cudaStreamEndCapture(b->st, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return bfail(DP_ECUDA, "graph capture failed: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return bfail(DP_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    b->graph_n_eval = n_eval;
    b->graph_diag = diag;
    b->graph_item_eval = b->item_eval;
    b->graph_item_imp = b->item_imp;
    b->graph_launches = launches;
    return DP_OK;
}

int pull_state(dp_batch* b)
{
    BCK(cudaMemcpyAsync(b->h_st, b->d_st, sizeof(BState) * b->count, cudaMemcpyDeviceToHost, b->st));
    BCK(cudaStreamSynchronize(b->st));
    return DP_OK;
}

// Stand-alone FP32 values for every transfer (after a polished solve the
// result lives in the FP64 buffers).
int narrow_all(dp_batch* b)
{
    for (int t = 0; t < b->count; ++t) {
        const BState& s = b->h_st[t];
        if (s.switch_outer < 0) continue;
        const int n = (int)b->nodes[t];
        narrow_kernel<<<(n + 255) / 256, 256, 0, b->st>>>(b->V64[s.cur64] + b->off[t], b->V32[s.cur] + b->off[t], n);
        BCK(cudaGetLastError());
        b->h_st[t].switch_outer = -1;
    }
    BCK(cudaMemcpyAsync(b->d_st, b->h_st, sizeof(BState) * b->count, cudaMemcpyHostToDevice, b->st));
    return DP_OK;
}

int check_index(const dp_batch* b, int32_t index, int64_t count)
{
    if (!b) return bfail(DP_EINVAL, "NULL batch");
    if (index < 0 || index >= b->count) return bfail(DP_EINVAL, "transfer index %d outside [0, %d)", index, b->count);
    if ((long long)count != b->nodes[index])
        return bfail(DP_EINVAL, "count %lld != %lld nodes of transfer %d", (long long)count, b->nodes[index], index);
    return DP_OK;
}

int set_params(dp_batch* b, const dp_solve_opts* o, int warm)
{
    BParams& P = *b->h_par;
    memset(&P, 0, sizeof P);
    P.tol = o ? o->tol : 0.0;
    P.switch_tol = o ? o->switch_tol : 0.0;
    P.max_outer = o ? std::max<long long>(o->max_sweeps, 1) : 1;
    P.n_eval = o ? o->n_eval : 0;
    P.polish = o ? o->polish : 0;
    P.walk = o ? o->walk : 0;
    P.warm = warm;
    P.feet8 = o ? (o->eval_solver != DP_EVAL_DIAG) : 1;
    BCK(cudaMemcpyAsync(b->d_par, b->h_par, sizeof(BParams), cudaMemcpyHostToDevice, b->st));
    return DP_OK;
}

// One stand-alone sweep of every transfer: the control stage, the sweep
// kernel (timed with events when ms is non-NULL) and the end stage.
int manual_sweep(dp_batch* b, int32_t mode, double* ms)
{
    int stage = mode == DP_SWEEP_IMPROVE_FULL ? kStManImpFull : mode == DP_SWEEP_IMPROVE_WALK ? kStManImpWalk
                                                                                                : kStManEval;
    BCK(launch_ctl(b, stage));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        BCK(cudaEventCreate(&e0));
        BCK(cudaEventCreate(&e1));
        BCK(cudaEventRecord(e0, b->st));
    }
    cudaError_t e = stage == kStManEval ? launch_eval(b, -1, 0, b->feet_valid)
                                        : launch_improve(b, false, stage == kStManImpFull);
    if (ms) cudaEventRecord(e1, b->st);
    if (e == cudaSuccess) e = launch_ctl(b, kStManEnd);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (ms && e == cudaSuccess) {
        float f = 0.0f;
        e = cudaEventElapsedTime(&f, e0, e1);
        *ms = f;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    BCK(e);
    if (stage != kStManEval) b->feet_valid = true;
    return pull_state(b);
}

}  // namespace

extern "C" {

int dp_batch_create(const dp_grid_desc* descs, int32_t count, void* stream, dp_batch** out)
{
    if (!out) return bfail(DP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs) return bfail(DP_EINVAL, "descs is NULL");
    if (count < 1 || count > kMaxBatch) return bfail(DP_EINVAL, "count %d outside [1, %d]", count, kMaxBatch);
    dp_batch* b = new (std::nothrow) dp_batch();
    if (!b) return bfail(DP_ENOMEM, "host allocation failed");
    auto bail = [&](int rc) {
        free_batch(b);
        return rc;
    };
    b->count = count;
    b->d.assign(descs, descs + count);
    b->g32.resize(count);
    b->g64.resize(count);
    b->off.resize(count);
    b->nodes.resize(count);
    b->targets.resize(count);
    b->dyn = descs[0].dynamics;
    std::vector<long long> line_off(count);
    long long n_lines = 0;
    for (int t = 0; t < count; ++t) {
        const dp_grid_desc& d = descs[t];
        long long n = 0;
        int rc = describe_full_grid(&d, &b->g64[t], &b->g32[t], &n);
        if (rc) {
            char msg[600];
            snprintf(msg, sizeof msg, "transfer %d: %s", t, dp_last_error());
            return bail(bfail(rc, "%s", msg));
        }
        if (d.precision != DP_FP32) return bail(bfail(DP_EINVAL, "transfer %d: batches take FP32 grids", t));
        if (d.dynamics != b->dyn) return bail(bfail(DP_EINVAL, "transfer %d: every transfer needs the same dynamics", t));
        b->nodes[t] = n;
        b->off[t] = b->total;
        b->total += (n + kAlignNodes - 1) / kAlignNodes * kAlignNodes;
        b->max_nodes = std::max(b->max_nodes, n);
        line_off[t] = n_lines;
        n_lines += n / d.n[3];
        long long nt = 1;
        for (int k = 0; k < 4; ++k) nt *= std::max(0, b->g32[t].thi[k] - b->g32[t].tlo[k] + 1);
        b->targets[t] = nt;
    }
    if (b->total > (1LL << 40)) return bail(bfail(DP_EINVAL, "batch too large"));
    if (cudaGetDevice(&b->device) != cudaSuccess) return bail(bfail(DP_ECUDA, "no CUDA device"));
    if (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return bail(bfail(DP_ECUDA, "cannot query the device"));
    if (stream) {
        b->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(bfail(DP_ECUDA, "stream creation failed"));
        b->own_stream = true;
    }

    int rc;
    const size_t T = (size_t)b->total;
    if ((rc = balloc(b, &b->V32[0], T)) || (rc = balloc(b, &b->V32[1], T)) || (rc = balloc(b, &b->code, T)) ||
        (rc = balloc(b, &b->feet_lo, T)) || (rc = balloc(b, &b->feet_hi, T)) || (rc = balloc(b, &b->acc, T)) ||
        (rc = balloc(b, &b->V64[0], T)) || (rc = balloc(b, &b->V64[1], T)) ||
        (rc = balloc(b, &b->lines, (size_t)n_lines)) || (rc = balloc(b, &b->hi64, 256)) ||
        (rc = balloc(b, &b->lo64, 256)) || (rc = balloc(b, &b->hi32, 256)) || (rc = balloc(b, &b->lo32, 256)) ||
        (rc = balloc(b, &b->d_geo, count)) || (rc = balloc(b, &b->d_off, count)) ||
        (rc = balloc(b, &b->d_st, count)) || (rc = balloc(b, &b->d_par, 1)) ||
        (rc = balloc(b, &b->d_prefix, (size_t)kLists * (count + 1))) ||
        (rc = balloc(b, &b->staging, (size_t)b->max_nodes)) || (rc = balloc(b, &b->d_bad, 1)))
        return bail(rc);
    if (cudaMallocHost(&b->h_st, sizeof(BState) * count) != cudaSuccess ||
        cudaMallocHost(&b->h_par, sizeof(BParams)) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(DP_ENOMEM, "pinned host allocation failed"));
    }
    BCK(launch_trig_tables(b->hi64, b->lo64, b->hi32, b->lo32, b->st));

    // line tables of every transfer (full box: every (r, v_r) row holds all v_t)
    {
        long long max_rows = 0;
        for (int t = 0; t < count; ++t) max_rows = std::max<long long>(max_rows, (long long)descs[t].n[0] * descs[t].n[1]);
        int4* rows = nullptr;
        long long* d_total = nullptr;
        if (cudaMalloc(&rows, sizeof(int4) * max_rows) != cudaSuccess ||
            cudaMalloc(&d_total, sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            if (rows) cudaFree(rows);
            return bail(bfail(DP_ENOMEM, "row table allocation failed"));
        }
        cudaError_t e = cudaMemsetAsync(b->d_bad, 0, sizeof(int), b->st);
        for (int t = 0; t < count && e == cudaSuccess; ++t) {
            const dp_grid_desc& d = descs[t];
            double h[4];
            for (int k = 0; k < 4; ++k) h[k] = (d.hi[k] - d.lo[k]) / (double)(d.n[k] - 1);
            e = launch_rows(rows, b->d_bad, d.n[0], d.n[1], d.n[2], d.n[3], d.lo, h, d.mu, 0, 0.0, 0.0, b->st);
            if (e == cudaSuccess) e = launch_row_offsets(rows, d.n[0] * d.n[1], d.n[3], d_total, b->st);
            if (e == cudaSuccess)
                e = launch_lines(rows, b->lines + line_off[t], d.n[0], d.n[1], d.n[2], d.n[3], b->st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
        cudaFree(rows);
        cudaFree(d_total);
        if (e != cudaSuccess) return bail(bfail(DP_ECUDA, "line tables: %s", cudaGetErrorString(e)));
    }
    for (int t = 0; t < count; ++t) {
        b->g32[t].lines = b->lines + line_off[t];
        b->g32[t].rows = nullptr;
        b->g32[t].row_org = nullptr;
        b->g32[t].tab_hi = b->hi32;
        b->g32[t].tab_lo = b->lo32;
        b->g64[t].lines = b->lines + line_off[t];
        b->g64[t].rows = nullptr;
        b->g64[t].row_org = nullptr;
        b->g64[t].tab_hi = b->hi64;
        b->g64[t].tab_lo = b->lo64;
    }
    if (cudaMemcpyAsync(b->d_geo, b->g32.data(), sizeof(Geo<float>) * count, cudaMemcpyHostToDevice, b->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_off, b->off.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, b->st) !=
            cudaSuccess ||
        cudaMemsetAsync(b->V32[0], 0, sizeof(float) * T, b->st) != cudaSuccess ||
        cudaMemsetAsync(b->V32[1], 0, sizeof(float) * T, b->st) != cudaSuccess ||
        cudaMemsetAsync(b->code, 0, sizeof(uint16_t) * T, b->st) != cudaSuccess ||
        cudaMemsetAsync(b->d_st, 0, sizeof(BState) * count, b->st) != cudaSuccess)
        return bail(bfail(DP_ECUDA, "batch initialisation failed"));
    memset(b->h_st, 0, sizeof(BState) * count);
    for (int t = 0; t < count; ++t) b->h_st[t].switch_outer = -1;
    if (cudaMemcpyAsync(b->d_st, b->h_st, sizeof(BState) * count, cudaMemcpyHostToDevice, b->st) != cudaSuccess ||
        cudaStreamSynchronize(b->st) != cudaSuccess)
        return bail(bfail(DP_ECUDA, "batch initialisation failed"));

    bool bad = false;
    if (b->dyn == DP_DYN_ORBIT) {
        bad = occupancy_blocks(batch_improve_kernel<float, kDynOrbit, kImproveFull>, b->sm_count, &b->blocks_imp32f) ||
              occupancy_blocks(batch_improve_kernel<float, kDynOrbit, kImproveWalk>, b->sm_count, &b->blocks_imp32w) ||
              occupancy_blocks(batch_improve_kernel<double, kDynOrbit, kImproveFull>, b->sm_count, &b->blocks_imp64f) ||
              occupancy_blocks(batch_improve_kernel<double, kDynOrbit, kImproveWalk>, b->sm_count, &b->blocks_imp64w) ||
              occupancy_blocks(batch_eval_kernel<kDynOrbit, true, false>, b->sm_count, &b->blocks_eval, kBatchEvalBlock) ||
              occupancy_blocks(batch_eval_kernel<kDynOrbit, false, false>, b->sm_count, &b->blocks_eval_nf, kBatchEvalBlock);
    } else {
        bad = occupancy_blocks(batch_improve_kernel<float, kDynUnitSpeed, kImproveFull>, b->sm_count,
                               &b->blocks_imp32f) ||
              occupancy_blocks(batch_improve_kernel<float, kDynUnitSpeed, kImproveWalk>, b->sm_count,
                               &b->blocks_imp32w) ||
              occupancy_blocks(batch_improve_kernel<double, kDynUnitSpeed, kImproveFull>, b->sm_count,
                               &b->blocks_imp64f) ||
              occupancy_blocks(batch_improve_kernel<double, kDynUnitSpeed, kImproveWalk>, b->sm_count,
                               &b->blocks_imp64w) ||
              occupancy_blocks(batch_eval_kernel<kDynUnitSpeed, true, false>, b->sm_count, &b->blocks_eval, kBatchEvalBlock) ||
              occupancy_blocks(batch_eval_kernel<kDynUnitSpeed, false, false>, b->sm_count, &b->blocks_eval_nf, kBatchEvalBlock);
    }
    bad = bad || occupancy_blocks(batch_widen_kernel, b->sm_count, &b->blocks_widen);
    if (bad) return bail(bfail(DP_ECUDA, "occupancy query failed"));
    *out = b;
    return DP_OK;
}

int dp_batch_destroy(dp_batch* b)
{
    free_batch(b);
    return DP_OK;
}

int dp_batch_get_info(const dp_batch* b, int32_t* count, int64_t* nodes_total, int64_t* nodes_target,
                      int32_t* item_eval, int32_t* item_improve, int64_t* device_bytes)
{
    if (!b) return bfail(DP_EINVAL, "NULL batch");
    if (count) *count = b->count;
    if (nodes_total) {
        long long s = 0;
        for (long long n : b->nodes) s += n;
        *nodes_total = s;
    }
    if (nodes_target) {
        long long s = 0;
        for (long long n : b->targets) s += n;
        *nodes_target = s;
    }
    if (item_eval) *item_eval = b->item_eval;
    if (item_improve) *item_improve = b->item_imp;
    if (device_bytes) *device_bytes = b->device_bytes;
    return DP_OK;
}

int dp_batch_set_items(dp_batch* b, int32_t item_eval, int32_t item_improve)
{
    if (!b) return bfail(DP_EINVAL, "NULL batch");
    if (item_eval < kBlock || item_eval > (1 << 20) || item_eval % kBlock || item_improve < kBlock ||
        item_improve > (1 << 20) || item_improve % kBlock)
        return bfail(DP_EINVAL, "item sizes must be multiples of %d in [%d, 2^20]", kBlock, kBlock);
    b->item_eval = item_eval;
    b->item_imp = item_improve;
    return DP_OK;
}

int dp_batch_sweep(dp_batch* b, int32_t mode, double* residual, double* ms)
{
    if (!b) return bfail(DP_EINVAL, "NULL batch");
    if (mode != DP_SWEEP_IMPROVE_FULL && mode != DP_SWEEP_IMPROVE_WALK && mode != DP_SWEEP_EVAL)
        return bfail(DP_EINVAL, "mode must be DP_SWEEP_IMPROVE_FULL, DP_SWEEP_IMPROVE_WALK or DP_SWEEP_EVAL");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(DP_ECUDA, "cudaSetDevice failed");
    int rc;
    if ((rc = pull_state(b)) || (rc = narrow_all(b)) || (rc = set_params(b, nullptr, 1))) return rc;
    if ((rc = manual_sweep(b, mode, ms))) return rc;
    int nonfinite = 0;
    for (int t = 0; t < b->count; ++t) {
        if (residual) residual[t] = b->h_st[t].res;
        nonfinite |= b->h_st[t].nonfinite;
    }
    if (nonfinite) return bfail(DP_ENONFINITE, "a sweep produced a non-finite value");
    return DP_OK;
}

int dp_batch_autotune(dp_batch* b, int32_t* item_eval, int32_t* item_improve)
{
    if (!b) return bfail(DP_EINVAL, "NULL batch");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(DP_ECUDA, "cudaSetDevice failed");
    int rc;
    if ((rc = pull_state(b))) return rc;
    for (int t = 0; t < b->count; ++t) {
        b->h_st[t].cur = 0;
        b->h_st[t].switch_outer = -1;
    }
    BCK(cudaMemcpyAsync(b->d_st, b->h_st, sizeof(BState) * b->count, cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemsetAsync(b->V32[0], 0, sizeof(float) * b->total, b->st));
    if ((rc = set_params(b, nullptr, 1))) return rc;
    // a full improvement from V = 0 gives every node a policy and frozen foot
    if ((rc = manual_sweep(b, DP_SWEEP_IMPROVE_FULL, nullptr))) return rc;
    double best_e = INFINITY, best_i = INFINITY;
    int pick_e = b->item_eval, pick_i = b->item_imp;
    const int keep_e = b->item_eval, keep_i = b->item_imp;
    for (int cand : kItemCandidates) {
        b->item_eval = cand;
        b->item_imp = keep_i;
        double t_e = 0.0, t_i = 0.0, ms = 0.0;
        if ((rc = manual_sweep(b, DP_SWEEP_EVAL, nullptr))) return rc;   // warm-up
        for (int r = 0; r < 3; ++r) {
            if ((rc = manual_sweep(b, DP_SWEEP_EVAL, &ms))) return rc;
            t_e += ms;
        }
        b->item_eval = keep_e;
        b->item_imp = cand;
        for (int r = 0; r < 2; ++r) {
            if ((rc = manual_sweep(b, DP_SWEEP_IMPROVE_WALK, &ms))) return rc;
            t_i += ms;
        }
        if (t_e < best_e) { best_e = t_e; pick_e = cand; }
        if (t_i < best_i) { best_i = t_i; pick_i = cand; }
    }
    b->item_eval = pick_e;
    b->item_imp = pick_i;
    // back to the cold state: V = 0, policy code 0
    for (int t = 0; t < b->count; ++t) b->h_st[t].cur = 0;
    BCK(cudaMemcpyAsync(b->d_st, b->h_st, sizeof(BState) * b->count, cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemsetAsync(b->V32[0], 0, sizeof(float) * b->total, b->st));
    BCK(cudaMemsetAsync(b->code, 0, sizeof(uint16_t) * b->total, b->st));
    BCK(cudaStreamSynchronize(b->st));
    b->feet_valid = false;
    if (item_eval) *item_eval = pick_e;
    if (item_improve) *item_improve = pick_i;
    return DP_OK;
}

int dp_batch_policy_iterate(dp_batch* b, const dp_solve_opts* o, dp_solve_stats* total, dp_batch_stats* per)
{
    if (!b || !o) return bfail(DP_EINVAL, "NULL argument");
    if (o->max_sweeps < 1 || o->n_eval < 0 || o->n_eval > 1024 || !(o->tol >= 0))
        return bfail(DP_EINVAL, "bad options (max_sweeps >= 1, 0 <= n_eval <= 1024, tol >= 0)");
    if (o->eval_solver != DP_EVAL_JACOBI && o->eval_solver != DP_EVAL_DIAG)
        return bfail(DP_EINVAL, "batched policy iteration evaluates by plain or diagonal-solved sweeps only");
    const bool diag = o->eval_solver == DP_EVAL_DIAG;
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(DP_ECUDA, "cudaSetDevice failed");
    const double t0 = now_ms();
    int rc;
    if ((rc = pull_state(b))) return rc;
    if (o->warm) {
        if ((rc = narrow_all(b))) return rc;
    } else {
        BCK(cudaMemsetAsync(b->V32[0], 0, sizeof(float) * b->total, b->st));
    }
    if ((rc = set_params(b, o, o->warm ? 1 : 0))) return rc;
    if ((rc = ensure_graph(b, o->n_eval, diag))) return rc;
    BCK(launch_ctl(b, kStBegin));
    const long long max_replays = o->max_sweeps / kChunksPerGraph + 4;
    long long replays = 0;
    for (;;) {
        BCK(cudaGraphLaunch(b->exec, b->st));
        ++replays;
        BCK(cudaMemcpyAsync(&b->h_par->active, &b->d_par->active, sizeof(int), cudaMemcpyDeviceToHost, b->st));
        BCK(cudaStreamSynchronize(b->st));
        if (b->h_par->active == 0 || replays >= max_replays) break;
    }
    if ((rc = pull_state(b))) return rc;
    // a transfer whose last improvement ran with FP64 values stored 24-bit
    // word pairs; stand-alone evaluation sweeps read 8-byte feet, so the
    // stored feet serve them only if no transfer switched
    b->feet_valid = true;
    for (int t = 0; t < b->count; ++t)
        if (b->h_st[t].switch_outer >= 0) b->feet_valid = false;

    dp_solve_stats S;
    memset(&S, 0, sizeof S);
    S.converged = 1;
    S.switch_outer = -1;
    int nonfinite = 0;
    for (int t = 0; t < b->count; ++t) {
        const BState& s = b->h_st[t];
        S.sweeps_improve += s.imp32;
        S.sweeps_eval += s.eval32;
        S.sweeps_improve_fp64 += s.imp64;
        S.sweeps_eval_fp64 += s.eval64;
        S.residual = std::max(S.residual, s.res);
        S.converged = S.converged && s.converged && !s.nonfinite;
        S.node_updates += (s.imp32 + s.eval32 + s.imp64 + s.eval64) * (b->nodes[t] - b->targets[t]);
        S.switch_outer = std::max<long long>(S.switch_outer, s.switch_outer);
        nonfinite |= s.nonfinite;
        if (per) {
            dp_batch_stats& P = per[t];
            P.sweeps_improve = s.imp32;
            P.sweeps_eval = s.eval32;
            P.sweeps_improve_fp64 = s.imp64;
            P.sweeps_eval_fp64 = s.eval64;
            P.residual = s.res;
            P.converged = s.converged && !s.nonfinite;
            P.nonfinite = s.nonfinite;
            P.switch_outer = s.switch_outer;
            P.nodes = b->nodes[t];
        }
    }
    S.launches = 1 + replays * b->graph_launches;
    S.ms_wall = now_ms() - t0;
    if (total) *total = S;
    if (nonfinite) return bfail(DP_ENONFINITE, "a transfer produced a non-finite value");
    if (!S.converged)
        return bfail(DP_ENOCONV, "not every transfer converged within %lld improvement sweeps (max residual %g)",
                     (long long)o->max_sweeps, S.residual);
    return DP_OK;
}

int dp_batch_get_value(const dp_batch* b, int32_t index, double* host_V, int64_t count)
{
    int rc = check_index(b, index, count);
    if (rc) return rc;
    if (!host_V) return bfail(DP_EINVAL, "host_V is NULL");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(DP_ECUDA, "cudaSetDevice failed");
    if ((rc = pull_state(const_cast<dp_batch*>(b)))) return rc;
    const BState& s = b->h_st[index];
    const long long o = b->off[index];
    if (s.switch_outer >= 0) {
        BCK(cudaMemcpyAsync(host_V, b->V64[s.cur64] + o, sizeof(double) * count, cudaMemcpyDeviceToHost, b->st));
    } else {
        BCK(launch_load_value(b->V32[s.cur] + o, b->staging, 1, (int)count, b->st));
        BCK(cudaMemcpyAsync(host_V, b->staging, sizeof(double) * count, cudaMemcpyDeviceToHost, b->st));
    }
    BCK(cudaStreamSynchronize(b->st));
    return DP_OK;
}

int dp_batch_set_value(dp_batch* b, int32_t index, const double* host_V, int64_t count)
{
    int rc = check_index(b, index, count);
    if (rc) return rc;
    if (!host_V) return bfail(DP_EINVAL, "host_V is NULL");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(DP_ECUDA, "cudaSetDevice failed");
    if ((rc = pull_state(b))) return rc;
    BState& s = b->h_st[index];
    s.switch_outer = -1;
    Geo<double> g = b->g64[index];
    g.n_nodes = (int)count;
    int h_bad = 0;
    BCK(cudaMemcpyAsync(b->staging, host_V, sizeof(double) * count, cudaMemcpyHostToDevice, b->st));
    BCK(launch_store_value(b->staging, b->V32[s.cur] + b->off[index], 1, (int)count, g, b->d_bad, b->st));
    BCK(cudaMemcpyAsync(&h_bad, b->d_bad, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BCK(cudaMemcpyAsync(b->d_st, b->h_st, sizeof(BState) * b->count, cudaMemcpyHostToDevice, b->st));
    BCK(cudaStreamSynchronize(b->st));
    if (h_bad) return bfail(DP_ENONFINITE, "V holds a non-finite value");
    return DP_OK;
}

int dp_batch_get_policy(const dp_batch* b, int32_t index, uint16_t* host_codes, int64_t count)
{
    int rc = check_index(b, index, count);
    if (rc) return rc;
    if (!host_codes) return bfail(DP_EINVAL, "host_codes is NULL");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(DP_ECUDA, "cudaSetDevice failed");
    BCK(cudaMemcpyAsync(host_codes, b->code + b->off[index], sizeof(uint16_t) * count, cudaMemcpyDeviceToHost,
                        b->st));
    BCK(cudaStreamSynchronize(b->st));
    return DP_OK;
}

int dp_batch_set_policy(dp_batch* b, int32_t index, const uint16_t* host_codes, int64_t count)
{
    int rc = check_index(b, index, count);
    if (rc) return rc;
    if (!host_codes) return bfail(DP_EINVAL, "host_codes is NULL");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(DP_ECUDA, "cudaSetDevice failed");
    BCK(cudaMemcpyAsync(b->code + b->off[index], host_codes, sizeof(uint16_t) * count, cudaMemcpyHostToDevice,
                        b->st));
    BCK(cudaStreamSynchronize(b->st));
    b->feet_valid = false;   // the stored feet belong to the previous policy
    return DP_OK;
}

}  // extern "C"
