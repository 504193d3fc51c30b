// dp_noalloc.cu -- dp_bellman_sweep_noalloc: one Jacobi sweep on caller-owned
// device buffers with no device allocation at all.
//
// Some callers cannot call cudaMalloc: flight or other real-time software
// that forbids allocation once it has started, and hosts whose device memory
// is owned by another allocator (a framework's caching allocator or a fixed
// pool that has to account for every byte), where an extra cudaMalloc can
// fail or fragment that pool.  dp_grid_create allocates, so such callers
// cannot hold a grid.  This call takes the grid description and the caller's
// device buffers, and keeps every table and accumulator the sweep needs (row
// and line tables of the node set, angle tables, the residual slot, the
// control block) in one file-scope __device__ array of fixed size, which
// every GPU that loads the library holds until the process exits.
#include <cstdio>
#include <cstring>

#include "dp.h"
#include "dp_host.h"

namespace dpk {
int record_error(int code, const char* msg);
int describe_full_grid(const dp_grid_desc* desc, Geo<double>* g64, Geo<float>* g32, long long* n_nodes);
}  // namespace dpk

using namespace dpk;

namespace {

constexpr long long kMaxRows = 4096;     // n0 n1
constexpr long long kMaxLines = 262144;  // n0 n1 n2
constexpr size_t kRowsOff = 0;
constexpr size_t kLinesOff = kRowsOff + kMaxRows * sizeof(int4);
constexpr size_t kTabOff = kLinesOff + kMaxLines * sizeof(unsigned);
constexpr size_t kHi64 = kTabOff, kLo64 = kHi64 + 256 * sizeof(double2);
constexpr size_t kHi32 = kLo64 + 256 * sizeof(double2), kLo32 = kHi32 + 256 * sizeof(float2);
constexpr size_t kTotalOff = kLo32 + 256 * sizeof(float2);
constexpr size_t kRingOff = kTotalOff + 256;
constexpr size_t kCtlOff = kRingOff + 256;
constexpr size_t kScratchBytes = kCtlOff + 256;
static_assert(kScratchBytes == 1127168, "scratch layout");

}  // namespace

// The shared scratch of dp_bellman_sweep_noalloc (all calls, all streams).
static __device__ __align__(256) unsigned char dp_noalloc_scratch[kScratchBytes];

namespace {

// Device address of the scratch array in the current context.  The lookup
// runs on every call: it is a host-side query that allocates nothing, and an
// address kept from an earlier call would belong to a dead context after
// cudaDeviceReset, or to another context when the caller has made a
// non-primary driver-API context current.  (Under lazy module loading the
// first lookup in a context loads the module, which places the array.)
int scratch_address(unsigned char** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, dp_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return record_error(DP_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
    }
    *out = (unsigned char*)p;
    return DP_OK;
}

// Internal sweep mode of the public DP_SWEEP_VI ... DP_SWEEP_EVAL.
int sweep_mode(int mode)
{
    switch (mode) {
    case DP_SWEEP_VI: return kVI;
    case DP_SWEEP_IMPROVE_FULL: return kImproveFull;
    case DP_SWEEP_IMPROVE_WALK: return kImproveWalk;
    case DP_SWEEP_EVAL: return kEval;
    }
    return -1;
}

int cuda_fail(const char* what, cudaError_t e)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return record_error(DP_ECUDA, buf);
}

template <typename G, typename S>
int run(const Geo<G>& geo, unsigned char* scr, int mode, const void* V_in, void* V_out, uint16_t* codes,
        int dyn, cudaStream_t st, int sm_count)
{
    SweepLaunch<G, S> L;
    L.g = geo;
    L.Vin = (const S*)V_in;
    L.Vout = (S*)V_out;
    L.code = codes;
    L.feet_lo = nullptr;
    L.feet_hi = nullptr;
    L.inc = nullptr;
    L.acc = nullptr;
    L.V64 = nullptr;
    L.incr_flags = 0;
    L.ctl = (Ctl*)(scr + kCtlOff);
    L.ring = (unsigned long long*)(scr + kRingOff);
    L.ring_mask = 0;
    L.sweep = 0;
    L.check_prev = 0;
    L.tol = 0.0;
    L.mode = mode;
    L.dyn = dyn;
    L.reduced = 0;
    L.stream = st;
    L.sm_count = sm_count;
    cudaError_t e = launch_sweep(L);
    return e == cudaSuccess ? DP_OK : cuda_fail("sweep launch", e);
}

}  // namespace

extern "C" int dp_bellman_sweep_noalloc(const dp_grid_desc* desc, int32_t mode, const void* V_in, void* V_out,
                                        uint16_t* codes, double* residual)
{
    Geo<double> g64;
    Geo<float> g32;
    long long n = 0;
    int rc = describe_full_grid(desc, &g64, &g32, &n);
    if (rc) return rc;
    const int kmode = sweep_mode(mode);
    if (kmode < 0) return record_error(DP_EINVAL, "unknown sweep mode");
    if (!V_in || !V_out || V_in == V_out) return record_error(DP_EINVAL, "V_in and V_out must be distinct device buffers");
    if (mode != DP_SWEEP_VI && !codes) return record_error(DP_EINVAL, "this sweep mode needs the policy buffer");
    const long long rows = (long long)desc->n[0] * desc->n[1];
    const long long lines = rows * desc->n[2];
    if (rows > kMaxRows || lines > kMaxLines)
        return record_error(DP_EINVAL, "grid too large for the no-allocation sweep: needs n0*n1 <= 4096 and "
                                       "n0*n1*n2 <= 262144 (the fixed scratch holds 1,127,168 bytes)");
    int dev = 0, sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    if ((e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail("device query", e);
    unsigned char* scr = nullptr;
    if ((rc = scratch_address(&scr))) return rc;
    cudaStream_t st = (cudaStream_t)desc->stream;

    // tables of the node set and the angles, rebuilt in the scratch each call
    int4* d_rows = (int4*)(scr + kRowsOff);
    unsigned* d_lines = (unsigned*)(scr + kLinesOff);
    double h[4];
    for (int k = 0; k < 4; ++k) h[k] = (desc->hi[k] - desc->lo[k]) / (double)(desc->n[k] - 1);
    if ((e = launch_rows(d_rows, (int*)(scr + kCtlOff), desc->n[0], desc->n[1], desc->n[2], desc->n[3], desc->lo, h,
                         desc->mu, 0, 0.0, 0.0, st)) != cudaSuccess ||
        (e = launch_row_offsets(d_rows, (int)rows, desc->n[3], (long long*)(scr + kTotalOff), st)) != cudaSuccess ||
        (e = launch_lines(d_rows, d_lines, desc->n[0], desc->n[1], desc->n[2], desc->n[3], st)) != cudaSuccess ||
        (e = launch_trig_tables((double2*)(scr + kHi64), (double2*)(scr + kLo64), (float2*)(scr + kHi32),
                                (float2*)(scr + kLo32), st)) != cudaSuccess)
        return cuda_fail("table set-up", e);
    // the residual slot and the control block start at zero every call
    if ((e = cudaMemsetAsync(scr + kRingOff, 0, 256, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(scr + kCtlOff, 0, 256, st)) != cudaSuccess)
        return cuda_fail("scratch reset", e);

    g64.rows = g32.rows = d_rows;
    g64.row_org = g32.row_org = nullptr;   // no frozen feet here
    g64.lines = g32.lines = d_lines;
    g64.tab_hi = (const double2*)(scr + kHi64);
    g64.tab_lo = (const double2*)(scr + kLo64);
    g32.tab_hi = (const float2*)(scr + kHi32);
    g32.tab_lo = (const float2*)(scr + kLo32);
    if (desc->precision == DP_FP64)
        rc = run<double, double>(g64, scr, kmode, V_in, V_out, codes, desc->dynamics, st, sm);
    else
        rc = run<float, float>(g32, scr, kmode, V_in, V_out, codes, desc->dynamics, st, sm);
    if (rc) return rc;

    unsigned long long bits = 0;
    Ctl ctl;
    memset(&ctl, 0, sizeof ctl);
    if ((e = cudaMemcpyAsync(&bits, scr + kRingOff, sizeof bits, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&ctl, scr + kCtlOff, sizeof ctl, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail("residual read-back", e);
    if (residual) memcpy(residual, &bits, sizeof bits);
    if (ctl.nonfinite) return record_error(DP_ENONFINITE, "the sweep produced a non-finite value");
    return DP_OK;
}
