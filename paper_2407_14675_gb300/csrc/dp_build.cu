// dp_build.cu -- grid construction kernels: angle tables, the (energy-band
// reduced) node set as per-row v_t intervals with compact offsets, the line
// table used to decode a compact index, and value conversions.
//
// Reduced grid (§3 "Grid and polar coordinates": the computational domain is
// cut down to where optimal trajectories stay): a node is stored iff its
// specific energy (v_r^2 + v_t^2)/2 - mu/r lies in [e_lo, e_hi].  For v_t > 0
// the energy rises with v_t, so each (i_r, i_vr) row keeps one contiguous run
// of v_t nodes and all masses; the row table stores its first compact index,
// first v_t index and length.  The energy is evaluated in FP64 with
// explicitly rounded operations (no contraction), the same operation order as
// the CPU oracle, so both sides decide membership identically.
#include "dp_host.h"

namespace dpk {

__global__ void trig_tables_kernel(double2* hi64, double2* lo64, float2* hi32, float2* lo32)
{
    int k = threadIdx.x;   // 256 threads
    double s, c;
    sincospi((double)k / 128.0, &s, &c);      // 2 pi (k * 256) / 65536
    hi64[k] = make_double2(s, c);
    hi32[k] = make_float2((float)s, (float)c);
    sincospi((double)k / 32768.0, &s, &c);    // 2 pi k / 65536
    lo64[k] = make_double2(s, c);
    lo32[k] = make_float2((float)s, (float)c);
}

cudaError_t launch_trig_tables(double2* hi64, double2* lo64, float2* hi32, float2* lo32, cudaStream_t st)
{
    trig_tables_kernel<<<1, 256, 0, st>>>(hi64, lo64, hi32, lo32);
    return cudaGetLastError();
}

struct BoxGeom {
    int n[4];
    double lo[4], h[4];
};

__device__ __forceinline__ double node_coord(const BoxGeom& b, int d, int i)
{
    return __dadd_rn(b.lo[d], __dmul_rn((double)i, b.h[d]));
}

// One thread per (i_r, i_vr) row: the contiguous v_t run of stored nodes.
__global__ void rows_kernel(int4* rows, int* err, BoxGeom b, double mu, int reduced, double e_lo, double e_hi)
{
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= b.n[0] * b.n[1]) return;
    int ir = row / b.n[1], iv = row % b.n[1];
    if (!reduced) {
        rows[row] = make_int4(0, 0, b.n[2], 0);
        return;
    }
    double r = node_coord(b, 0, ir), vr = node_coord(b, 1, iv);
    int first = -1, last = -1, count = 0;
    for (int it = 0; it < b.n[2]; ++it) {
        double vt = node_coord(b, 2, it);
        double e = __dsub_rn(__dmul_rn(0.5, __dadd_rn(__dmul_rn(vr, vr), __dmul_rn(vt, vt))), __ddiv_rn(mu, r));
        if (e >= e_lo && e <= e_hi) {
            if (first < 0) first = it;
            last = it;
            ++count;
        }
    }
    if (count > 0 && last - first + 1 != count) atomicOr(err, 1);
    rows[row] = make_int4(0, count > 0 ? first : 0, count, 0);
}

cudaError_t launch_rows(int4* rows, int* err, int n0, int n1, int n2, int n3, const double* lo,
                        const double* h, double mu, int reduced, double e_lo, double e_hi, cudaStream_t st)
{
    BoxGeom b;
    b.n[0] = n0; b.n[1] = n1; b.n[2] = n2; b.n[3] = n3;
    for (int d = 0; d < 4; ++d) { b.lo[d] = lo[d]; b.h[d] = h[d]; }
    int n_rows = n0 * n1;
    rows_kernel<<<(n_rows + 255) / 256, 256, 0, st>>>(rows, err, b, mu, reduced, e_lo, e_hi);
    return cudaGetLastError();
}

// Exclusive prefix sum of len * n_m over rows (one block, chunked): the
// compact index of each row's first node.  total receives the node count;
// org (nullable) each row's origin, first index - lo_vt * n_m.
__global__ void row_offsets_kernel(int4* rows, int n_rows, int n_m, long long* total, int* org)
{
    __shared__ long long part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int chunk = (n_rows + T - 1) / T;
    const int a = t * chunk, b = min(a + chunk, n_rows);
    long long s = 0;
    for (int r = a; r < b; ++r) s += (long long)rows[r].z * n_m;
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {       // inclusive Hillis-Steele scan
        long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (int r = a; r < b; ++r) {
        rows[r].x = (int)run;
        if (org) org[r] = (int)(run - (long long)rows[r].y * n_m);
        run += (long long)rows[r].z * n_m;
    }
    if (t == T - 1) *total = part[t];
}

cudaError_t launch_row_offsets(int4* rows, int n_rows, int n_m, long long* total, cudaStream_t st, int* org)
{
    row_offsets_kernel<<<1, 1024, 0, st>>>(rows, n_rows, n_m, total, org);
    return cudaGetLastError();
}

// One thread per (row, i_vt): the packed line table.
__global__ void lines_kernel(const int4* rows, unsigned* lines, int n0, int n1, int n2, int n_m)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n0 * n1 * n2) return;
    int row = (int)(t / n2), it = (int)(t % n2);
    int4 R = rows[row];
    if (it < R.y || it >= R.y + R.z) return;
    int ir = row / n1, iv = row % n1;
    int line = R.x / n_m + (it - R.y);
    lines[line] = (unsigned)ir | ((unsigned)iv << 10) | ((unsigned)it << 20);
}

cudaError_t launch_lines(const int4* rows, unsigned* lines, int n0, int n1, int n2, int n_m, cudaStream_t st)
{
    long long n = (long long)n0 * n1 * n2;
    lines_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rows, lines, n0, n1, n2, n_m);
    return cudaGetLastError();
}

// Host values (FP64 or FP32, compact order) into storage precision; target
// nodes 0.  A first pass flags non-finite input; the store pass then leaves V
// untouched.
template <typename H>
__global__ void check_finite_kernel(const H* src, int n, int* bad)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && !isfinite(src[j])) atomicOr(bad, 1);
}

template <typename H>
__global__ void store_value_kernel(const H* src, void* dst, int fp32, Geo<double> g, const int* bad)
{
    if (*bad) return;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    int i[4];
    decode_node(g, j, i);
    const bool t = in_target(g, i);
    if (fp32) ((float*)dst)[j] = t ? 0.0f : (float)src[j];
    else ((double*)dst)[j] = t ? 0.0 : (double)src[j];
}

template <typename H>
cudaError_t store_value(const H* src, void* dst, int fp32, int n, const Geo<double>& g, int* bad, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    check_finite_kernel<H><<<(n + 255) / 256, 256, 0, st>>>(src, n, bad);
    store_value_kernel<H><<<(n + 255) / 256, 256, 0, st>>>(src, dst, fp32, g, bad);
    return cudaGetLastError();
}

cudaError_t launch_store_value(const double* src, void* dst, int fp32, int n, const Geo<double>& g, int* bad,
                               cudaStream_t st)
{
    return store_value(src, dst, fp32, n, g, bad, st);
}

cudaError_t launch_store_value(const float* src, void* dst, int fp32, int n, const Geo<double>& g, int* bad,
                               cudaStream_t st)
{
    return store_value(src, dst, fp32, n, g, bad, st);
}

// Stored values (FP32 or FP64) into a staging buffer of type H.
template <typename H>
__global__ void load_value_kernel(const void* src, H* dst, int fp32, int n)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    dst[j] = fp32 ? (H)((const float*)src)[j] : (H)((const double*)src)[j];
}

cudaError_t launch_load_value(const void* src, double* dst, int fp32, int n, cudaStream_t st)
{
    load_value_kernel<double><<<(n + 255) / 256, 256, 0, st>>>(src, dst, fp32, n);
    return cudaGetLastError();
}

cudaError_t launch_load_value(const void* src, float* dst, int fp32, int n, cudaStream_t st)
{
    load_value_kernel<float><<<(n + 255) / 256, 256, 0, st>>>(src, dst, fp32, n);
    return cudaGetLastError();
}

__global__ void widen_kernel(const float* src, double* dst, int n)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = (double)src[j];
}

cudaError_t launch_widen(const float* src, double* dst, int n, cudaStream_t st)
{
    widen_kernel<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

// Warm start of grid gd from the value and policy of grid gs (the same
// problem at another resolution or box): Q1 interpolation of gs's value at
// every stored node of gd (Md where the node lies outside gs's box or its gs
// cell has a corner outside gs's node set), and the policy code of the
// nearest gs node (0 where that node is not stored).  Target nodes of gd get
// value 0.  FP64 coordinates and blend; the same strict outside test as the
// sweeps.
template <typename S, bool SRC_REDUCED, bool PER3>
__global__ void prolong_kernel(Geo<double> gs, const S* __restrict__ Vs, const uint16_t* __restrict__ Cs,
                               Geo<double> gd, void* Vd, int fp32_dst, uint16_t* __restrict__ Cd, double Md)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= gd.n_nodes) return;
    int id[4];
    decode_node(gd, j, id);
    double v = 0.0;
    uint16_t code = 0;
    if (!in_target(gd, id)) {
        double s[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) s[d] = (gd.lo[d] + (double)id[d] * gd.h[d] - gs.lo[d]) / gs.h[d];
        const int zero[4] = {0, 0, 0, 0};
        int c[4];
        double t[4];
        Corners<double> K;
        const bool out = foot_cell<double, PER3>(gs, zero, s, c, t) ||
                         load_corners<double, double, S, SRC_REDUCED, PER3>(gs, Vs, c, (S)0, K);
        v = out ? Md : K.blend(t);
        // nearest source node for the policy
        int nn[4];
        bool have = true;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            int k = (int)floor(s[d] + 0.5);
            if (PER3 && d == 3) k = ((k % gs.n[3]) + gs.n[3]) % gs.n[3];
            nn[d] = min(max(k, 0), gs.n[d] - 1);
        }
        long long idx;
        if (!SRC_REDUCED) {
            idx = (((long long)nn[0] * gs.n[1] + nn[1]) * gs.n[2] + nn[2]) * gs.n[3] + nn[3];
        } else {
            const int4 R = gs.rows[nn[0] * gs.n[1] + nn[1]];
            have = nn[2] >= R.y && nn[2] < R.y + R.z;
            idx = have ? (long long)R.x + (long long)(nn[2] - R.y) * gs.n_m + nn[3] : 0;
        }
        code = have ? Cs[idx] : (uint16_t)0;
    }
    if (fp32_dst) ((float*)Vd)[j] = (float)v;
    else ((double*)Vd)[j] = v;
    Cd[j] = code;
}

template <typename S>
static cudaError_t launch_prolong_t(const Geo<double>& gs, const S* Vs, const uint16_t* Cs, int src_reduced,
                                    int periodic, const Geo<double>& gd, void* Vd, int fp32_dst, uint16_t* Cd,
                                    double Md, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((gd.n_nodes + 255) / 256);
    if (periodic)
        prolong_kernel<S, false, true><<<blocks, 256, 0, st>>>(gs, Vs, Cs, gd, Vd, fp32_dst, Cd, Md);
    else if (src_reduced)
        prolong_kernel<S, true, false><<<blocks, 256, 0, st>>>(gs, Vs, Cs, gd, Vd, fp32_dst, Cd, Md);
    else
        prolong_kernel<S, false, false><<<blocks, 256, 0, st>>>(gs, Vs, Cs, gd, Vd, fp32_dst, Cd, Md);
    return cudaGetLastError();
}

cudaError_t launch_prolong(const Geo<double>& gs, const void* Vs, int src_fp32, const uint16_t* Cs, int src_reduced,
                           int periodic, const Geo<double>& gd, void* Vd, int fp32_dst, uint16_t* Cd, double Md,
                           cudaStream_t st)
{
    if (src_fp32)
        return launch_prolong_t<float>(gs, (const float*)Vs, Cs, src_reduced, periodic, gd, Vd, fp32_dst, Cd, Md, st);
    return launch_prolong_t<double>(gs, (const double*)Vs, Cs, src_reduced, periodic, gd, Vd, fp32_dst, Cd, Md, st);
}

__global__ void box_index_kernel(Geo<double> g, long long* out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    int i[4];
    decode_node(g, j, i);
    out[j] = (((long long)i[0] * g.n[1] + i[1]) * g.n[2] + i[2]) * g.n[3] + i[3];
}

cudaError_t launch_box_index(const Geo<double>& g, long long* out, cudaStream_t st)
{
    box_index_kernel<<<(g.n_nodes + 255) / 256, 256, 0, st>>>(g, out);
    return cudaGetLastError();
}

}  // namespace dpk
