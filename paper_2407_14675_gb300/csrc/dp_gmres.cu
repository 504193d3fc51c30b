// dp_gmres.cu -- policy evaluation by restarted GMRES.
//
// §3, after Eq. (14): with the control frozen, the evaluation step of policy
// iteration (Eq. (13)) is a linear system whose row j holds the Q1 weights of
// node j's foot, and the paper solves it with GMRES.  A = I - beta W_f is
// never assembled: a product A x is one gather-and-blend pass over the nodes,
// the work of one evaluation sweep (FP32 grids read the frozen feet that the
// improvement sweep stored, FP64 grids recompute the foot from the policy
// code).  The penalty M and the running cost are the constant part b of the
// affine map T_f(V) = b + beta W_f V, so they never enter a product.
//
// One cycle corrects a value V whose image T_f(V) is already known:
//   r0 = T_f(V) - V, Arnoldi on A from r0 (m steps, classical Gram-Schmidt,
//   optionally twice), y = argmin ||beta0 e1 - H y||, V <- V + Q y.
// The basis vectors are stored unnormalised, with scale[i] = 1 / ||Q_i||.
// An Arnoldi step is three launches: the product (gather-bound, one node per
// thread at the evaluation sweep's occupancy), the projections, and the
// update with the norm (both streaming, tiles of kGmTile nodes with 16-byte
// loads).  A streaming launch sums its dot products per block into a partial
// row, and the last block to finish adds the rows in a fixed order (the
// result does not depend on block scheduling) and does the O(m) Hessenberg
// and Givens work on one thread.  No block waits for another.
//
// Element-wise work and the warp reductions run in the basis precision VT
// (FP32 on FP32 grids: the FP64 pipe of this GPU is a small fraction of its
// FP32 pipe, and FP64 adds in every lane of the warp trees made the
// orthogonalisation FP64-bound).  Each warp's total over 128 products is
// widened to FP64 for the block and grid sums and the Hessenberg problem.
#include "dp_sweep.cuh"

namespace dpk {
namespace {

constexpr int kGmBlock = 256;
constexpr int kGmS = 4;                     // nodes per thread and tile (four consecutive
                                            // nodes per thread in the streaming loops)
constexpr int kGmTile = kGmBlock * kGmS;
constexpr int kGmWarps = kGmBlock / 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-block sums: every warp adds into its own row.
struct BlockSums {
    double acc[kGmWarps][kGmLd];
};

__device__ __forceinline__ void sums_zero(BlockSums& S)
{
    for (int c = threadIdx.x; c < kGmWarps * kGmLd; c += kGmBlock) (&S.acc[0][0])[c] = 0.0;
    __syncthreads();
}

// Adds the warp's total of v to column c.  Every lane of the warp calls it.
// The warp tree runs in v's precision (a pairwise sum of 32 per-thread
// partials); only its total is widened to FP64.
template <typename T>
__device__ __forceinline__ void sums_add(BlockSums& S, int c, T v)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) S.acc[threadIdx.x >> 5][c] += (double)v;
}

// Stores the block's columns [0, ncol) in its partial row.  Returns true in
// every thread of the last block to finish, with red[c] = the sum over all
// blocks (lane-strided over blocks, then a fixed shuffle tree).
__device__ bool sums_finish(BlockSums& S, int ncol, double* __restrict__ partial, GmCtl* gc, double* red)
{
    __shared__ int s_last;
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += kGmBlock) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kGmWarps; ++w) v += S.acc[w][c];
        partial[(size_t)blockIdx.x * kGmLd + c] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&gc->counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < ncol; c += kGmWarps) {
        double v = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(&partial[(size_t)b * kGmLd + c]);
        v = warp_sum(v);
        if (lane == 0) red[c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) gc->counter = 0;
    return true;
}

// Four consecutive entries j4..j4+3 of a vector (j4 a multiple of 4 and the
// vector 16-byte aligned: one or two 16-byte accesses); entries at or past n
// read as 0 and are not written.
__device__ __forceinline__ void ld4(const float* p, float v[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4])
{
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4])
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
template <typename T>
__device__ __forceinline__ void load4(const T* p, int j4, int n, T v[4])
{
    if (j4 + 3 < n) {
        ld4(p + j4, v);
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) v[s] = j4 + s < n ? p[j4 + s] : (T)0;
    }
}
template <typename T>
__device__ __forceinline__ void store4(T* p, int j4, int n, const T v[4])
{
    if (j4 + 3 < n) {
        st4(p + j4, v);
    } else {
#pragma unroll
        for (int s = 0; s < 4; ++s)
            if (j4 + s < n) p[j4 + s] = v[s];
    }
}

// (A x)_j = x_j - beta (W_f x)_j from node j's frozen foot (FP32 geometry).
// A foot outside the box or the node set, and a target node, have no W row.
template <bool REDUCED, int DYN, typename W>
__device__ __forceinline__ float apply_a_feet(const Geo<float>& g, const float* __restrict__ x, int j, W w,
                                              const uint16_t* __restrict__ code)
{
    const float xj = x[j];
    const int kind = foot_kind(w);
    float D = 0.0f;
    if (kind == kFootInside) D = eval_foot<REDUCED>(g, x, j, w, 0.0f);
    else if (kind == kFootRecompute) D = incr_recompute<REDUCED, DYN>(g, x, j, code[j]);
    return xj - fmaf(g.beta_hi, D, g.beta_lo * D);
}

// The same product with the foot recomputed from the policy code (FP64).  The
// geometry carries M = 0, so a foot outside the box blends to 0.
template <bool REDUCED, int DYN>
__device__ __forceinline__ double apply_a_node(const Geo<double>& g, const double* __restrict__ x, int j,
                                               const uint16_t* __restrict__ code)
{
    const double xj = x[j];
    NodeEval<double, double, REDUCED, DYN> ev;
    decode_node(g, j, ev.i);
    if (in_target(g, ev.i)) return xj;
    setup_node<double, double, DYN>(ev, g, x, xj);
    const int c = code[j];
    double D;
    if (DYN == kDynPolar && g.off && c == kCodeOff) D = ev.at_sc(0.0, 0.0);
    else D = ev.at_code(c);
    return xj - g.beta64 * (xj + D);
}

// The same from an FP64 frozen foot (offsets word and fractions).
template <bool REDUCED, int DYN>
__device__ __forceinline__ double apply_a_feet64(const Geo<double>& g, const double* __restrict__ x, int j,
                                                 const Feet64& f64, const uint16_t* __restrict__ code)
{
    constexpr bool kPer = DYN == kDynPolar;
    const double xj = x[j];
    const unsigned long long w = __ldcs(&f64.w[j]);
    const int kind = (int)((w >> 32) & 3u);
    if (kind == kFootInside) {
        int i[4], cl[4];
        decode_node(g, j, i);
#pragma unroll
        for (int d = 0; d < 4; ++d) cl[d] = i[d] + (int)(signed char)((w >> (8 * d)) & 0xffu);
        if (kPer) cl[3] = cl[3] < 0 ? cl[3] + g.n[3] : (cl[3] >= g.n[3] ? cl[3] - g.n[3] : cl[3]);
        const double2 ta = __ldcs(&f64.t[2 * (size_t)j]), tb = __ldcs(&f64.t[2 * (size_t)j + 1]);
        const double t[4] = {ta.x, ta.y, tb.x, tb.y};
        Corners<double> K;
        load_corners<double, double, double, REDUCED, kPer>(g, x, cl, 0.0, K);
        return xj - g.beta64 * K.blend(t);
    }
    if (kind == kFootRecompute) return apply_a_node<REDUCED, DYN>(g, x, j, code);
    return xj;   // outside or target: no W row
}

// r0 = V_next - V_in into Q_0, and ||r0||.
template <typename VV, typename VT>
__global__ void __launch_bounds__(kGmBlock)
gm_start_kernel(const VV* __restrict__ Vin, const VV* __restrict__ Vnext, VT* __restrict__ q0, int n,
                double* __restrict__ partial, GmCtl* __restrict__ gc)
{
    __shared__ BlockSums S;
    __shared__ double red[kGmLd];
    sums_zero(S);
    const int tiles = (n + kGmTile - 1) / kGmTile;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int j4 = tile * kGmTile + kGmS * threadIdx.x;
        VV a[kGmS], b[kGmS];
        VT r[kGmS];
        load4(Vin, j4, n, a);
        load4(Vnext, j4, n, b);
        VT nrm = (VT)0;
#pragma unroll
        for (int s = 0; s < kGmS; ++s) {
            r[s] = (VT)(b[s] - a[s]);
            nrm += r[s] * r[s];
        }
        store4(q0, j4, n, r);
        sums_add(S, 0, nrm);
    }
    if (!sums_finish(S, 1, partial, gc, red)) return;
    if (threadIdx.x == 0) {
        const double b = sqrt(red[0]);
        const bool ok = b > 0.0 && isfinite(b);
        gc->beta0 = b;
        gc->gv[0] = b;
        gc->rel = ok ? 1.0 : 0.0;
        gc->k = 0;
        gc->scale[0] = ok ? 1.0 / b : 0.0;
        gc->done = ok ? 0 : 1;
    }
}

// Arnoldi step k, the product: Q_{k+1} = A q_k (q_k = scale[k] Q_k).  One
// node per thread, nodes of a warp adjacent, the next node's foot and value
// fetched while this node's corners are in flight (as in the evaluation
// sweep); compiled for the sweep's occupancy on FP32 grids.
template <typename G>
constexpr int matvec_min_blocks() { return std::is_same<G, float>::value ? 6 : 2; }

template <typename G, typename VT, bool REDUCED, int DYN>
__global__ void __launch_bounds__(kGmBlock, matvec_min_blocks<G>())
gm_matvec_kernel(const __grid_constant__ Geo<G> g, VT* __restrict__ Q, long long ldq, int k,
                 const uint16_t* __restrict__ code, const unsigned long long* __restrict__ feet_lo,
                 const unsigned* __restrict__ feet_hi, const Feet64 f64, const GmCtl* __restrict__ gc)
{
    if (*(const volatile int*)&gc->done) return;
    const VT* x = Q + (size_t)k * ldq;
    VT* w = Q + (size_t)(k + 1) * ldq;
    const VT sk = (VT)gc->scale[k];
    const int n = g.n_nodes;
    const int stride = gridDim.x * kGmBlock;
    if constexpr (std::is_same<G, float>::value) {
        int j = blockIdx.x * kGmBlock + threadIdx.x;
        if (feet_hi) {
            // the word pair of the FP64-value phase
            FootWord next{0ull, 0u};
            if (j < n) next = FootWord{__ldcs(&feet_lo[j]), __ldcs(&feet_hi[j])};
            for (; j < n; j += stride) {
                const FootWord fw = next;
                if (j + stride < n) next = FootWord{__ldcs(&feet_lo[j + stride]), __ldcs(&feet_hi[j + stride])};
                w[j] = sk * apply_a_feet<REDUCED, DYN>(g, x, j, fw, code);
            }
        } else {
            // 8-byte feet of the FP32-value phase
            unsigned long long next = 0ull;
            if (j < n) next = __ldcs(&feet_lo[j]);
            for (; j < n; j += stride) {
                const unsigned long long fw = next;
                if (j + stride < n) next = __ldcs(&feet_lo[j + stride]);
                w[j] = sk * apply_a_feet<REDUCED, DYN>(g, x, j, fw, code);
            }
        }
    } else if (f64.w) {
        for (int j = blockIdx.x * kGmBlock + threadIdx.x; j < n; j += stride)
            w[j] = sk * apply_a_feet64<REDUCED, DYN>(g, x, j, f64, code);
    } else {
        for (int j = blockIdx.x * kGmBlock + threadIdx.x; j < n; j += stride)
            w[j] = sk * apply_a_node<REDUCED, DYN>(g, x, j, code);
    }
}

// Closes column k once ||Q_{k+1}||^2 is known: rotations, residual estimate,
// and, when the cycle ends, the back substitution R y = g into coef (as
// coefficients of the raw Q_i).  One thread.
__device__ void finalize_column(GmCtl* gc, int k, int m, double rtol, double nrm2)
{
    const double nu = sqrt(fmax(nrm2, 0.0));
    for (int i = 0; i < k; ++i) {
        const double a = gc->H[i][k], b = gc->H[i + 1][k];
        gc->H[i][k] = gc->cs[i] * a + gc->sn[i] * b;
        gc->H[i + 1][k] = -gc->sn[i] * a + gc->cs[i] * b;
    }
    const double a = gc->H[k][k];
    const double r = hypot(a, nu);
    int kk = k + 1;
    bool stop = kk >= m;
    if (!(r > 0.0) || !isfinite(r)) {
        kk = k;             // no usable column: solve with the previous ones
        stop = true;
    } else {
        const double c = a / r, s = nu / r;
        gc->cs[k] = c;
        gc->sn[k] = s;
        gc->H[k][k] = r;
        gc->H[k + 1][k] = 0.0;
        gc->gv[k + 1] = -s * gc->gv[k];
        gc->gv[k] = c * gc->gv[k];
        gc->scale[k + 1] = nu > 0.0 ? 1.0 / nu : 0.0;
        gc->rel = fabs(gc->gv[k + 1]) / gc->beta0;
        // converged, or the Krylov space is (numerically) invariant
        if (gc->rel <= rtol || !(nu > 1e-14 * r)) stop = true;
    }
    gc->k = kk;
    if (stop) {
        for (int i = kk - 1; i >= 0; --i) {
            double v = gc->gv[i];
            for (int l = i + 1; l < kk; ++l) v -= gc->H[i][l] * gc->coef[l];
            gc->coef[i] = v / gc->H[i][i];
        }
        for (int i = 0; i < kk; ++i) gc->coef[i] *= gc->scale[i];
        gc->done = 1;
    }
}

// Arnoldi step k, Gram-Schmidt on Q_{k+1}.  SUB: Q_{k+1} -= sum_i coef_i Q_i.
// DOTS: the projections h_ik = <q_i, Q_{k+1}> of the result, which set column
// k of H (first pass, !SUB) or correct it (second pass) and become the next
// coefficients; otherwise the norm that closes the column.
template <typename VT, bool SUB, bool DOTS>
__global__ void __launch_bounds__(kGmBlock)
gm_update_kernel(VT* __restrict__ Q, long long ldq, int n, int k, int m, double rtol, double* __restrict__ partial,
                 GmCtl* __restrict__ gc)
{
    if (*(volatile int*)&gc->done) return;
    __shared__ BlockSums S;
    __shared__ double red[kGmLd];
    __shared__ VT s_coef[kGmMaxRestart + 1];
    if (SUB)
        for (int i = threadIdx.x; i <= k; i += kGmBlock) s_coef[i] = (VT)gc->coef[i];
    sums_zero(S);
    VT* w = Q + (size_t)(k + 1) * ldq;
    const int tiles = (n + kGmTile - 1) / kGmTile;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int j4 = tile * kGmTile + kGmS * threadIdx.x;
        VT wv[kGmS];
        load4(w, j4, n, wv);
        if constexpr (SUB) {
#pragma unroll 4
            for (int i = 0; i <= k; ++i) {
                VT q[kGmS];
                load4(Q + (size_t)i * ldq, j4, n, q);
                const VT c = s_coef[i];
#pragma unroll
                for (int s = 0; s < kGmS; ++s) wv[s] -= c * q[s];
            }
            store4(w, j4, n, wv);
        }
        VT nrm = (VT)0;
#pragma unroll
        for (int s = 0; s < kGmS; ++s) nrm += wv[s] * wv[s];
        if constexpr (DOTS) {
#pragma unroll 4
            for (int i = 0; i <= k; ++i) {
                VT q[kGmS];
                load4(Q + (size_t)i * ldq, j4, n, q);
                VT d = (VT)0;
#pragma unroll
                for (int s = 0; s < kGmS; ++s) d += q[s] * wv[s];
                sums_add(S, i, d);
            }
        } else {
            sums_add(S, 0, nrm);
        }
    }
    if (!sums_finish(S, DOTS ? k + 1 : 1, partial, gc, red)) return;
    if (threadIdx.x == 0) {
        if constexpr (DOTS) {
            for (int i = 0; i <= k; ++i) {
                const double h = gc->scale[i] * red[i];
                gc->H[i][k] = SUB ? gc->H[i][k] + h : h;
                gc->coef[i] = h * gc->scale[i];
            }
        } else {
            finalize_column(gc, k, m, rtol, red[0]);
        }
    }
}

// V_next = V_in + sum_i coef_i Q_i over the cycle's k columns; the
// correction is summed in the basis precision and added once to V_in.
template <typename VV, typename VT>
__global__ void __launch_bounds__(kGmBlock)
gm_apply_kernel(const VV* __restrict__ Vin, VV* __restrict__ Vnext, const VT* __restrict__ Q, long long ldq, int n,
                const GmCtl* __restrict__ gc, Ctl* __restrict__ ctl)
{
    __shared__ VT s_coef[kGmMaxRestart + 1];
    const int kk = gc->k;
    for (int i = threadIdx.x; i < kk; i += kGmBlock) s_coef[i] = (VT)gc->coef[i];
    __syncthreads();
    bool bad = false;
    const int tiles = (n + kGmTile - 1) / kGmTile;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int j4 = tile * kGmTile + kGmS * threadIdx.x;
        VT e[kGmS];
#pragma unroll
        for (int s = 0; s < kGmS; ++s) e[s] = (VT)0;
#pragma unroll 4
        for (int i = 0; i < kk; ++i) {
            VT q[kGmS];
            load4(Q + (size_t)i * ldq, j4, n, q);
            const VT c = s_coef[i];
#pragma unroll
            for (int s = 0; s < kGmS; ++s) e[s] += c * q[s];
        }
        VV v[kGmS];
        load4(Vin, j4, n, v);
#pragma unroll
        for (int s = 0; s < kGmS; ++s) {
            v[s] += (VV)e[s];
            bad = bad || (j4 + s < n && !isfinite(v[s]));
        }
        store4(Vnext, j4, n, v);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->nonfinite, 1);
}

// Frozen feet of the resident policy, the words an improvement sweep stores:
// the word pair when feet_hi is given (FP64-value phase), else the 8-byte
// word (FP32-value phase).
template <bool REDUCED, int DYN>
__global__ void __launch_bounds__(kGmBlock)
feet_kernel(const __grid_constant__ Geo<float> g, const uint16_t* __restrict__ code,
            unsigned long long* __restrict__ feet_lo, unsigned* __restrict__ feet_hi)
{
    for (int j = blockIdx.x * kGmBlock + threadIdx.x; j < g.n_nodes; j += gridDim.x * kGmBlock) {
        CachedEval<float, float, REDUCED, DYN, float, false> ev;
        decode_node(g, j, ev.i);
        const bool target = in_target(g, ev.i);
        if (!target) setup_node<float, float, DYN>(ev, g, (const float*)nullptr, 0.0f);
        if (feet_hi) {
            const FootWord w = target ? foot_word_kind(kFootTarget) : ev.foot_of(code[j]);
            feet_lo[j] = w.lo;
            feet_hi[j] = w.hi;
        } else {
            feet_lo[j] = target ? foot8_kind(kFootTarget) : ev.foot8_of(code[j]);
        }
    }
}

// Blocks for a tiled launch: resident blocks on every SM, at most one per
// tile and at most max_blocks (rows of the partial-sum buffer).
template <typename K>
int tiled_blocks(K kern, int n, int sm_count, int max_blocks, int& per_sm)
{
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGmBlock, 0) != cudaSuccess) per_sm = 1;
        if (per_sm < 1) per_sm = 1;
    }
    long long tiles = ((long long)n + kGmTile - 1) / kGmTile;
    long long b = (long long)per_sm * sm_count;
    if (b > max_blocks) b = max_blocks;
    if (b > tiles) b = tiles;
    return b < 1 ? 1 : (int)b;
}

template <typename G, typename VT, bool REDUCED, int DYN>
cudaError_t launch_arnoldi(const GmArgs<G, VT>& a, int k)
{
    auto kern = gm_matvec_kernel<G, VT, REDUCED, DYN>;
    static int per_sm = 0;
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGmBlock, 0) != cudaSuccess) per_sm = 1;
        if (per_sm < 1) per_sm = 1;
    }
    const long long need = ((long long)a.g.n_nodes + kGmBlock - 1) / kGmBlock;
    const long long cap = (long long)per_sm * a.sm_count;
    const int b = (int)(need < cap ? (need < 1 ? 1 : need) : cap);
    kern<<<b, kGmBlock, 0, a.stream>>>(a.g, a.Q, a.ldq, k, a.code, a.feet_lo, a.feet_hi, a.f64, a.gctl);
    return cudaGetLastError();
}

template <typename VT, bool SUB, bool DOTS>
cudaError_t launch_update(const GmArgs<float, VT>& a, int n, int k)
{
    auto kern = gm_update_kernel<VT, SUB, DOTS>;
    static int per_sm = 0;
    const int b = tiled_blocks(kern, n, a.sm_count, a.max_blocks, per_sm);
    kern<<<b, kGmBlock, 0, a.stream>>>(a.Q, a.ldq, n, k, a.m, a.rtol, a.partial, a.gctl);
    return cudaGetLastError();
}
template <typename VT, bool SUB, bool DOTS>
cudaError_t launch_update(const GmArgs<double, VT>& a, int n, int k)
{
    auto kern = gm_update_kernel<VT, SUB, DOTS>;
    static int per_sm = 0;
    const int b = tiled_blocks(kern, n, a.sm_count, a.max_blocks, per_sm);
    kern<<<b, kGmBlock, 0, a.stream>>>(a.Q, a.ldq, n, k, a.m, a.rtol, a.partial, a.gctl);
    return cudaGetLastError();
}

cudaError_t dispatch_arnoldi(const GmArgs<float, float>& a, int k)
{
    if (a.dyn == kDynUnitSpeed && !a.reduced) return launch_arnoldi<float, float, false, kDynUnitSpeed>(a, k);
    if (a.dyn == kDynOrbit) {
        if (a.reduced) return launch_arnoldi<float, float, true, kDynOrbit>(a, k);
        return launch_arnoldi<float, float, false, kDynOrbit>(a, k);
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_arnoldi(const GmArgs<double, double>& a, int k)
{
    if (a.dyn == kDynUnitSpeed && !a.reduced) return launch_arnoldi<double, double, false, kDynUnitSpeed>(a, k);
    if (a.dyn == kDynPolar && !a.reduced) return launch_arnoldi<double, double, false, kDynPolar>(a, k);
    if (a.dyn == kDynOrbit) {
        if (a.reduced) return launch_arnoldi<double, double, true, kDynOrbit>(a, k);
        return launch_arnoldi<double, double, false, kDynOrbit>(a, k);
    }
    return cudaErrorInvalidValue;
}

template <typename G, typename VT, typename VV>
cudaError_t cycle(const GmArgs<G, VT>& a, const VV* Vin, VV* Vnext)
{
    if (a.m < 1 || a.m > kGmMaxRestart || !a.Q || !a.partial || !a.gctl) return cudaErrorInvalidValue;
    if (std::is_same<G, float>::value && !a.feet_lo) return cudaErrorInvalidValue;
    const int n = a.g.n_nodes;
    cudaError_t e;
    {
        auto kern = gm_start_kernel<VV, VT>;
        static int per_sm = 0;
        const int b = tiled_blocks(kern, n, a.sm_count, a.max_blocks, per_sm);
        kern<<<b, kGmBlock, 0, a.stream>>>(Vin, Vnext, a.Q, n, a.partial, a.gctl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int k = 0; k < a.m; ++k) {
        if ((e = dispatch_arnoldi(a, k)) != cudaSuccess) return e;
        if ((e = launch_update<VT, false, true>(a, n, k)) != cudaSuccess) return e;      // projections
        if (a.reorth && (e = launch_update<VT, true, true>(a, n, k)) != cudaSuccess) return e;
        if ((e = launch_update<VT, true, false>(a, n, k)) != cudaSuccess) return e;      // update + norm
    }
    auto kern = gm_apply_kernel<VV, VT>;
    static int per_sm = 0;
    const int b = tiled_blocks(kern, n, a.sm_count, a.max_blocks, per_sm);
    kern<<<b, kGmBlock, 0, a.stream>>>(Vin, Vnext, a.Q, a.ldq, n, a.gctl, a.ctl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gm_cycle(const GmArgs<float, float>& a, const float* Vin, float* Vnext) { return cycle(a, Vin, Vnext); }
cudaError_t gm_cycle(const GmArgs<float, float>& a, const double* Vin, double* Vnext) { return cycle(a, Vin, Vnext); }
cudaError_t gm_cycle(const GmArgs<double, double>& a, const double* Vin, double* Vnext)
{
    return cycle(a, Vin, Vnext);
}

cudaError_t launch_feet(const Geo<float>& g, const uint16_t* code, unsigned long long* feet_lo, unsigned* feet_hi,
                        int dyn, int reduced, int sm_count, cudaStream_t st)
{
    const long long need = ((long long)g.n_nodes + kGmBlock - 1) / kGmBlock;
    const int blocks = (int)(need < 8LL * sm_count ? need : 8LL * sm_count);
    if (blocks < 1) return cudaSuccess;
    if (dyn == kDynUnitSpeed && !reduced)
        feet_kernel<false, kDynUnitSpeed><<<blocks, kGmBlock, 0, st>>>(g, code, feet_lo, feet_hi);
    else if (dyn == kDynOrbit && reduced)
        feet_kernel<true, kDynOrbit><<<blocks, kGmBlock, 0, st>>>(g, code, feet_lo, feet_hi);
    else if (dyn == kDynOrbit)
        feet_kernel<false, kDynOrbit><<<blocks, kGmBlock, 0, st>>>(g, code, feet_lo, feet_hi);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace dpk
