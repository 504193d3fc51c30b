// dp_mlp.cu -- the learned warm start: a 4 -> 256 -> 256 -> 256 -> 3 BF16 MLP
// (exact-erf GELU, FP32 accumulation) trained on the GPU on (state, V / M,
// cos alpha*, sin alpha*) samples of a solved grid, then evaluated on every
// node of another grid to initialise V and the policy of policy iteration.
// Not part of the paper: the network only supplies the starting point, and
// the Bellman sweeps alone decide the result.
//
// The two 256 x 256 layers (98.6 % of the FLOPs) run on the fifth-generation
// tensor cores: tcgen05.mma kind::f16, BF16 operands staged in shared memory,
// FP32 accumulators in TMEM, fused epilogues (bias + GELU forward, GELU'
// backward, split-K atomic accumulation for weight gradients).  The 4-wide
// input layer, the 3-wide output layer, the reductions and Adam run on the
// CUDA cores.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "dp.h"
#include "dp_host.h"
#include "dp_umma.cuh"

namespace dpk {
int record_error(int code, const char* msg);

// View of a grid's resident state (defined in dp_api.cu).
struct GridView {
    Geo<double> g64;
    int fp32;
    const void* V;       // storage precision (FP32 or FP64), compact order
    double* V64;         // FP64 value when the grid holds one (else NULL)
    uint16_t* code;
    long long n;
    double M;
    double lo[4], hi[4];
    cudaStream_t st;
    const double2* tab_hi64;
    const double2* tab_lo64;
};
int grid_view(dp_grid* g, GridView* v);
void grid_after_warm_start(dp_grid* g);
}  // namespace dpk

using namespace dpk;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int kH = 256;                       // hidden width
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * 4, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + 3 * kH;
constexpr int kParams = kOffB4 + 3;           // 133,635
constexpr int kTileM = 128, kTileN = 128, kKC = 256;
// Shared memory of a K slice of A and B: 128 KB for a whole 256-wide slice
// (one CTA per SM; small batches: every slice at once), 64 KB for 128-wide
// slices (three CTAs per SM overlap one another's loads and epilogues).
constexpr int gemm_smem(int kc) { return (kTileM + kTileN) * kc * 2; }
// MN-major operands (kEpiSplitMN) get 32 KB more: the MMAs of a 256-wide
// slice then read inside the allocation for either assignment of its
// descriptors' two byte offsets (2048 along K, 128 along MN), at most
// 92,416 bytes past an operand's start.
constexpr int kMNPad = 32768;
template <int EPI, int KC>
constexpr int gemm_smem_of() { return gemm_smem(KC) + (EPI == 3 /* kEpiSplitMN */ ? kMNPad : 0); }
constexpr int kWaitPolls = 1 << 22;
constexpr float kInvSqrt2 = 0.70710678118654752f, kInvSqrt2Pi = 0.39894228040143268f;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * kInvSqrt2)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * kInvSqrt2)) + z * kInvSqrt2Pi * expf(-0.5f * z * z);
}

// 8 consecutive BF16 values (one 16-byte load) as floats.
__device__ __forceinline__ void load_row8(const bf16* p, float a[8])
{
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&u[q]);
        a[2 * q] = __low2float(h2);
        a[2 * q + 1] = __high2float(h2);
    }
}

enum { kEpiFwd = 0, kEpiBwd = 1, kEpiAtomic = 2, kEpiSplitMN = 3 };

// Four doubles by value (the network's input box corners).
struct Box4 {
    double x, y, z, w;
};

// 16-byte asynchronous copy global -> shared (both 16-byte aligned), and the
// wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// C[128 x 128 tile] = A[rows, K range] * B[256, K range]^T on tcgen05.
//   A: bf16 [*, lda] row-major (K contiguous); B: bf16 [256, ldb] row-major.
//   Tile rows start at 128 blockIdx.x, columns at 128 blockIdx.y; K range
//   [k_per_cta blockIdx.z, +k_per_cta), staged 256 at a time: every thread
//   issues its 16-byte asynchronous copies of the whole slice at once, then
//   one thread issues the 16 MMAs (K = 16 each) and commits them to an
//   mbarrier.
//   kEpiFwd:    z = acc + bias -> zout (optional, FP32), h = GELU(z) -> hout (bf16)
//   kEpiBwd:    dz = acc * GELU'(zin) -> hout (bf16)
//   kEpiAtomic: cacc += acc (FP32, split-K weight gradients)
//   kEpiSplitMN: both operands MN-major, A[K range, 128 blockIdx.x + i] and
//     B[K range, 128 blockIdx.y + j] row-major with the tile's rows / columns
//     contiguous (a weight gradient dz^T h straight from the activations, no
//     transposed copies); the tile is stored, not added, at split blockIdx.z
//     of cacc (256 x 256 floats per split), for a reduction in a fixed
//     order.  Core matrix (K block kb,
//     MN block mb) holds 8 K-rows of 8 contiguous MN elements at byte
//     (kb * 16 + mb) * 128: 128 bytes to the next MN block, 2048 to the next
//     K block.
template <int EPI, int KC>
__global__ void __launch_bounds__(128)
mlp_gemm_kernel(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B, int ldb, int k_per_cta,
                const float* __restrict__ bias, float* __restrict__ zout, const float* __restrict__ zin,
                bf16* __restrict__ hout, float* __restrict__ cacc, int* __restrict__ err, int polls)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                        // 128 x KC bf16
    unsigned char* sB = smem + kTileM * KC * 2;      // 128 x KC bf16
    __shared__ unsigned tmem_slot;
    __shared__ __align__(8) unsigned long long mbar;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(&tmem_slot, kTileN);
    if (tid == 0) mbar_init(&mbar);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const unsigned tmem = tmem_slot;
    const size_t row0 = (size_t)blockIdx.x * kTileM;
    const int n0 = blockIdx.y * kTileN;
    const int kbeg = blockIdx.z * k_per_cta;
    constexpr bool kMN = EPI == kEpiSplitMN;
    constexpr unsigned idesc = umma_idesc_bf16(kTileM, kTileN) | (kMN ? (1u << 15) | (1u << 16) : 0u);
    constexpr int kGroups = KC / 8;                  // 16-byte groups per row of a slice

    int phase = 0;
    bool ok = true;
    for (int k0 = kbeg; k0 < kbeg + k_per_cta; k0 += KC) {
        // core-matrix staging: (row, kb) -> ((row / 8) * kGroups + kb) * 128 + (row % 8) * 16.
        // A warp takes 8 rows x 4 consecutive 16-byte groups: 64 contiguous bytes
        // of each row in global memory, 512 contiguous bytes (no bank conflict)
        // in shared memory.
        // the 16-byte groups go straight to shared memory (cp.async): every
        // group of the slice is in flight at once, none through registers
        if constexpr (kMN) {
            // a warp takes 8 K-rows x 4 consecutive MN blocks: 64 contiguous
            // bytes of each row in global memory, 512 in shared memory
#pragma unroll
            for (int q = 0; q < kTileM * kGroups / 128; ++q) {
                const int v = tid + 128 * q, grp = v >> 5, ln = v & 31;
                const int kr = (grp >> 2) * 8 + (ln & 7), mb = (grp & 3) * 4 + (ln >> 3);
                cp_async16(sA + (size_t)v * 16, A + (size_t)(k0 + kr) * lda + row0 + mb * 8);
            }
#pragma unroll
            for (int q = 0; q < kTileN * kGroups / 128; ++q) {
                const int v = tid + 128 * q, grp = v >> 5, ln = v & 31;
                const int kr = (grp >> 2) * 8 + (ln & 7), mb = (grp & 3) * 4 + (ln >> 3);
                cp_async16(sB + (size_t)v * 16, B + (size_t)(k0 + kr) * ldb + n0 + mb * 8);
            }
        } else {
#pragma unroll
            for (int q = 0; q < kTileM * kGroups / 128; ++q) {
                const int v = tid + 128 * q, grp = v >> 5, ln = v & 31;
                const int row = (grp / (kGroups / 4)) * 8 + (ln & 7), kb = (grp % (kGroups / 4)) * 4 + (ln >> 3);
                cp_async16(sA + (size_t)v * 16, A + (row0 + row) * (size_t)lda + k0 + kb * 8);
            }
#pragma unroll
            for (int q = 0; q < kTileN * kGroups / 128; ++q) {
                const int v = tid + 128 * q, grp = v >> 5, ln = v & 31;
                const int row = (grp / (kGroups / 4)) * 8 + (ln & 7), kb = (grp % (kGroups / 4)) * 4 + (ln >> 3);
                cp_async16(sB + (size_t)v * 16, B + (size_t)(n0 + row) * ldb + k0 + kb * 8);
            }
        }
        cp_async_wait_all();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int s = 0; s < KC / 16; ++s) {
                // K step s: two K blocks (K-major: 256 bytes on; MN-major: 4096)
                const unsigned long long ad =
                    kMN ? umma_desc(smem_u32(sA) + s * 4096, 2048, 128) : umma_desc(smem_u32(sA) + s * 256, 128, kGroups * 128);
                const unsigned long long bd =
                    kMN ? umma_desc(smem_u32(sB) + s * 4096, 2048, 128) : umma_desc(smem_u32(sB) + s * 256, 128, kGroups * 128);
                umma_bf16(tmem, ad, bd, idesc, (k0 > kbeg || s > 0) ? 1u : 0u);
            }
            umma_commit(&mbar);
        }
        if (!mbar_wait(&mbar, phase, polls)) {
            // give up (error flag), but let the committed MMAs finish before
            // the accumulator is freed and the staging buffers are released
            ok = false;
            if (lane == 0) atomicOr(err, 1);
            mbar_wait(&mbar, phase, kWaitPolls);
        }
        phase ^= 1;
        __syncthreads();
        if (!__syncthreads_and(ok)) break;
    }
    fence_after_sync();
    if (ok) {
        const size_t r = row0 + warp * 32 + lane;   // TMEM lane = tile row
        for (int c0 = 0; c0 < kTileN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + c0, v);
            const size_t off = r * kH + n0 + c0;     // 16 consecutive columns, 64-byte aligned
            if (EPI == kEpiAtomic) {
                // four 16-byte reductions (the row's 16 columns are 64-byte aligned)
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    atomicAdd(reinterpret_cast<float4*>(cacc + off + q), make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]));
                continue;
            }
            if (EPI == kEpiSplitMN) {
                float* dst = cacc + (size_t)blockIdx.z * kH * kH + off;
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4*>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                continue;
            }
            float z[16];
            if (EPI == kEpiFwd) {
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 b = *(const float4*)(bias + n0 + c0 + q);
                    z[q] = v[q] + b.x; z[q + 1] = v[q + 1] + b.y; z[q + 2] = v[q + 2] + b.z; z[q + 3] = v[q + 3] + b.w;
                    if (zout) *(float4*)(zout + off + q) = make_float4(z[q], z[q + 1], z[q + 2], z[q + 3]);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) z[q] = gelu(z[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 zi = *(const float4*)(zin + off + q);
                    z[q] = v[q] * gelu_grad(zi.x); z[q + 1] = v[q + 1] * gelu_grad(zi.y);
                    z[q + 2] = v[q + 2] * gelu_grad(zi.z); z[q + 3] = v[q + 3] * gelu_grad(zi.w);
                }
            }
            unsigned pk[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(z[2 * q], z[2 * q + 1]);
                pk[q] = *(const unsigned*)&h2;
            }
            *(uint4*)(hout + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *(uint4*)(hout + off + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTileN);
}

// GEMM of a large batch (inference over a grid, and the training steps'
// hidden layers), persistent: each CTA takes one 128-column half of the
// layer (its 128 x 256 slice of the weights stays in shared memory, 64 KB)
// and walks row tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The next
// tile's 128 x 256 activations are copied (cp.async) into the second of two
// 64 KB buffers while the MMAs and the epilogue of the current tile run.
// Same staging layout, MMAs and epilogue arithmetic as mlp_gemm_kernel<EPI>
// (kEpiFwd with optional zout, or kEpiBwd).
// Thirty-two warps: eight per quarter of the TMEM lanes, each taking 16 of
// the tile's 128 columns in the epilogue (with 16 warps of 32 columns each,
// fewer warps hide the activation's latency: about 1 % slower training and 2 %
// slower inference).
constexpr int kPersistSmem = (kTileN + 2 * kTileM) * kKC * 2;   // 192 KB
constexpr int kPersistThreads = 1024;
constexpr int kPersistParts = kPersistThreads / 128;            // column parts per TMEM lane quarter

// RED (backward only) adds the sums over each row tile that the next
// gradients need, so that no separate pass re-reads dz: RED = 1 the column
// sums of dz (a bias gradient), RED = 5 also the sums of dz times each of the
// four inputs xin (rows x 4, the first layer's weight gradient), both from
// the FP32 values before dz is rounded to BF16.  Tile t's sums go to
// red[t * RED * 256 ..]: for RED = 5 the 4 x 256 weight-gradient entries
// (feature-major) then the 256 bias-gradient entries, the layout of W1, b1
// in the parameter vector.  Each lane sums its rows in order, a fixed
// shuffle tree combines the lanes of a warp, the CTA adds its four row
// quarters in order, and the tiles are summed afterwards in a fixed order.
template <int EPI, int RED = 0>
__global__ void __launch_bounds__(kPersistThreads)
mlp_persistent_kernel(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B, int ldb, int tiles,
                      const float* __restrict__ bias, float* __restrict__ zout, const float* __restrict__ zin,
                      bf16* __restrict__ hout, const float* __restrict__ xin, float* __restrict__ red,
                      int* __restrict__ err, int polls)
{
    static_assert(RED == 0 || (EPI == kEpiBwd && (RED == 1 || RED == 5)), "tile sums of the backward pass");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem;                                  // 128 x 256
    unsigned char* sA[2] = {smem + kTileN * kKC * 2, smem + (kTileN + kTileM) * kKC * 2};
    __shared__ unsigned tmem_slot;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ float sBias[kTileN];                              // this CTA's 128 biases
    __shared__ float sRed[4][RED > 0 ? RED * kTileN : 1];        // per row quarter: the tile sums
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * kTileN;
    if (EPI == kEpiFwd && tid < kTileN) sBias[tid] = bias[n0 + tid];
    if (warp == 0) tmem_alloc(&tmem_slot, kTileN);
    if (tid == 0) mbar_init(&mbar);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const unsigned tmem = tmem_slot;
    constexpr unsigned idesc = umma_idesc_bf16(kTileM, kTileN);
    constexpr int kGroups = kKC / 8;

    // (row, kb) -> ((row / 8) * kGroups + kb) * 128 + (row % 8) * 16, a warp
    // taking 8 rows x 4 consecutive 16-byte groups
    auto stage = [&](unsigned char* dst, const bf16* src, size_t ld, size_t r0) {
#pragma unroll 4
        for (int q = 0; q < kTileM * kGroups / kPersistThreads; ++q) {
            const int v = tid + kPersistThreads * q, grp = v >> 5, ln = v & 31;
            const int row = (grp / (kGroups / 4)) * 8 + (ln & 7), kb = (grp % (kGroups / 4)) * 4 + (ln >> 3);
            cp_async16(dst + (size_t)v * 16, src + (r0 + row) * ld + kb * 8);
        }
    };
    stage(sB, B, (size_t)ldb, (size_t)n0);
    int t = blockIdx.x;
    if (t < tiles) stage(sA[0], A, (size_t)lda, (size_t)t * kTileM);
    cp_async_wait_all();
    fence_async_smem();
    __syncthreads();

    int phase = 0, buf = 0;
    bool ok = true;
    for (; t < tiles; t += gridDim.x, buf ^= 1) {
        if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int s = 0; s < kKC / 16; ++s) {
                const unsigned long long ad = umma_desc(smem_u32(sA[buf]) + s * 256, 128, kGroups * 128);
                const unsigned long long bd = umma_desc(smem_u32(sB) + s * 256, 128, kGroups * 128);
                umma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
            }
            umma_commit(&mbar);
        }
        // the next tile's activations, into the other buffer (its last
        // reader, the previous tile's MMAs, has completed)
        const int tn = t + gridDim.x;
        if (tn < tiles) stage(sA[buf ^ 1], A, (size_t)lda, (size_t)tn * kTileM);
        if (!mbar_wait(&mbar, phase, polls)) {
            ok = false;
            if (lane == 0) atomicOr(err, 1);
            mbar_wait(&mbar, phase, kWaitPolls);   // the committed MMAs finish first
        }
        phase ^= 1;
        fence_after_sync();
        if (!__syncthreads_and(ok)) {
            cp_async_wait_all();   // no copy may outlive the CTA
            break;
        }
        // Each warp takes a 32-row x kCols-column block of the accumulator
        // (TMEM lane = tile row, so the load gives lane l row l).  The block
        // passes through shared memory -- the current tile's activation
        // buffer, whose last reader, the MMAs, has completed -- so that in
        // step k lane l holds row kRps k + l / kLpr and the four columns from
        // 4 (l % kLpr): the global loads and stores then cover whole row
        // segments instead of one 16-byte piece of 32 rows.  The 16-byte
        // chunks of a row are XOR-swizzled so that both passes are free of
        // bank conflicts.
        const int quarter = warp & 3, part = warp >> 2;
        constexpr int kCols = kTileN / kPersistParts;   // columns per warp: one TMEM load, one wait
        constexpr int kLpr = kCols / 4;                 // lanes per row (16-byte chunks of a row)
        constexpr int kRps = 32 / kLpr;                 // rows per step
        static_assert(kCols == 16 || kCols == 32, "one 16- or 32-column TMEM load per thread");
        static_assert(kPersistThreads / 32 * 32 * kCols * 4 <= kTileM * kKC * 2, "scratch fits the A buffer");
        const int c0 = part * kCols, rr = lane / kLpr, cc = lane % kLpr;
        float* S = (float*)sA[buf] + warp * 32 * kCols;
        const size_t g0 = ((size_t)t * kTileM + quarter * 32 + rr) * kH + n0 + c0 + 4 * cc;
        auto goff = [&](int k) { return g0 + (size_t)(kRps * k) * kH; };
        auto sw = [](int row, int c) { return row * kCols + ((c ^ ((row / (8 / kLpr)) % kLpr)) << 2); };
        float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f}, cw[4][4] = {};   // RED: column sums, times x
        float4 zi[kLpr];
        if (EPI == kEpiBwd) {
            // the pre-activations are loaded before the accumulator's wait
#pragma unroll
            for (int k = 0; k < kLpr; ++k) zi[k] = *(const float4*)(zin + goff(k));
        }
        {
            float v[kCols];
            const unsigned ta = tmem + ((unsigned)(quarter * 32) << 16) + c0;
            if constexpr (kCols == 32) tmem_ld32(ta, v);
            else tmem_ld16(ta, v);
#pragma unroll
            for (int c = 0; c < kLpr; ++c)
                *(float4*)(S + sw(lane, c)) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kLpr; ++k) {
            const float4 a = *(const float4*)(S + sw(kRps * k + rr, cc));
            float y[4];
            if (EPI == kEpiFwd) {
                const float4 z = make_float4(a.x + sBias[c0 + 4 * cc], a.y + sBias[c0 + 4 * cc + 1],
                                             a.z + sBias[c0 + 4 * cc + 2], a.w + sBias[c0 + 4 * cc + 3]);
                if (zout) *(float4*)(zout + goff(k)) = z;
                y[0] = gelu(z.x); y[1] = gelu(z.y); y[2] = gelu(z.z); y[3] = gelu(z.w);
            } else {
                y[0] = a.x * gelu_grad(zi[k].x); y[1] = a.y * gelu_grad(zi[k].y);
                y[2] = a.z * gelu_grad(zi[k].z); y[3] = a.w * gelu_grad(zi[k].w);
                if (RED > 0) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) cs[i] += y[i];
                }
                if (RED == 5) {
                    const float4 xk = *(const float4*)(xin + 4 * ((size_t)t * kTileM + quarter * 32 + kRps * k + rr));
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        cw[i][0] += y[i] * xk.x; cw[i][1] += y[i] * xk.y;
                        cw[i][2] += y[i] * xk.z; cw[i][3] += y[i] * xk.w;
                    }
                }
            }
            if (RED != 5) {
                const __nv_bfloat162 p0 = __floats2bfloat162_rn(y[0], y[1]), p1 = __floats2bfloat162_rn(y[2], y[3]);
                *(uint2*)(hout + goff(k)) = make_uint2(*(const unsigned*)&p0, *(const unsigned*)&p1);
            }
        }
        if (RED > 0) {
            // lanes with the same columns (equal lane % kLpr) hold the other rows
#pragma unroll
            for (int o = kLpr; o < 32; o <<= 1) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    cs[i] += __shfl_xor_sync(0xffffffffu, cs[i], o);
                    if (RED == 5) {
#pragma unroll
                        for (int d = 0; d < 4; ++d) cw[i][d] += __shfl_xor_sync(0xffffffffu, cw[i][d], o);
                    }
                }
            }
            if (rr == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int col = c0 + 4 * cc + i;
                    if (RED == 5) {
#pragma unroll
                        for (int d = 0; d < 4; ++d) sRed[quarter][col * 4 + d] = cw[i][d];
                        sRed[quarter][4 * kTileN + col] = cs[i];
                    } else {
                        sRed[quarter][col] = cs[i];
                    }
                }
            }
        }
        // the epilogue's TMEM reads finish before the next tile's MMAs
        // overwrite the accumulator; the next activations must have landed
        cp_async_wait_all();
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (RED > 0) {
            // the four row quarters in order (read before the next tile's
            // epilogue, which follows the next block-wide barrier, writes sRed)
            float* rt = red + (size_t)t * (RED * kH);
            for (int i = tid; i < RED * kTileN; i += kPersistThreads) {
                const float v = ((sRed[0][i] + sRed[1][i]) + sRed[2][i]) + sRed[3][i];
                const size_t gi = RED == 5 ? (i < 4 * kTileN ? (size_t)n0 * 4 + i : (size_t)4 * kH + n0 + (i - 4 * kTileN))
                                           : (size_t)n0 + i;
                rt[gi] = v;
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTileN);
}

// Inputs (normalised to [-1, 1]^4) and targets (V / M, cos, sin) of nodes
// idx = (mult * (start + i) + offset) mod n of a grid (a seeded permutation).
// Without V only the inputs are written.  Inputs are normalised to the
// network's box (nlo, nhi).
// Training-step state in device memory, so that one captured step can be
// replayed: the epoch's permutation (mult, offset), the first sample of the
// step, and the Adam step count.
struct TrainState {
    long long mult, offset, start;
    int t;
    float lr;        // > 0: the epoch's Adam step size (replaces the kernel argument)
};

template <typename S>
__global__ void batch_from_grid_kernel(Geo<double> g, const S* __restrict__ V, const uint16_t* __restrict__ code,
                                       const double2* __restrict__ thi, const double2* __restrict__ tlo,
                                       long long n, long long mult, long long offset, long long start, int count,
                                       double invM, Box4 nlo, Box4 nhi, float* __restrict__ x,
                                       float* __restrict__ t, const TrainState* __restrict__ ts = nullptr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (ts) {
        mult = ts->mult;
        offset = ts->offset;
        start = ts->start;
    }
    const long long j = (long long)(((unsigned long long)mult * (unsigned long long)(start + i) +
                                     (unsigned long long)offset) % (unsigned long long)n);
    int id[4];
    decode_node(g, (int)j, id);
    const double lo[4] = {nlo.x, nlo.y, nlo.z, nlo.w}, hi[4] = {nhi.x, nhi.y, nhi.z, nhi.w};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const double xd = g.lo[d] + (double)id[d] * g.h[d];
        x[4 * i + d] = (float)(2.0 * (xd - lo[d]) / (hi[d] - lo[d]) - 1.0);
    }
    if (!V) return;
    const int c = code[j];
    const double2 a = thi[c >> 8], b = tlo[c & 255];
    t[3 * i + 0] = (float)((double)V[j] * invM);
    t[3 * i + 1] = (float)(a.y * b.y - a.x * b.x);   // cos
    t[3 * i + 2] = (float)(a.x * b.y + a.y * b.x);   // sin
}

// Arbitrary states (device, n x 4 double) normalised to [-1, 1]^4.
__global__ void states_in_kernel(const double* __restrict__ s, int count, Box4 lo, Box4 hi,
                                 float* __restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    x[4 * i + 0] = (float)(2.0 * (s[4 * i + 0] - lo.x) / (hi.x - lo.x) - 1.0);
    x[4 * i + 1] = (float)(2.0 * (s[4 * i + 1] - lo.y) / (hi.y - lo.y) - 1.0);
    x[4 * i + 2] = (float)(2.0 * (s[4 * i + 2] - lo.z) / (hi.z - lo.z) - 1.0);
    x[4 * i + 3] = (float)(2.0 * (s[4 * i + 3] - lo.w) / (hi.w - lo.w) - 1.0);
}

// Layer 1 (4 -> 256) with GELU: 32 threads per sample, thread `lane` takes
// the features lane + 32 q (conflict-free reads of the transposed W1 in shared
// memory, each warp store 64 contiguous bytes).  Rows >= count are zero.
__global__ void l1_fwd_kernel(const float* __restrict__ x, const float* __restrict__ P, int count, int rows,
                              float* __restrict__ z1, bf16* __restrict__ h1)
{
    __shared__ float sWt[4 * kH + kH];   // W1 transposed (4 x 256), then b1
    for (int i = threadIdx.x; i < 4 * kH; i += blockDim.x) sWt[(i & 3) * kH + (i >> 2)] = P[kOffW1 + i];
    for (int i = threadIdx.x; i < kH; i += blockDim.x) sWt[4 * kH + i] = P[kOffB1 + i];
    __syncthreads();
    const long long total = (long long)rows * 32;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e >> 5), lane = (int)(e & 31);
        float4 xs = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (s < count) xs = *reinterpret_cast<const float4*>(x + 4 * (size_t)s);
#pragma unroll
        for (int q = 0; q < kH / 32; ++q) {
            const int o = lane + 32 * q;
            const float z = s < count ? sWt[4 * kH + o] + sWt[o] * xs.x + sWt[kH + o] * xs.y +
                                            sWt[2 * kH + o] * xs.z + sWt[3 * kH + o] * xs.w
                                      : 0.0f;
            h1[(size_t)s * kH + o] = __float2bfloat16(s < count ? gelu(z) : 0.0f);
            if (z1) z1[(size_t)s * kH + o] = z;
        }
    }
}

// Output layer (256 -> 3): one warp per sample, each lane 8 consecutive
// features (one 16-byte load), the three sums reduced across the warp.
__global__ void out_kernel(const bf16* __restrict__ h3, const float* __restrict__ P, int count,
                           float* __restrict__ y)
{
    __shared__ float sW[3 * kH + 3];
    for (int i = threadIdx.x; i < 3 * kH + 3; i += blockDim.x) sW[i] = P[kOffW4 + i];   // W4 then b4
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int s = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (s >= count) return;
    float a[8];
    load_row8(h3 + (size_t)s * kH + lane * 8, a);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) sum += sW[k * kH + lane * 8 + q] * a[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) y[3 * (size_t)s + k] = sum + sW[3 * kH + k];
    }
}

// The output layer of a training step with the first part of its backward
// pass, one warp per sample (grid-stride over the samples): y = W4 h3 + b4,
// the loss gradient dy = 2 (y - t) / (3 B), the loss sum, the output layer's
// gradients dW4 = dy h3^T and db4 = sum dy, and dz3 = (dy W4) * GELU'(z3) for
// the lane's 8 features with its sum db3 (FP32, before the BF16 rounding of
// dz3).  Each lane sums its samples in order, the block sums its warps in
// order, and the block's sums go to part[blockIdx.x] for a reduction in a
// fixed order: db3, dW4, db4 (laid out as b3, W4, b4 are in the parameter
// vector), then the loss.
constexpr int kOutPart = 4 * kH + 4;
__global__ void __launch_bounds__(256) out_train_kernel(const bf16* __restrict__ h3, const float* __restrict__ P,
                                                        const float* __restrict__ t, const float* __restrict__ z3,
                                                        int count, float inv_n, bf16* __restrict__ dz3,
                                                        float* __restrict__ part)
{
    __shared__ float sW[3 * kH + 3];
    __shared__ float sP[8][kOutPart];   // per warp: db3, dW4, db4, loss
    for (int i = threadIdx.x; i < 3 * kH + 3; i += blockDim.x) sW[i] = P[kOffW4 + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warps = (int)((gridDim.x * (size_t)blockDim.x) >> 5);
    float w[3][8] = {}, b[3] = {}, d3[8] = {}, l = 0.0f;
    for (int s = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5); s < count; s += warps) {
        float a[8];
        load_row8(h3 + (size_t)s * kH + lane * 8, a);
        float dy[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float sum = 0.0f;
#pragma unroll
            for (int q = 0; q < 8; ++q) sum += sW[k * kH + lane * 8 + q] * a[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            const float r = (sum + sW[3 * kH + k]) - t[3 * (size_t)s + k];
            l += r * r;
            dy[k] = 2.0f * r * inv_n;
            b[k] += dy[k];
#pragma unroll
            for (int q = 0; q < 8; ++q) w[k][q] += dy[k] * a[q];
        }
        const float4* zp = reinterpret_cast<const float4*>(z3 + (size_t)s * kH + lane * 8);
        const float4 z0 = zp[0], z1 = zp[1];
        const float z[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
        unsigned u[4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const int i = lane * 8 + q;
            const float g0 = dy[0] * sW[i] + dy[1] * sW[kH + i] + dy[2] * sW[2 * kH + i];
            const float g1 = dy[0] * sW[i + 1] + dy[1] * sW[kH + i + 1] + dy[2] * sW[2 * kH + i + 1];
            const float e0 = g0 * gelu_grad(z[q]), e1 = g1 * gelu_grad(z[q + 1]);
            d3[q] += e0;
            d3[q + 1] += e1;
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(e0, e1);
            u[q / 2] = *reinterpret_cast<const unsigned*>(&h2);
        }
        *reinterpret_cast<uint4*>(dz3 + (size_t)s * kH + lane * 8) = make_uint4(u[0], u[1], u[2], u[3]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) sP[warp][lane * 8 + q] = d3[q];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int q = 0; q < 8; ++q) sP[warp][kH + k * kH + lane * 8 + q] = w[k][q];
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) sP[warp][4 * kH + k] = b[k];
        sP[warp][4 * kH + 3] = l;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOutPart; i += blockDim.x) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += sP[k][i];
        part[(size_t)blockIdx.x * kOutPart + i] = acc;
    }
}

// Fixed-order reductions of per-block partial sums: out[i] (+)= sum over k
// of part[k * stride + i], i < len (accumulate: add to out instead of
// storing).  Long outputs take a thread per output, which sums k in order;
// short outputs with many partials a warp per output, lane l summing
// partials l, l + 32, ... in order before a fixed shuffle tree combines the
// lanes.  Two such reductions run in one launch: blocks [0, a.blocks) take
// segment a, the rest segment b (b.blocks = 0: none).
struct RedSeg {
    const float* part;
    int n_part, stride, len;
    float* out;
    int accumulate;
    int warp;     // 1: a warp per output (8 per block), 0: a thread per output
    int blocks;
};

__global__ void sum_segments_kernel(RedSeg a, RedSeg b)
{
    const bool first = (int)blockIdx.x < a.blocks;
    const RedSeg& r = first ? a : b;
    const int blk = first ? (int)blockIdx.x : (int)blockIdx.x - a.blocks;
    if (r.warp) {
        const int i = (int)((blk * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
        if (i >= r.len) return;
        float acc = 0.0f;
        for (int k = lane; k < r.n_part; k += 32) acc += r.part[(size_t)k * r.stride + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) r.out[i] = r.accumulate ? r.out[i] + acc : acc;
    } else {
        const int i = blk * blockDim.x + threadIdx.x;
        if (i >= r.len) return;
        float acc = 0.0f;
        for (int k = 0; k < r.n_part; ++k) acc += r.part[(size_t)k * r.stride + i];
        r.out[i] = r.accumulate ? r.out[i] + acc : acc;
    }
}

// Per-feature reductions over a chunk of samples (thread = feature), for
// batches below kManyRows rows (larger ones are summed per tile in the
// persistent backward GEMM's epilogue), in
// sample order:  db[o] = sum_s dz[s][o];  with X = 4 also
// dW[o][d] = sum_s dz[s][o] x[s][d].  Block b writes its sums to
// part[b][0 .. 4 X + ... ): dW (256 X values, feature-major) then db (256),
// for a reduction in a fixed order.  X (0 or 4) is a template argument so
// that the accumulators stay in registers; the inputs x of each 256-sample
// slice of the chunk are staged in shared memory.
template <int X>
__global__ void feat_reduce_kernel(const bf16* __restrict__ dz, const float* __restrict__ x, int rows, int chunk,
                                   float* __restrict__ part)
{
    __shared__ float4 sx[X == 4 ? 256 : 1];
    const int o = threadIdx.x;   // 256 threads
    const int s0 = blockIdx.x * chunk, s1 = min(rows, s0 + chunk);
    float b = 0.0f, w[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int sb = s0; sb < s1; sb += 256) {
        const int se = min(s1, sb + 256);
        if constexpr (X == 4) {
            __syncthreads();
            if (sb + o < se) sx[o] = reinterpret_cast<const float4*>(x)[sb + o];
            __syncthreads();
        }
#pragma unroll 8
        for (int s = sb; s < se; ++s) {
            const float g = __bfloat162float(dz[(size_t)s * kH + o]);
            b += g;
            if constexpr (X == 4) {
                const float4 xs = sx[s - sb];
                w[0] += g * xs.x;
                w[1] += g * xs.y;
                w[2] += g * xs.z;
                w[3] += g * xs.w;
            }
        }
    }
    float* pb = part + (size_t)blockIdx.x * (kH * X + kH);
    if constexpr (X == 4) {
#pragma unroll
        for (int d = 0; d < 4; ++d) pb[o * 4 + d] = w[d];
    }
    pb[kH * X + o] = b;
}

// Adam on the FP32 master parameters, writing the BF16 copies of W2, W3 and
// their transposes used by the tensor-core GEMMs as it goes.
// The step count t (1 for the first step) comes from device memory; the
// bias corrections are 1 - beta^t.  advance > 0 (a replayed training step):
// the last block to finish moves the step on -- the next step's first
// sample start += advance and t += 1 -- once every block has read t and the
// step size; *arrive counts the finished blocks and is back at 0 afterwards.
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                            TrainState* __restrict__ ts, bf16* __restrict__ W2, bf16* __restrict__ W3,
                            bf16* __restrict__ W2T, bf16* __restrict__ W3T, unsigned* __restrict__ arrive,
                            int advance)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float tf = (float)ts->t;
        if (ts->lr > 0.0f) lr = ts->lr;
        const float bc1 = 1.0f - powf(b1, tf), bc2 = 1.0f - powf(b2, tf);
        const float g = G[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float p = P[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        P[i] = p;
        const bool w2 = i >= kOffW2 && i < kOffW2 + kH * kH, w3 = i >= kOffW3 && i < kOffW3 + kH * kH;
        if (w2 || w3) {
            const int e = i - (w2 ? kOffW2 : kOffW3), o = e / kH, c = e % kH;
            (w2 ? W2 : W3)[e] = __float2bfloat16(p);
            (w2 ? W2T : W3T)[c * kH + o] = __float2bfloat16(p);
        }
    }
    if (advance > 0) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(arrive, 1u) == gridDim.x - 1) {
                ts->start += advance;
                ts->t += 1;
                *arrive = 0u;
            }
        }
    }
}

// Sets the Adam step count (eager steps outside a replayed graph).
__global__ void set_step_kernel(TrainState* ts, int t)
{
    ts->t = t;
    ts->lr = 0.0f;   // the step size of the call
}

__global__ void bf16_weights_kernel(const float* __restrict__ P, bf16* __restrict__ W2, bf16* __restrict__ W3,
                                    bf16* __restrict__ W2T, bf16* __restrict__ W3T)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // kH * kH threads
    if (e >= kH * kH) return;
    const int o = e / kH, i = e % kH;
    W2[e] = __float2bfloat16(P[kOffW2 + e]);
    W3[e] = __float2bfloat16(P[kOffW3 + e]);
    W2T[i * kH + o] = __float2bfloat16(P[kOffW2 + e]);
    W3T[i * kH + o] = __float2bfloat16(P[kOffW3 + e]);
}

// Warm start: V = M clamp(V/M-hat, 0, 1) (target nodes 0) and the code of
// atan2(sin-hat, cos-hat), for compact nodes [start, start + count).
template <typename S>
__global__ void warm_write_kernel(Geo<double> g, const float* __restrict__ y, long long start, int count, double M,
                                  S* __restrict__ V, uint16_t* __restrict__ code)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const long long j = start + i;
    int id[4];
    decode_node(g, (int)j, id);
    const double v = fmin(fmax((double)y[3 * i], 0.0), 1.0) * M;
    V[j] = in_target(g, id) ? (S)0 : (S)v;
    const double a = atan2((double)y[3 * i + 2], (double)y[3 * i + 1]);   // (-pi, pi]
    long long c = llrint(a * (65536.0 / 6.283185307179586476925286766559));
    code[j] = (uint16_t)(c & 65535);
}

int fail_cuda(const char* what, cudaError_t e)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return record_error(DP_ECUDA, buf);
}

#define MCK(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return fail_cuda(#call, e_);       \
    } while (0)

}  // namespace

struct dp_mlp {
    int device = 0;
    int sm_count = 1;
    cudaStream_t st = nullptr;
    int cap = 0;                       // activation rows (multiple of 512)
    double lo[4], hi[4];               // input box (normalisation)
    long long step = 0;
    float *P = nullptr, *G = nullptr, *Am = nullptr, *Av = nullptr;
    bf16 *W2b = nullptr, *W3b = nullptr, *W2T = nullptr, *W3T = nullptr;
    float *x = nullptr, *t = nullptr, *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *y = nullptr;
    bf16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dz1 = nullptr, *dz2 = nullptr, *dz3 = nullptr;
    double* states = nullptr;
    float* loss = nullptr;
    float* part = nullptr;             // partial sums of the backward pass (kPartFloats)
    float* red = nullptr;              // per-row-tile sums of the fused backward GEMMs (cap / 128 x 5 x 256)
    unsigned* arrive = nullptr;        // blocks of the Adam kernel that have finished (0 between launches)
    int* err = nullptr;
    float* h_loss = nullptr;           // pinned
    int* h_err = nullptr;
    int wait_polls = kWaitPolls;       // polls of the first wait for the MMAs (test hook)
    TrainState* ts = nullptr;          // training-step state (device)
    TrainState* h_ts = nullptr;        // pinned staging of its per-epoch values
    cudaStream_t cst = nullptr;        // private stream: training steps are captured and replayed there
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

void free_mlp(dp_mlp* m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->st) cudaStreamSynchronize(m->st);
    void* ps[] = {m->P, m->G, m->Am, m->Av, m->W2b, m->W3b, m->W2T, m->W3T, m->x, m->t, m->z1, m->z2, m->z3, m->y,
                  m->h1, m->h2, m->h3, m->dz1, m->dz2, m->dz3, m->states, m->loss, m->part, m->red, m->arrive, m->err};
    for (void* p : ps)
        if (p) cudaFree(p);
    if (m->h_loss) cudaFreeHost(m->h_loss);
    if (m->h_err) cudaFreeHost(m->h_err);
    if (m->ts) cudaFree(m->ts);
    if (m->h_ts) cudaFreeHost(m->h_ts);
    if (m->ev_in) cudaEventDestroy(m->ev_in);
    if (m->ev_out) cudaEventDestroy(m->ev_out);
    if (m->cst) cudaStreamDestroy(m->cst);
    delete m;
}

template <typename T>
cudaError_t malloc_n(T** p, size_t n)
{
    return cudaMalloc((void**)p, n * sizeof(T));
}

int refresh_bf16(dp_mlp* m)
{
    bf16_weights_kernel<<<kH * kH / 256, 256, 0, m->st>>>(m->P, m->W2b, m->W3b, m->W2T, m->W3T);
    MCK(cudaGetLastError());
    return DP_OK;
}

// A kernel's dynamic shared-memory limit, raised once per device (function
// attributes hold per device, so a process that drives several GPUs raises
// it on each).
constexpr int kMaxDevices = 64;

template <typename K>
cudaError_t raise_smem_limit(K kernel, int bytes, std::atomic<bool> (&done)[kMaxDevices])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[dev].store(true, std::memory_order_release);
    return e;
}

template <int EPI, int KC>
cudaError_t gemm_kc(dp_mlp* m, const bf16* A, int lda, const bf16* B, int ldb, int rows, int k_total, int k_split,
                    const float* bias, float* zout, const float* zin, bf16* hout, float* cacc)
{
    static std::atomic<bool> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(mlp_gemm_kernel<EPI, KC>, gemm_smem_of<EPI, KC>(), attr);
    if (e != cudaSuccess) return e;
    dim3 grid(rows / kTileM, kH / kTileN, k_split);
    mlp_gemm_kernel<EPI, KC><<<grid, 128, gemm_smem_of<EPI, KC>(), m->st>>>(A, lda, B, ldb, k_total / k_split, bias, zout, zin,
                                                                   hout, cacc, m->err, m->wait_polls);
    return cudaGetLastError();
}

// Large batches (inference over a grid) stage K in 128-wide halves so that
// three CTAs share an SM; small ones (training) stage the whole 256-wide K
// slice at once; split-K weight gradients take one 256-wide slice per CTA.
constexpr int kManyRows = 16384;

// Partial sums of the backward pass (one buffer, reused by each reduction in
// turn): split-K tiles of a weight gradient, the output layer's per-block
// sums, and below kManyRows rows the feature reductions' per-block sums (the
// persistent backward GEMMs write their per-tile sums to dp_mlp::red
// instead).  Split-K 32 for the weight gradients (fewer splits serialise the
// K loop of each CTA, more write more partial tiles).
constexpr int kSplitMax = 32, kOutBlocks = 1024, kRedBlocks = 256;
constexpr size_t kPartFloats = (size_t)kSplitMax * kH * kH;   // >= kOutBlocks * kOutPart, kRedBlocks * 5 * kH

// The persistent kernel over rows (a multiple of 128, at least kManyRows) with
// K = 256; RED > 0 (backward): the per-tile sums into red.
template <int EPI, int RED = 0>
cudaError_t persistent(dp_mlp* m, const bf16* A, int lda, const bf16* B, int ldb, int rows, const float* bias,
                       float* zout, const float* zin, bf16* hout, const float* xin = nullptr, float* red = nullptr)
{
    static std::atomic<bool> attr[kMaxDevices];
    cudaError_t e = raise_smem_limit(mlp_persistent_kernel<EPI, RED>, kPersistSmem, attr);
    if (e != cudaSuccess) return e;
    const int tiles = rows / kTileM;
    const int per_half = std::max(1, std::min(tiles, m->sm_count / 2));
    dim3 grid(per_half, kH / kTileN);
    mlp_persistent_kernel<EPI, RED><<<grid, kPersistThreads, kPersistSmem, m->st>>>(
        A, lda, B, ldb, tiles, bias, zout, zin, hout, xin, red, m->err, m->wait_polls);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t gemm(dp_mlp* m, const bf16* A, int lda, const bf16* B, int ldb, int rows, int k_total, int k_split,
                 const float* bias, float* zout, const float* zin, bf16* hout, float* cacc)
{
    if constexpr (EPI == kEpiFwd || EPI == kEpiBwd) {
        if (rows >= kManyRows && k_total == kKC && k_split == 1)
            return persistent<EPI>(m, A, lda, B, ldb, rows, bias, zout, zin, hout);
    }
    if (EPI != kEpiAtomic && EPI != kEpiSplitMN && rows >= kManyRows)
        return gemm_kc<EPI, kKC / 2>(m, A, lda, B, ldb, rows, k_total, k_split, bias, zout, zin, hout, cacc);
    return gemm_kc<EPI, kKC>(m, A, lda, B, ldb, rows, k_total, k_split, bias, zout, zin, hout, cacc);
}

// Hidden layers of the forward pass of `count` rows held in m->x (rows
// padded to a multiple of 128), through h3.  save: keep z1..z3 for a
// backward pass.
int forward_hidden(dp_mlp* m, int count, bool save)
{
    const int rows = (count + kTileM - 1) / kTileM * kTileM;
    const long long e8 = (long long)rows * 32;
    const unsigned b1 = (unsigned)std::min<long long>((e8 + 255) / 256, 8LL * m->sm_count);
    l1_fwd_kernel<<<b1, 256, 0, m->st>>>(m->x, m->P, count, rows, save ? m->z1 : nullptr, m->h1);
    MCK(cudaGetLastError());
    MCK(gemm<kEpiFwd>(m, m->h1, kH, m->W2b, kH, rows, kH, 1, m->P + kOffB2, save ? m->z2 : nullptr, nullptr, m->h2,
                      nullptr));
    MCK(gemm<kEpiFwd>(m, m->h2, kH, m->W3b, kH, rows, kH, 1, m->P + kOffB3, save ? m->z3 : nullptr, nullptr, m->h3,
                      nullptr));
    return DP_OK;
}

// Forward of `count` rows into m->y.
int forward(dp_mlp* m, int count)
{
    int rc;
    if ((rc = forward_hidden(m, count, false))) return rc;
    out_kernel<<<(count + 7) / 8, 256, 0, m->st>>>(m->h3, m->P, count, m->y);
    MCK(cudaGetLastError());
    return DP_OK;
}

// Gradients of the mean squared error over a batch of `count` rows (count a
// multiple of 512; m->x / m->t hold the batch) into m->G, the loss sum added
// to m->loss.  The output layer and its backward pass run in one kernel.
int forward_backward(dp_mlp* m, int count, float inv_n)
{
    const int rows = count;
    int rc;
    if ((rc = forward_hidden(m, count, true))) return rc;
    // every gradient sum goes through per-block partial sums and a reduction
    // in a fixed order, so that a training run is reproducible bit for bit
    auto seg = [](const float* part, int n_part, int stride, int len, float* out, int accumulate) {
        RedSeg r{part, n_part, stride, len, out, accumulate, len <= 8192 ? 1 : 0, 0};   // short: a warp each
        r.blocks = r.warp ? (len + 7) / 8 : (len + 255) / 256;
        return r;
    };
    auto reduce2 = [&](const RedSeg& a, const RedSeg& b) {   // both in one launch
        sum_segments_kernel<<<a.blocks + b.blocks, 256, 0, m->st>>>(a, b);
        return cudaGetLastError();
    };
    auto reduce = [&](const float* part, int n_part, int stride, int len, float* out, int accumulate) {
        return reduce2(seg(part, n_part, stride, len, out, accumulate), RedSeg{});
    };
    const int ob = (int)std::min<long long>(std::min<long long>((count + 7) / 8, 2LL * m->sm_count), kOutBlocks);
    out_train_kernel<<<ob, 256, 0, m->st>>>(m->h3, m->P, m->t, m->z3, count, inv_n, m->dz3, m->part);
    MCK(cudaGetLastError());
    MCK(reduce2(seg(m->part, ob, kOutPart, 4 * kH + 3, m->G + kOffB3, 0),      // db3, dW4, db4
                seg(m->part + 4 * kH + 3, ob, kOutPart, 1, m->loss, 1)));       // the loss sum, accumulated
    // split-K of the weight-gradient GEMMs: a divisor of rows / 256, at most kSplitMax
    int ks = std::min(rows / kKC, kSplitMax);
    while ((rows / kKC) % ks) --ks;
    if (rows >= kManyRows) {
        // persistent backward GEMMs with the bias and first-layer gradients
        // summed per row tile in their epilogues (dz1 is never stored)
        const int tiles = rows / kTileM;
        // layer 3: dz2 = (dz3 W3) * GELU'(z2) with db2; dW3 = dz3^T h2
        MCK((persistent<kEpiBwd, 1>(m, m->dz3, kH, m->W3T, kH, rows, nullptr, nullptr, m->z2, m->dz2, nullptr,
                                    m->red)));
        MCK(gemm<kEpiSplitMN>(m, m->dz3, kH, m->h2, kH, kH, rows, ks, nullptr, nullptr, nullptr, nullptr, m->part));
        MCK(reduce2(seg(m->part, ks, kH * kH, kH * kH, m->G + kOffW3, 0), seg(m->red, tiles, kH, kH, m->G + kOffB2, 0)));
        // layer 2: dz1 = (dz2 W2) * GELU'(z1) summed into dW1 = dz1^T x and
        // db1; dW2 = dz2^T h1
        MCK((persistent<kEpiBwd, 5>(m, m->dz2, kH, m->W2T, kH, rows, nullptr, nullptr, m->z1, nullptr, m->x,
                                    m->red)));
        MCK(gemm<kEpiSplitMN>(m, m->dz2, kH, m->h1, kH, kH, rows, ks, nullptr, nullptr, nullptr, nullptr, m->part));
        MCK(reduce2(seg(m->part, ks, kH * kH, kH * kH, m->G + kOffW2, 0),
                    seg(m->red, tiles, 5 * kH, 5 * kH, m->G + kOffW1, 0)));
        return DP_OK;
    }
    // rows per block of the feature reductions: at most kRedBlocks blocks
    const int chunk = std::max(64, (rows + kRedBlocks - 1) / kRedBlocks);
    const int nb = (rows + chunk - 1) / chunk;
    // layer 3: dz2 = (dz3 W3) * GELU'(z2); dW3 = dz3^T h2
    MCK(gemm<kEpiBwd>(m, m->dz3, kH, m->W3T, kH, rows, kH, 1, nullptr, nullptr, m->z2, m->dz2, nullptr));
    MCK(gemm<kEpiSplitMN>(m, m->dz3, kH, m->h2, kH, kH, rows, ks, nullptr, nullptr, nullptr, nullptr, m->part));
    MCK(reduce(m->part, ks, kH * kH, kH * kH, m->G + kOffW3, 0));
    // layer 2: dz1 = (dz2 W2) * GELU'(z1); dW2 = dz2^T h1; db2 = sum dz2
    MCK(gemm<kEpiBwd>(m, m->dz2, kH, m->W2T, kH, rows, kH, 1, nullptr, nullptr, m->z1, m->dz1, nullptr));
    MCK(gemm<kEpiSplitMN>(m, m->dz2, kH, m->h1, kH, kH, rows, ks, nullptr, nullptr, nullptr, nullptr, m->part));
    MCK(reduce(m->part, ks, kH * kH, kH * kH, m->G + kOffW2, 0));
    feat_reduce_kernel<0><<<nb, 256, 0, m->st>>>(m->dz2, nullptr, rows, chunk, m->part);
    MCK(cudaGetLastError());
    MCK(reduce(m->part, nb, kH, kH, m->G + kOffB2, 0));
    // layer 1: dW1 = dz1^T x, db1 = sum dz1 (contiguous in G)
    feat_reduce_kernel<4><<<nb, 256, 0, m->st>>>(m->dz1, m->x, rows, chunk, m->part);
    MCK(cudaGetLastError());
    MCK(reduce(m->part, nb, kH * 4 + kH, kH * 4 + kH, m->G + kOffW1, 0));
    return DP_OK;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) with the gradient in m->G and the
// step count in m->ts, then the BF16 copies of the weights.
int adam_launch(dp_mlp* m, double lr, int advance = 0)
{
    adam_kernel<<<(kParams + 255) / 256, 256, 0, m->st>>>(m->P, m->G, m->Am, m->Av, kParams, (float)lr, 0.9f, 0.999f,
                                                          1e-8f, m->ts, m->W2b, m->W3b, m->W2T, m->W3T, m->arrive,
                                                          advance);
    MCK(cudaGetLastError());
    return DP_OK;
}

// One Adam step with the gradient in m->G (the next step count).
int adam_step(dp_mlp* m, double lr)
{
    ++m->step;
    set_step_kernel<<<1, 1, 0, m->st>>>(m->ts, (int)m->step);
    MCK(cudaGetLastError());
    return adam_launch(m, lr);
}

int check_err(dp_mlp* m)
{
    MCK(cudaMemcpyAsync(m->h_err, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    if (*m->h_err) {
        // the kernels that gave up drained their MMAs and freed their TMEM:
        // clear the flag so that the next call starts clean
        *m->h_err = 0;
        MCK(cudaMemsetAsync(m->err, 0, sizeof(int), m->st));
        MCK(cudaStreamSynchronize(m->st));
        return record_error(DP_ETIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs");
    }
    return DP_OK;
}

}  // namespace

namespace {

// One training step on a batch of the grid's nodes, everything on m->st:
// the batch of samples start .. start + B - 1 of the epoch's permutation (from
// m->ts), forward, backward, Adam with step count m->ts->t, then the next
// step's start and count.  Replayable: no argument changes between steps.
int train_step(dp_mlp* m, const GridView& gv, int B, Box4 nlo, Box4 nhi, double lr)
{
    const double invM = 1.0 / gv.M;
    if (gv.fp32 && !gv.V64)
        batch_from_grid_kernel<float><<<(B + 255) / 256, 256, 0, m->st>>>(
            gv.g64, (const float*)gv.V, gv.code, gv.tab_hi64, gv.tab_lo64, gv.n, 0, 0, 0, B, invM, nlo, nhi, m->x,
            m->t, m->ts);
    else
        batch_from_grid_kernel<double><<<(B + 255) / 256, 256, 0, m->st>>>(
            gv.g64, gv.V64 ? gv.V64 : (const double*)gv.V, gv.code, gv.tab_hi64, gv.tab_lo64, gv.n, 0, 0, 0, B, invM,
            nlo, nhi, m->x, m->t, m->ts);
    MCK(cudaGetLastError());
    int rc;
    if ((rc = forward_backward(m, B, 1.0f / (3.0f * B)))) return rc;
    return adam_launch(m, lr, B);   // with the next step's start and count
}

// The epochs of dp_mlp_train_grid.  The first step runs as launched (it also
// sets the kernels' attributes); the next one is captured as a CUDA graph
// and every later step replays it, which removes the host's 13 launches
// per step.
int train_grid_steps(dp_mlp* m, const GridView& gv, const dp_mlp_train_opts* o, dp_mlp_train_stats* stats)
{
    const long long n = gv.n;
    const int B = o->batch;
    const long long steps_per_epoch = n / B;
    const Box4 nlo{m->lo[0], m->lo[1], m->lo[2], m->lo[3]};
    const Box4 nhi{m->hi[0], m->hi[1], m->hi[2], m->hi[3]};
    double last_loss = 0.0, first_loss = -1.0;
    unsigned long long rng = o->seed ? o->seed : 14675ull;
    auto next = [&]() {   // splitmix64: seeds of the per-epoch permutation
        rng += 0x9E3779B97F4A7C15ull;
        unsigned long long z = rng;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto gcd = [](unsigned long long a, unsigned long long b) { while (b) { unsigned long long t = a % b; a = b; b = t; } return a; };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto done = [&](int rc) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return rc;
    };
    int rc;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
        (e = cudaEventRecord(e0, m->st)) != cudaSuccess)
        return done(fail_cuda("training events", e));
    for (int ep = 0; ep < o->epochs; ++ep) {
        unsigned long long mult = (next() % (unsigned long long)n) | 1ull;
        while (gcd(mult, (unsigned long long)n) != 1) mult = (mult + 2) % (unsigned long long)n;
        const unsigned long long off = next() % (unsigned long long)n;
        // the previous epoch's copy from h_ts has completed (check_err synchronised)
        // the epoch's step size: geometric from lr to lr_final over the epochs
        double lr_ep = o->lr;
        if (o->lr_final > 0 && o->epochs > 1) lr_ep = o->lr * pow(o->lr_final / o->lr, (double)ep / (o->epochs - 1));
        *m->h_ts = TrainState{(long long)mult, (long long)off, 0, (int)(m->step + 1), (float)lr_ep};
        if ((e = cudaMemcpyAsync(m->ts, m->h_ts, sizeof(TrainState), cudaMemcpyHostToDevice, m->st)) != cudaSuccess ||
            (e = cudaMemsetAsync(m->loss, 0, sizeof(float), m->st)) != cudaSuccess)
            return done(fail_cuda("training state", e));
        for (long long s = 0; s < steps_per_epoch; ++s) {
            if (exec) {
                if ((e = cudaGraphLaunch(exec, m->st)) != cudaSuccess) return done(fail_cuda("graph launch", e));
            } else if (ep == 0 && s == 0) {
                if ((rc = train_step(m, gv, B, nlo, nhi, o->lr))) return done(rc);
            } else {
                if ((e = cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                    return done(fail_cuda("stream capture", e));
                const int rs = train_step(m, gv, B, nlo, nhi, o->lr);
                e = cudaStreamEndCapture(m->st, &graph);
                if (rs) return done(rs);
                if (e != cudaSuccess) return done(fail_cuda("stream capture", e));
                if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess ||
                    (e = cudaGraphLaunch(exec, m->st)) != cudaSuccess)
                    return done(fail_cuda("training graph", e));
            }
        }
        m->step += steps_per_epoch;
        if ((e = cudaMemcpyAsync(m->h_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st)) != cudaSuccess)
            return done(fail_cuda("loss read-back", e));
        if ((rc = check_err(m))) return done(rc);
        last_loss = *m->h_loss / (3.0 * B * (double)steps_per_epoch);
        if (first_loss < 0) first_loss = last_loss;
    }
    if ((e = cudaEventRecord(e1, m->st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess)
        return done(fail_cuda("training events", e));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (stats) {
        stats->epochs = o->epochs;
        stats->steps = steps_per_epoch * o->epochs;
        stats->samples = (int64_t)B * steps_per_epoch * o->epochs;
        stats->first_epoch_loss = first_loss;
        stats->last_epoch_loss = last_loss;
        stats->ms = ms;
        stats->flops = 3.0 * 2.0 * 132864.0 * (double)stats->samples;   // forward + 2x backward
    }
    return done(DP_OK);
}

}  // namespace

extern "C" {

int64_t dp_mlp_param_count(void) { return kParams; }

int dp_mlp_create(const double* lo, const double* hi, int32_t batch_capacity, void* stream, dp_mlp** out)
{
    if (!out || !lo || !hi) return record_error(DP_EINVAL, "NULL argument");
    *out = nullptr;
    if (batch_capacity < 512 || batch_capacity % 512 != 0 || batch_capacity > (1 << 20))
        return record_error(DP_EINVAL, "batch_capacity must be a multiple of 512 in [512, 2^20]");
    for (int d = 0; d < 4; ++d)
        if (!(lo[d] < hi[d])) return record_error(DP_EINVAL, "input box needs lo < hi");
    dp_mlp* m = new (std::nothrow) dp_mlp();
    if (!m) return record_error(DP_ENOMEM, "host allocation failed");
    m->st = (cudaStream_t)stream;
    m->cap = batch_capacity;
    for (int d = 0; d < 4; ++d) { m->lo[d] = lo[d]; m->hi[d] = hi[d]; }
    cudaGetDevice(&m->device);
    cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
    const size_t C = (size_t)m->cap, CH = C * kH;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) { if (e == cudaSuccess) e = malloc_n(p, n); };
    A(&m->P, kParams); A(&m->G, kParams); A(&m->Am, kParams); A(&m->Av, kParams);
    A(&m->W2b, kH * kH); A(&m->W3b, kH * kH); A(&m->W2T, kH * kH); A(&m->W3T, kH * kH);
    A(&m->x, C * 4); A(&m->t, C * 3); A(&m->y, C * 3);
    A(&m->z1, CH); A(&m->z2, CH); A(&m->z3, CH);
    A(&m->h1, CH); A(&m->h2, CH); A(&m->h3, CH); A(&m->dz1, CH); A(&m->dz2, CH); A(&m->dz3, CH);
    A(&m->states, C * 4); A(&m->loss, 1); A(&m->err, 1); A(&m->part, kPartFloats);
    A(&m->red, C / kTileM * 5 * kH); A(&m->arrive, 1);
    A(&m->ts, 1);
    if (e == cudaSuccess) e = cudaMallocHost(&m->h_loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMallocHost(&m->h_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&m->h_ts, sizeof(TrainState));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->cst, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_mlp(m);
        return record_error(DP_ENOMEM, "device allocation of the network failed");
    }
    cudaMemsetAsync(m->Am, 0, sizeof(float) * kParams, m->st);
    cudaMemsetAsync(m->Av, 0, sizeof(float) * kParams, m->st);
    cudaMemsetAsync(m->err, 0, sizeof(int), m->st);
    cudaMemsetAsync(m->arrive, 0, sizeof(unsigned), m->st);
    *out = m;
    return DP_OK;
}

int dp_mlp_destroy(dp_mlp* m)
{
    free_mlp(m);
    return DP_OK;
}

int dp_mlp_set_params(dp_mlp* m, const float* params, int64_t count)
{
    if (!m || !params) return record_error(DP_EINVAL, "NULL argument");
    if (count != kParams) return record_error(DP_EINVAL, "parameter count mismatch");
    MCK(cudaMemcpyAsync(m->P, params, sizeof(float) * kParams, cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemsetAsync(m->Am, 0, sizeof(float) * kParams, m->st));
    MCK(cudaMemsetAsync(m->Av, 0, sizeof(float) * kParams, m->st));
    m->step = 0;
    int rc = refresh_bf16(m);
    if (rc) return rc;
    MCK(cudaStreamSynchronize(m->st));
    return DP_OK;
}

int dp_mlp_get_params(const dp_mlp* m, float* params, int64_t count)
{
    if (!m || !params) return record_error(DP_EINVAL, "NULL argument");
    if (count != kParams) return record_error(DP_EINVAL, "parameter count mismatch");
    MCK(cudaMemcpyAsync(params, m->P, sizeof(float) * kParams, cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    return DP_OK;
}

int dp_mlp_forward(dp_mlp* m, const double* states, int32_t n, float* out)
{
    if (!m || (n > 0 && (!states || !out))) return record_error(DP_EINVAL, "NULL argument");
    if (n < 0) return record_error(DP_EINVAL, "n < 0");
    const Box4 lo{m->lo[0], m->lo[1], m->lo[2], m->lo[3]};
    const Box4 hi{m->hi[0], m->hi[1], m->hi[2], m->hi[3]};
    for (int s0 = 0; s0 < n; s0 += m->cap) {
        const int cnt = std::min(m->cap, n - s0);
        MCK(cudaMemcpyAsync(m->states, states + 4 * (size_t)s0, sizeof(double) * 4 * cnt, cudaMemcpyHostToDevice,
                            m->st));
        states_in_kernel<<<(cnt + 255) / 256, 256, 0, m->st>>>(m->states, cnt, lo, hi, m->x);
        MCK(cudaGetLastError());
        int rc = forward(m, cnt);
        if (rc) return rc;
        MCK(cudaMemcpyAsync(out + 3 * (size_t)s0, m->y, sizeof(float) * 3 * cnt, cudaMemcpyDeviceToHost, m->st));
    }
    return check_err(m);
}

int dp_mlp_gradients(dp_mlp* m, const double* states, const float* targets, int32_t n, float* grads, float* loss)
{
    if (!m || !states || !targets || !grads) return record_error(DP_EINVAL, "NULL argument");
    if (n < 512 || n % 512 != 0 || n > m->cap) return record_error(DP_EINVAL, "n must be a multiple of 512 <= capacity");
    const Box4 lo{m->lo[0], m->lo[1], m->lo[2], m->lo[3]};
    const Box4 hi{m->hi[0], m->hi[1], m->hi[2], m->hi[3]};
    MCK(cudaMemcpyAsync(m->states, states, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemcpyAsync(m->t, targets, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, m->st));
    states_in_kernel<<<(n + 255) / 256, 256, 0, m->st>>>(m->states, n, lo, hi, m->x);
    MCK(cudaMemsetAsync(m->loss, 0, sizeof(float), m->st));
    int rc = forward_backward(m, n, 1.0f / (3.0f * n));
    if (rc) return rc;
    MCK(cudaMemcpyAsync(grads, m->G, sizeof(float) * kParams, cudaMemcpyDeviceToHost, m->st));
    MCK(cudaMemcpyAsync(m->h_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->st));
    if ((rc = check_err(m))) return rc;
    if (loss) *loss = *m->h_loss / (3.0f * n);
    return DP_OK;
}

int dp_mlp_apply_gradients(dp_mlp* m, const float* grads, int64_t count, double lr)
{
    if (!m || !grads) return record_error(DP_EINVAL, "NULL argument");
    if (count != kParams) return record_error(DP_EINVAL, "parameter count mismatch");
    if (!(lr > 0)) return record_error(DP_EINVAL, "lr must be positive");
    MCK(cudaMemcpyAsync(m->G, grads, sizeof(float) * kParams, cudaMemcpyHostToDevice, m->st));
    int rc = adam_step(m, lr);
    if (rc) return rc;
    MCK(cudaStreamSynchronize(m->st));
    return DP_OK;
}

int dp_mlp_set_wait_limit(dp_mlp* m, int32_t polls)
{
    if (!m || polls < -1) return record_error(DP_EINVAL, "bad argument");
    m->wait_polls = polls >= 0 ? polls : kWaitPolls;
    return DP_OK;
}

int dp_mlp_train_grid(dp_mlp* m, dp_grid* grid, const dp_mlp_train_opts* o, dp_mlp_train_stats* stats)
{
    if (!m || !grid || !o) return record_error(DP_EINVAL, "NULL argument");
    if (o->batch < 512 || o->batch % 512 != 0 || o->batch > m->cap || o->epochs < 0 || !(o->lr > 0) ||
        !(o->lr_final >= 0))
        return record_error(DP_EINVAL, "bad training options");
    GridView gv;
    int rc = grid_view(grid, &gv);
    if (rc) return rc;
    if (gv.n < o->batch) return record_error(DP_EINVAL, "grid smaller than one batch");
    // the steps run on the network's private stream, ordered after the
    // caller's stream and before its later work
    cudaStream_t user = m->st;
    MCK(cudaEventRecord(m->ev_in, user));
    MCK(cudaStreamWaitEvent(m->cst, m->ev_in, 0));
    m->st = m->cst;
    rc = train_grid_steps(m, gv, o, stats);
    m->st = user;
    cudaError_t e = cudaEventRecord(m->ev_out, m->cst);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, m->ev_out, 0);
    if (rc) return rc;
    MCK(e);
    return DP_OK;
}

int dp_warm_start(dp_mlp* m, dp_grid* grid, double* ms_out)
{
    if (!m || !grid) return record_error(DP_EINVAL, "NULL argument");
    GridView gv;
    int rc = grid_view(grid, &gv);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    MCK(cudaEventCreate(&e0));
    MCK(cudaEventCreate(&e1));
    MCK(cudaEventRecord(e0, m->st));
    // node coordinates of this grid, normalised to the network's own box
    Geo<double> g = gv.g64;
    const Box4 nlo{m->lo[0], m->lo[1], m->lo[2], m->lo[3]};
    const Box4 nhi{m->hi[0], m->hi[1], m->hi[2], m->hi[3]};
    for (long long s0 = 0; s0 < gv.n; s0 += m->cap) {
        const int cnt = (int)std::min<long long>(m->cap, gv.n - s0);
        batch_from_grid_kernel<double><<<(cnt + 255) / 256, 256, 0, m->st>>>(
            g, (const double*)nullptr, gv.code, gv.tab_hi64, gv.tab_lo64, gv.n, 1, 0, s0, cnt, 0.0, nlo, nhi, m->x,
            nullptr);
        MCK(cudaGetLastError());
        if ((rc = forward(m, cnt))) return rc;
        // the value goes to the storage-precision buffer (an FP32 grid holding
        // FP64 values after a polish returns to its FP32 values)
        if (gv.fp32)
            warm_write_kernel<float><<<(cnt + 255) / 256, 256, 0, m->st>>>(g, m->y, s0, cnt, gv.M, (float*)gv.V,
                                                                         gv.code);
        else
            warm_write_kernel<double><<<(cnt + 255) / 256, 256, 0, m->st>>>(g, m->y, s0, cnt, gv.M, (double*)gv.V,
                                                                          gv.code);
        MCK(cudaGetLastError());
    }
    MCK(cudaEventRecord(e1, m->st));
    if ((rc = check_err(m))) return rc;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_out) *ms_out = ms;
    grid_after_warm_start(grid);
    return DP_OK;
}

}  // extern "C"
