// Learned warm start: the network of include/lskum_mlp.h on the Blackwell
// tensor cores.
//
// Every matrix product D[M x N] = A[M x K] B[N x K]^T of training and
// inference runs in k_gemm: one CTA of 4 warps owns a 128-row tile of D in
// tensor memory (TMEM, FP32, one lane per row); K is staged through shared
// memory in chunks of 64 (A: 128 x 64, B: N x 64 BF16) in the canonical
// K-major, non-swizzled core-matrix layout (8 rows x 16 bytes per core
// matrix, k-groups 128 B apart, 8-row groups 1024 B apart), and one elected
// thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
// K = 16 per instruction) and commits to an mbarrier that all threads wait
// on.  The epilogue reads the accumulator back with tcgen05.ld (32x32b: each
// thread one row) and fuses what follows the product:
//   kFwdHidden  Z + b -> GELU -> BF16 activations (row-major and transposed)
//               and GELU'(Z) for the backward pass;
//   kFwdOut     Z + b -> outputs (FP32);
//   kBwdData    (G W) * GELU'(Z) -> BF16 gradients (row-major and transposed);
//   kWgrad      split-K partial sums of G^T A for the weight gradients.
// Inference (forward pass, prediction into a solver state) instead runs
// k_mlp_fused: persistent CTAs keep all five layers' weights in shared memory
// and carry each 128-point tile through the five products with the
// activations staying on the SM (see the comment above that kernel).
// Operand layouts: activations and gradients are kept both point-major
// ([points][features], the A operand of forward and backward-data products)
// and feature-major ([features][points], the operands of weight-gradient
// products, where the points are the reduction dimension); the weights both
// as W [out][in] (forward) and W^T [in][out] (backward data).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lskum_mlp.h"
#include "lskum_mlp_internal.h"

namespace {

constexpr int kFreq = 16, kIn = 34, kInPad = 48, kWidth = 128, kOut = 4, kOutPad = 16;
constexpr int kLayers = 5;
constexpr int kInTrue[kLayers] = {kIn, kWidth, kWidth, kWidth, kWidth};
constexpr int kInP[kLayers] = {kInPad, kWidth, kWidth, kWidth, kWidth};
constexpr int kOutTrue[kLayers] = {kWidth, kWidth, kWidth, kWidth, kOut};
constexpr int kOutP[kLayers] = {kWidth, kWidth, kWidth, kWidth, kOutPad};
constexpr int kSplitK = 128;  // points per CTA in weight-gradient products
constexpr int kBatchAlign = 512;

constexpr int n_params_total()
{
    int s = 0;
    for (int l = 0; l < kLayers; l++) s += kOutTrue[l] * kInTrue[l] + kOutTrue[l];
    return s;
}
constexpr int kNParams = n_params_total();  // 54,532

enum Epi { kFwdHidden = 0, kFwdOut = 1, kBwdData = 2, kWgrad = 3 };

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_smem_to_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the barrier phase with a time limit (limit_ns; 1 s unless a test
// shortens it): false if it never came.
__device__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K), stride-dimension byte offset
// (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M = 128.
template <int N>
__host__ __device__ constexpr uint32_t idesc_bf16()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 FP32 accumulator columns of this thread's row (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t *>(&h);
}

__device__ __forceinline__ float bf16_val(uint16_t b)
{
    return __uint_as_float((uint32_t)b << 16);
}

__device__ __forceinline__ float gelu(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// the product kernel
// ---------------------------------------------------------------------------
struct GemmArgs {
    const uint16_t *A;  // [rows][lda] BF16, K contiguous; rows >= a_rows read as 0
    int lda, a_rows;
    const uint16_t *B;  // [N rows][ldb]; rows >= b_rows read as 0
    int ldb, b_rows;
    int K, k_split;     // K extent (multiple of 16); K per CTA along grid.y
    int m_valid;        // rows of D that hold data; the tile's other rows get zeros
    const float *bias;  // [N] (kFwdHidden, kFwdOut)
    const float *gp_in; // [rows][128] GELU'(Z) of the product's output features (kBwdData)
    float *gp_out;      // [rows][128] (kFwdHidden, may be null)
    uint16_t *out;      // [rows][ldo] BF16
    int ldo;
    uint16_t *out_t;    // [N][ldt] BF16 transposed (may be null)
    int ldt;
    float *out_f;       // kFwdOut: [rows][4]; kWgrad: [split][m_valid][N]
    int *err;
    uint64_t wait_ns;   // time limit of each wait for the tensor core
    int skip_products;  // failure-path test: issue neither products nor commit
};

// 24 KB of dynamic shared memory is requested on top of the 32 KB of operand
// buffers so that at most 4 CTAs share an SM: 4 x 128 TMEM columns = 512.
constexpr int kPadSmem = 24 * 1024;

template <int EPI, int N>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g)
{
    static_assert(N % 16 == 0 && N >= 16 && N <= 128, "N");
    constexpr uint32_t kCols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
    constexpr uint32_t kIdesc = idesc_bf16<N>();
    __shared__ __align__(1024) uint8_t sA[128 * 64 * 2];
    __shared__ __align__(1024) uint8_t sB[128 * 64 * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    extern __shared__ uint8_t pad_smem[];
    (void)pad_smem;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
    const int kb = blockIdx.y * g.k_split;
    const int ke = min(g.K, kb + g.k_split);
    if (warp == 0) tmem_alloc(&tslot, kCols);
    if (tid == 0) mbar_init(&bar, 1);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tslot;

    uint32_t parity = 0;
    int ok = 1;
    const bool any = ke > kb;
    for (int kc = kb; kc < ke && ok; kc += 64) {
        const int kw = min(64, ke - kc);  // a multiple of 16
        const int kg = kw >> 3;           // 16-byte k-groups in this chunk
        for (int v = tid; v < 128 * kg; v += 128) {
            const int r = v / kg, j = v - r * kg;
            const int row = m0 + r;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (row < g.a_rows) val = *reinterpret_cast<const uint4 *>(g.A + (size_t)row * g.lda + kc + 8 * j);
            *reinterpret_cast<uint4 *>(sA + ((r >> 3) * 8 + j) * 128 + (r & 7) * 16) = val;
        }
        for (int v = tid; v < N * kg; v += 128) {
            const int r = v / kg, j = v - r * kg;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (r < g.b_rows) val = *reinterpret_cast<const uint4 *>(g.B + (size_t)r * g.ldb + kc + 8 * j);
            *reinterpret_cast<uint4 *>(sB + ((r >> 3) * 8 + j) * 128 + (r & 7) * 16) = val;
        }
        fence_smem_to_async();
        __syncthreads();
        if (tid == 0 && !g.skip_products) {
            fence_after_sync();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int s = 0; s < (kw >> 4); s++)
                mma_bf16(tmem, smem_desc(a0 + 256u * s, 128u, 1024u), smem_desc(b0 + 256u * s, 128u, 1024u), kIdesc,
                         (kc > kb || s > 0) ? 1u : 0u);
            mma_commit(&bar);
        }
        ok = __syncthreads_and(mbar_wait_bounded(&bar, parity, g.wait_ns) ? 1 : 0);
        parity ^= 1u;
    }
    fence_after_sync();

    const int r = warp * 32 + lane;
    const int row = m0 + r;
    const bool live = row < g.m_valid;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            if (any) tmem_ld16(taddr + (uint32_t)c0, v);
            else
#pragma unroll
                for (int i = 0; i < 16; i++) v[i] = 0.f;
            if (EPI == kWgrad) {
                if (live) {
                    float *o = g.out_f + ((size_t)blockIdx.y * g.m_valid + row) * N + c0;
#pragma unroll
                    for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4 *>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                }
                continue;
            }
            if (EPI == kFwdOut) {
                if (live && c0 == 0)
#pragma unroll
                    for (int i = 0; i < kOut; i++) g.out_f[(size_t)row * kOut + i] = v[i] + g.bias[i];
                continue;
            }
            uint16_t h[16];
            float gp[16];
#pragma unroll
            for (int i = 0; i < 16; i++) {
                float y = 0.f;
                gp[i] = 0.f;
                if (live) {
                    if (EPI == kFwdHidden) {
                        const float z = v[i] + g.bias[c0 + i];
                        y = gelu(z);
                        gp[i] = gelu_grad(z);
                    } else {  // kBwdData
                        y = v[i] * g.gp_in[(size_t)row * kWidth + c0 + i];
                    }
                }
                h[i] = bf16_bits(y);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(g.out + (size_t)row * g.ldo + c0);
            dst[0] = make_uint4(h[0] | (uint32_t)h[1] << 16, h[2] | (uint32_t)h[3] << 16, h[4] | (uint32_t)h[5] << 16,
                                h[6] | (uint32_t)h[7] << 16);
            dst[1] = make_uint4(h[8] | (uint32_t)h[9] << 16, h[10] | (uint32_t)h[11] << 16,
                                h[12] | (uint32_t)h[13] << 16, h[14] | (uint32_t)h[15] << 16);
            if (g.out_t)
#pragma unroll
                for (int i = 0; i < 16; i++) g.out_t[(size_t)(c0 + i) * g.ldt + row] = h[i];
            if (EPI == kFwdHidden && g.gp_out) {
                float *o = g.gp_out + (size_t)row * kWidth + c0;
#pragma unroll
                for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4 *>(o + i) = make_float4(gp[i], gp[i + 1], gp[i + 2], gp[i + 3]);
            }
        }
    } else if (tid == 0) {
        atomicExch(g.err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
// Network inputs of one point (x, y, wall distance, M, AoA deg) into X row i
// (BF16, 48 columns) and column i of Xt.
__device__ __forceinline__ void write_features(const float *B, float x, float y, float d, float mach, float aoa,
                                               uint16_t *X, uint16_t *Xt, int i, int ldt)
{
    const float X0 = x - 0.5f;
    const float r = sqrtf(X0 * X0 + y * y);
    const float z0 = X0 / (1.f + r), z1 = y / (1.f + r), z2 = d / (1.f + d);
    uint16_t h[kInPad];
#pragma unroll
    for (int f = 0; f < kFreq; f++) {
        const float t = B[3 * f] * z0 + B[3 * f + 1] * z1 + B[3 * f + 2] * z2;
        float s, c;
        sincospif(2.f * t, &s, &c);
        h[f] = bf16_bits(s);
        h[kFreq + f] = bf16_bits(c);
    }
    h[2 * kFreq] = bf16_bits(mach);
    h[2 * kFreq + 1] = bf16_bits(aoa * 0.1f);
#pragma unroll
    for (int f = kIn; f < kInPad; f++) h[f] = 0;
    uint4 *dst = reinterpret_cast<uint4 *>(X + (size_t)i * kInPad);
#pragma unroll
    for (int q = 0; q < kInPad / 8; q++)
        dst[q] = make_uint4(h[8 * q] | (uint32_t)h[8 * q + 1] << 16, h[8 * q + 2] | (uint32_t)h[8 * q + 3] << 16,
                            h[8 * q + 4] | (uint32_t)h[8 * q + 5] << 16, h[8 * q + 6] | (uint32_t)h[8 * q + 7] << 16);
    if (Xt)
#pragma unroll
        for (int f = 0; f < kInPad; f++) Xt[(size_t)f * ldt + i] = h[f];
}

__device__ __forceinline__ void zero_features(uint16_t *X, uint16_t *Xt, int i, int ldt)
{
    uint4 *dst = reinterpret_cast<uint4 *>(X + (size_t)i * kInPad);
    for (int q = 0; q < kInPad / 8; q++) dst[q] = make_uint4(0u, 0u, 0u, 0u);
    if (Xt)
        for (int f = 0; f < kInPad; f++) Xt[(size_t)f * ldt + i] = 0;
}

// Rows [0, rows): sample idx[i] (or i without idx) of in5 for i < n, zeros after.
__global__ void k_features(const float *in5, const int32_t *idx, int n, int rows, const float *B, uint16_t *X,
                           uint16_t *Xt, int ldt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    if (i >= n) {
        zero_features(X, Xt, i, ldt);
        return;
    }
    const float *s = in5 + (size_t)(idx ? idx[i] : i) * 5;
    write_features(B, s[0], s[1], s[2], s[3], s[4], X, Xt, i, ldt);
}

// Given inputs X [n][34] (FP32) -> BF16 X rows and Xt columns, zeros up to rows.
__global__ void k_inputs_from_f32(const float *Xf, int n, int rows, uint16_t *X, uint16_t *Xt, int ldt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    for (int f = 0; f < kInPad; f++) {
        const uint16_t h = (i < n && f < kIn) ? bf16_bits(Xf[(size_t)i * kIn + f]) : (uint16_t)0;
        X[(size_t)i * kInPad + f] = h;
        if (Xt) Xt[(size_t)f * ldt + i] = h;
    }
}

// BF16 X rows back to FP32 [n][34].
__global__ void k_inputs_to_f32(const uint16_t *X, int n, float *Xf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int f = 0; f < kIn; f++) Xf[(size_t)i * kIn + f] = bf16_val(X[(size_t)i * kInPad + f]);
}

// Loss and output gradient: E = O - T, loss += sum E^2 / (4 n), G = 2 E / (4 n)
// (BF16, G [rows][16] and Gt [16][ldt]); rows >= n get zeros.
__global__ void __launch_bounds__(256) k_loss(const float *O, const float *T, const int32_t *idx, int n, int rows,
                                              uint16_t *G, uint16_t *Gt, int ldt, double *loss)
{
    __shared__ double red[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e2 = 0.0;
    if (i < rows) {
        const float sc = 2.f / (4.f * (float)n);
        for (int c = 0; c < kOut; c++) {
            uint16_t h = 0;
            if (i < n) {
                const float e = O[(size_t)i * kOut + c] - T[(size_t)(idx ? idx[i] : i) * kOut + c];
                e2 += (double)e * e;
                h = bf16_bits(sc * e);
            }
            G[(size_t)i * kOutPad + c] = h;
            Gt[(size_t)c * ldt + i] = h;
        }
    }
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; w++) s += red[w];
        atomicAdd(loss, s / (4.0 * n));
    }
}

// Bias gradient: db[o] = sum over points of Gt[o][p] (fixed order).
__global__ void __launch_bounds__(256) k_colsum(const uint16_t *Gt, int ldt, int cols, float *db)
{
    __shared__ float red[8];
    const int o = blockIdx.x;
    float s = 0.f;
    for (int p = threadIdx.x; p < cols; p += 256) s += bf16_val(Gt[(size_t)o * ldt + p]);
    for (int q = 16; q > 0; q >>= 1) s += __shfl_xor_sync(0xffffffffu, s, q);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; w++) t += red[w];
        db[o] = t;
    }
}

// Weight gradient: dW[o][i] = sum over splits of partial[s][o][i] (i < in_true).
__global__ void k_reduce_wgrad(const float *part, int splits, int m_valid, int N, int in_true, float *dW)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m_valid * in_true) return;
    const int o = t / in_true, i = t - o * in_true;
    float s = 0.f;
    for (int q = 0; q < splits; q++) s += part[((size_t)q * m_valid + o) * N + i];
    dW[t] = s;
}

__global__ void k_adam(float *p, float *m, float *v, const float *g, int n, float lr, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

struct PackArgs {
    const float *params;
    uint16_t *W[kLayers], *Wt[kLayers];
    int off[kLayers], in_true[kLayers], in_pad[kLayers], out_true[kLayers], out_pad[kLayers];
};

// BF16 copies of the weights: W [out_pad][in_pad] and W^T [in_pad][out_pad], zero padded.
__global__ void k_pack(PackArgs a)
{
    const int l = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int ip = a.in_pad[l], op = a.out_pad[l];
    if (t >= ip * op) return;
    const int o = t / ip, i = t - o * ip;
    const float w = (o < a.out_true[l] && i < a.in_true[l]) ? a.params[a.off[l] + o * a.in_true[l] + i] : 0.f;
    const uint16_t h = bf16_bits(w);
    a.W[l][(size_t)o * ip + i] = h;
    a.Wt[l][(size_t)i * op + o] = h;
}

// ---------------------------------------------------------------------------
// fused forward pass (inference): all five layers of a 128-point tile in one
// CTA, weights resident in shared memory, activations never leave the SM
// ---------------------------------------------------------------------------
// Shared memory (dynamic): the BF16 weights of the five layers in the
// core-matrix layout (W1 128x48, W2..W4 128x128, W5 16x128: 112 KB), the
// input tile (128x48) and the hidden tile (128x128) that each layer's
// epilogue overwrites with the next layer's input, and the biases.  Persistent
// CTAs (one per SM, 8 warps) loop over the tiles.  Per layer one thread issues
// the K/16 products into a 128-column TMEM accumulator; warps w and w + 4 read
// the same 32 accumulator lanes (rows) and split the columns.
constexpr int kFusedThreads = 256;
constexpr int kSmemW1 = 128 * kInPad * 2, kSmemW = 128 * 128 * 2, kSmemW5 = kOutPad * 128 * 2;
constexpr int kSmemX = 128 * kInPad * 2, kSmemH = 128 * 128 * 2;
constexpr int kOffW1 = 0, kOffW2 = kOffW1 + kSmemW1, kOffW5 = kOffW2 + 3 * kSmemW, kOffX = kOffW5 + kSmemW5,
              kOffH = kOffX + kSmemX, kOffBias = kOffH + kSmemH;
constexpr int kBiasFloats = 4 * kWidth + kOutPad;
constexpr int kFusedSmem = kOffBias + kBiasFloats * 4;

enum FusedSrc { kSrcBuffer = 0, kSrcView = 1 };

struct FusedArgs {
    const uint16_t *W[kLayers];  // global BF16 weights [out_pad][in_pad]
    const float *params;
    int off[kLayers];
    int n;                       // rows (points)
    const uint16_t *X;           // kSrcBuffer: [n][48] BF16 inputs
    float *O;                    // kSrcBuffer: [n][4] outputs
    lskum::MlpView v;            // kSrcView: points k0 + i of the view, state written
    int k0;
    const float *fourier;
    int *err;
    uint64_t wait_ns;   // time limit of each wait for the tensor core
    int skip_products;  // failure-path test: issue neither products nor commit
};

// Write a row of 16-bit values (8 per 16-byte chunk) into a core-matrix tile.
__device__ __forceinline__ void store_row_chunk(uint8_t *tile, int kg_stride, int r, int j, const uint16_t *h8)
{
    *reinterpret_cast<uint4 *>(tile + ((r >> 3) * kg_stride + j) * 128 + (r & 7) * 16) =
        make_uint4(h8[0] | (uint32_t)h8[1] << 16, h8[2] | (uint32_t)h8[3] << 16, h8[4] | (uint32_t)h8[5] << 16,
                   h8[6] | (uint32_t)h8[7] << 16);
}

template <int SRC>
__global__ void __launch_bounds__(kFusedThreads, 1) k_mlp_fused(FusedArgs a)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *sbias = reinterpret_cast<float *>(sm + kOffBias);
    // weights and biases, once per CTA
    for (int l = 0; l < kLayers; l++) {
        const int ip = l == 0 ? kInPad : kWidth, op = l == 4 ? kOutPad : kWidth, kg = ip / 8;
        uint8_t *dst = sm + (l == 0 ? kOffW1 : (l == 4 ? kOffW5 : kOffW2 + (l - 1) * kSmemW));
        for (int v = tid; v < op * kg; v += kFusedThreads) {
            const int r = v / kg, j = v - r * kg;
            *reinterpret_cast<uint4 *>(dst + ((r >> 3) * kg + j) * 128 + (r & 7) * 16) =
                *reinterpret_cast<const uint4 *>(a.W[l] + (size_t)r * ip + 8 * j);
        }
    }
    for (int i = tid; i < kBiasFloats; i += kFusedThreads) {
        const int l = i / kWidth, c = i - l * kWidth;
        sbias[i] = (l < 4) ? a.params[a.off[l] + kWidth * (l == 0 ? kIn : kWidth) + c]
                           : (c < kOut ? a.params[a.off[4] + kOut * kWidth + c] : 0.f);
    }
    if (warp == 0) tmem_alloc(&tslot, 128);
    if (tid == 0) mbar_init(&bar, 1);
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t sX = smem_u32(sm + kOffX), sH = smem_u32(sm + kOffH);
    uint32_t parity = 0;
    int ok = 1;
    const int n_tiles = (a.n + 127) / 128;
    const int r_epi = 32 * (warp & 3) + lane;  // accumulator row (lane) this thread reads
    const int c_half = (warp >> 2) * 64;       // its 64 columns
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int p0 = t * 128;
        // 1. the input tile
        if (tid < 128) {
            const int i = p0 + tid;
            uint16_t h[kInPad];
            if (i < a.n) {
                if (SRC == kSrcBuffer) {
                    const uint4 *src = reinterpret_cast<const uint4 *>(a.X + (size_t)i * kInPad);
#pragma unroll
                    for (int q = 0; q < kInPad / 8; q++) {
                        const uint4 u = src[q];
                        h[8 * q] = u.x & 0xFFFF; h[8 * q + 1] = u.x >> 16; h[8 * q + 2] = u.y & 0xFFFF;
                        h[8 * q + 3] = u.y >> 16; h[8 * q + 4] = u.z & 0xFFFF; h[8 * q + 5] = u.z >> 16;
                        h[8 * q + 6] = u.w & 0xFFFF; h[8 * q + 7] = u.w >> 16;
                    }
                } else {
                    const int k = a.k0 + i;
                    const int b = a.v.case_of[k];
                    const float X0 = a.v.x[k] - 0.5f, y = a.v.y[k], d = a.v.dwall[k];
                    const float r = sqrtf(X0 * X0 + y * y);
                    const float z0 = X0 / (1.f + r), z1 = y / (1.f + r), z2 = d / (1.f + d);
#pragma unroll
                    for (int f = 0; f < kFreq; f++) {
                        const float tt = a.fourier[3 * f] * z0 + a.fourier[3 * f + 1] * z1 + a.fourier[3 * f + 2] * z2;
                        float sn, cs;
                        sincospif(2.f * tt, &sn, &cs);
                        h[f] = bf16_bits(sn);
                        h[kFreq + f] = bf16_bits(cs);
                    }
                    h[2 * kFreq] = bf16_bits(a.v.case_mach[b]);
                    h[2 * kFreq + 1] = bf16_bits(a.v.case_aoa[b] * 0.1f);
#pragma unroll
                    for (int f = kIn; f < kInPad; f++) h[f] = 0;
                }
            } else {
#pragma unroll
                for (int f = 0; f < kInPad; f++) h[f] = 0;
            }
#pragma unroll
            for (int j = 0; j < kInPad / 8; j++) store_row_chunk(sm + kOffX, kInPad / 8, tid, j, h + 8 * j);
        }
        fence_smem_to_async();
        __syncthreads();
        // 2. the four hidden layers
        for (int l = 0; l < 4 && ok; l++) {
            if (tid == 0 && !a.skip_products) {
                fence_after_sync();
                const int kg = l == 0 ? kInPad / 8 : kWidth / 8;
                const uint32_t a0 = l == 0 ? sX : sH;
                const uint32_t b0 = smem_u32(sm + (l == 0 ? kOffW1 : kOffW2 + (l - 1) * kSmemW));
                for (int s = 0; s < kg / 2; s++)
                    mma_bf16(tmem, smem_desc(a0 + 256u * s, 128u, 128u * kg), smem_desc(b0 + 256u * s, 128u, 128u * kg),
                             idesc_bf16<128>(), s > 0 ? 1u : 0u);
                mma_commit(&bar);
            }
            ok = __syncthreads_and(mbar_wait_bounded(&bar, parity, a.wait_ns) ? 1 : 0);
            parity ^= 1u;
            if (!ok) break;
            fence_after_sync();
#pragma unroll 1
            for (int c0 = c_half; c0 < c_half + 64; c0 += 16) {
                float v[16];
                tmem_ld16(taddr + (uint32_t)c0, v);
                uint16_t h[16];
#pragma unroll
                for (int q = 0; q < 16; q++) h[q] = bf16_bits(gelu(v[q] + sbias[l * kWidth + c0 + q]));
                store_row_chunk(sm + kOffH, kWidth / 8, r_epi, c0 / 8, h);
                store_row_chunk(sm + kOffH, kWidth / 8, r_epi, c0 / 8 + 1, h + 8);
            }
            fence_before_sync();
            fence_smem_to_async();
            __syncthreads();
        }
        if (!ok) break;
        // 3. the output layer (N = 16, four used)
        if (tid == 0 && !a.skip_products) {
            fence_after_sync();
            const uint32_t b0 = smem_u32(sm + kOffW5);
            for (int s = 0; s < kWidth / 16; s++)
                mma_bf16(tmem, smem_desc(sH + 256u * s, 128u, 128u * (kWidth / 8)),
                         smem_desc(b0 + 256u * s, 128u, 128u * (kWidth / 8)), idesc_bf16<16>(), s > 0 ? 1u : 0u);
            mma_commit(&bar);
        }
        ok = __syncthreads_and(mbar_wait_bounded(&bar, parity, a.wait_ns) ? 1 : 0);
        parity ^= 1u;
        if (!ok) break;
        fence_after_sync();
        if (warp < 4) {
            float v[16];
            tmem_ld16(taddr, v);
            const int i = p0 + r_epi;
            if (i < a.n) {
                float o[kOut];
#pragma unroll
                for (int q = 0; q < kOut; q++) o[q] = v[q] + sbias[4 * kWidth + q];
                if (SRC == kSrcBuffer) {
                    *reinterpret_cast<float4 *>(a.O + (size_t)i * kOut) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
                    const int k = a.k0 + i;
                    const int b = a.v.case_of[k];
                    const int ld = a.v.ld;
                    if (a.v.flag[k] == LSKUM_OUTER) {  // the context's own free stream, bit for bit
#pragma unroll
                        for (int q = 0; q < 4; q++) a.v.U[q * ld + k] = a.v.case_Uinf[4 * b + q];
                    } else {
                        const double rho = exp((double)o[0]);
                        const double u = a.v.case_uv[2 * b] + (double)o[1];
                        const double w = a.v.case_uv[2 * b + 1] + (double)o[2];
                        const double p = exp((double)o[3]) / 1.4;
                        a.v.U[k] = rho;
                        a.v.U[ld + k] = rho * u;
                        a.v.U[2 * ld + k] = rho * w;
                        a.v.U[3 * ld + k] = p / 0.4 + 0.5 * rho * (u * u + w * w);
                    }
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// Free stream of each point's case (all points of [0, n)).
__global__ void k_free_stream(lskum::MlpView v, const uint8_t *keep)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.n) return;
    const int b = v.case_of[k];
    if (keep && keep[b]) return;
    const int ld = v.ld;
#pragma unroll
    for (int q = 0; q < 4; q++) v.U[q * ld + k] = v.case_Uinf[4 * b + q];
}

// Training samples from a view's state: inputs (x, y, d, M, AoA) and targets.
__global__ void k_gather_samples(lskum::MlpView v, const int32_t *pts, int n, float *in5, float *tgt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = pts[i];
    const int b = v.case_of[k];
    const int ld = v.ld;
    const double rho = v.U[k], u = v.U[ld + k] / rho, w = v.U[2 * ld + k] / rho;
    const double p = 0.4 * (v.U[3 * ld + k] - 0.5 * rho * (u * u + w * w));
    in5[(size_t)i * 5] = v.x[k];
    in5[(size_t)i * 5 + 1] = v.y[k];
    in5[(size_t)i * 5 + 2] = v.dwall[k];
    in5[(size_t)i * 5 + 3] = v.case_mach[b];
    in5[(size_t)i * 5 + 4] = v.case_aoa[b];
    tgt[(size_t)i * 4] = (float)log(rho);
    tgt[(size_t)i * 4 + 1] = (float)(u - v.case_uv[2 * b]);
    tgt[(size_t)i * 4 + 2] = (float)(w - v.case_uv[2 * b + 1]);
    tgt[(size_t)i * 4 + 3] = (float)log(p * 1.4);
}

__global__ void k_wall_distance(const float *x, const float *y, const int32_t *case_of, int n, const float4 *seg,
                                const int32_t *seg_off, float *dwall)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int b = case_of[k];
    const float px = x[k], py = y[k];
    float best = 1e30f;
    for (int s = seg_off[b]; s < seg_off[b + 1]; s++) {
        const float4 e = seg[s];
        const float ex = e.z - e.x, ey = e.w - e.y;
        const float L2 = ex * ex + ey * ey;
        float t = L2 > 0.f ? ((px - e.x) * ex + (py - e.y) * ey) / L2 : 0.f;
        t = fminf(fmaxf(t, 0.f), 1.f);
        const float dx = px - (e.x + t * ex), dy = py - (e.y + t * ey);
        best = fminf(best, dx * dx + dy * dy);
    }
    dwall[k] = sqrtf(best);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t &s)
{
    return (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
}

template <int EPI, int N>
cudaError_t gemm(const GemmArgs &g, int grid_x, int grid_y, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm<EPI, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPadSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_gemm<EPI, N><<<dim3(grid_x, grid_y), 128, kPadSmem, s>>>(g);
    return cudaGetLastError();
}

}  // namespace

struct lskum_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t P = 0;  // batch capacity (multiple of kBatchAlign)
    std::vector<void *> allocs;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grads = nullptr, *fourier = nullptr;
    uint16_t *W[kLayers] = {}, *Wt[kLayers] = {};
    int off[kLayers] = {};
    uint16_t *X = nullptr, *Xt = nullptr, *H[4] = {}, *Ht[4] = {}, *G5 = nullptr, *G5t = nullptr, *G[4] = {},
             *Gt[4] = {};
    float *GP[4] = {}, *O = nullptr, *part = nullptr, *Xf = nullptr, *Tf = nullptr;
    double *loss = nullptr;
    int *err = nullptr;
    uint64_t wait_ns = 1000000000ull;  // time limit of the tensor-core waits
    int skip_products = 0;             // failure-path test switch (lskum_mlp_set_wait_test)
    int32_t *idx = nullptr;
    // sample store
    float *s_in = nullptr, *s_tgt = nullptr;
    int32_t n_samples = 0, cap_samples = 0;
    int adam_t = 0;
    std::string msg = "no error";
};

namespace {

thread_local std::string g_mlp_create_error = "no error";

lskum_status mfail(lskum_mlp *m, lskum_status s, const std::string &what)
{
    if (m) m->msg = what;
    else g_mlp_create_error = what;
    return s;
}

lskum_status mcuda(lskum_mlp *m, cudaError_t e, const char *what)
{
    return mfail(m, e == cudaErrorMemoryAllocation ? LSKUM_ERR_OOM : LSKUM_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t dalloc(lskum_mlp *m, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    m->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), m->stream);
}

cudaError_t pack(lskum_mlp *m)
{
    PackArgs a;
    a.params = m->params;
    for (int l = 0; l < kLayers; l++) {
        a.W[l] = m->W[l];
        a.Wt[l] = m->Wt[l];
        a.off[l] = m->off[l];
        a.in_true[l] = kInTrue[l];
        a.in_pad[l] = kInP[l];
        a.out_true[l] = kOutTrue[l];
        a.out_pad[l] = kOutP[l];
    }
    k_pack<<<dim3((kWidth * kWidth + 255) / 256, kLayers), 256, 0, m->stream>>>(a);
    return cudaGetLastError();
}

// Forward pass of rows [0, rows) already in m->X (BF16); n valid rows.
// train: also the transposed activations and GELU'(Z).
cudaError_t forward(lskum_mlp *m, int n, int rows, bool train)
{
    const int P = m->P;
    const int gx = rows / 128;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 4 && e == cudaSuccess; l++) {
        GemmArgs g{};
        g.A = l == 0 ? m->X : m->H[l - 1];
        g.lda = l == 0 ? kInPad : kWidth;
        g.a_rows = n;
        g.B = m->W[l];
        g.ldb = kInP[l];
        g.b_rows = kWidth;
        g.K = kInP[l];
        g.k_split = g.K;
        g.m_valid = n;
        g.bias = m->params + m->off[l] + kOutTrue[l] * kInTrue[l];
        g.gp_out = train ? m->GP[l] : nullptr;
        g.out = m->H[l];
        g.ldo = kWidth;
        g.out_t = train ? m->Ht[l] : nullptr;
        g.ldt = P;
        g.err = m->err;
        g.wait_ns = m->wait_ns;
        g.skip_products = m->skip_products;
        e = gemm<kFwdHidden, 128>(g, gx, 1, m->stream);
    }
    if (e != cudaSuccess) return e;
    GemmArgs g{};
    g.A = m->H[3];
    g.lda = kWidth;
    g.a_rows = n;
    g.B = m->W[4];
    g.ldb = kWidth;
    g.b_rows = kOutPad;
    g.K = kWidth;
    g.k_split = kWidth;
    g.m_valid = n;
    g.bias = m->params + m->off[4] + kOut * kWidth;
    g.out_f = m->O;
    g.err = m->err;
    g.wait_ns = m->wait_ns;
    g.skip_products = m->skip_products;
    return gemm<kFwdOut, 16>(g, gx, 1, m->stream);
}

// Backward pass after forward(train) and k_loss: gradients into m->grads.
cudaError_t backward(lskum_mlp *m, int n, int rows)
{
    const int P = m->P;
    const int gx = rows / 128;
    const int splits = rows / kSplitK;
    cudaError_t e = cudaSuccess;
    for (int l = 4; l >= 0 && e == cudaSuccess; l--) {
        // weight gradient of layer l: (G_l)^T A_{l-1}, points as the reduction
        GemmArgs w{};
        w.A = l == 4 ? m->G5t : m->Gt[l];
        w.lda = P;
        w.a_rows = l == 4 ? kOutPad : kWidth;
        w.B = l == 0 ? m->Xt : m->Ht[l - 1];
        w.ldb = P;
        w.b_rows = kInP[l];
        w.K = rows;
        w.k_split = kSplitK;
        w.m_valid = kOutTrue[l];
        w.out_f = m->part;
        w.err = m->err;
        w.wait_ns = m->wait_ns;
        w.skip_products = m->skip_products;
        e = l == 0 ? gemm<kWgrad, kInPad>(w, 1, splits, m->stream) : gemm<kWgrad, 128>(w, 1, splits, m->stream);
        if (e != cudaSuccess) break;
        const int nw = kOutTrue[l] * kInTrue[l];
        k_reduce_wgrad<<<(nw + 255) / 256, 256, 0, m->stream>>>(m->part, splits, kOutTrue[l], kInP[l], kInTrue[l],
                                                                 m->grads + m->off[l]);
        k_colsum<<<kOutTrue[l], 256, 0, m->stream>>>(l == 4 ? m->G5t : m->Gt[l], P, rows,
                                                     m->grads + m->off[l] + nw);
        if (l == 0) break;
        // data gradient into layer l's input: (G_l W_l) * GELU'(Z_{l-1})
        GemmArgs d{};
        d.A = l == 4 ? m->G5 : m->G[l];
        d.lda = l == 4 ? kOutPad : kWidth;
        d.a_rows = n;
        d.B = m->Wt[l];
        d.ldb = kOutP[l];
        d.b_rows = kWidth;
        d.K = kOutP[l];
        d.k_split = d.K;
        d.m_valid = n;
        d.gp_in = m->GP[l - 1];
        d.out = m->G[l - 1];
        d.ldo = kWidth;
        d.out_t = m->Gt[l - 1];
        d.ldt = P;
        d.err = m->err;
        d.wait_ns = m->wait_ns;
        d.skip_products = m->skip_products;
        e = gemm<kBwdData, 128>(d, gx, 1, m->stream);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

lskum_status check_err(lskum_mlp *m)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mcuda(m, e, "network kernels");
    if (h) {
        cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
        char buf[96];
        snprintf(buf, sizeof(buf), "tensor-core product did not complete within %.3g s", (double)m->wait_ns * 1e-9);
        return mfail(m, LSKUM_ERR_TIMEOUT, buf);
    }
    return LSKUM_OK;
}

int round_rows(int n)
{
    return std::max(kBatchAlign, (n + kBatchAlign - 1) / kBatchAlign * kBatchAlign);
}

// One training step on rows [0, n) of X/Xt (already filled), targets T via idx.
cudaError_t train_step(lskum_mlp *m, int n, const float *T, const int32_t *idx)
{
    const int rows = round_rows(n);
    cudaError_t e = forward(m, n, rows, true);
    if (e == cudaSuccess) {
        k_loss<<<(rows + 255) / 256, 256, 0, m->stream>>>(m->O, T, idx, n, rows, m->G5, m->G5t, m->P, m->loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward(m, n, rows);
    return e;
}

cudaError_t adam(lskum_mlp *m, float lr)
{
    m->adam_t += 1;
    const double bc1 = 1.0 - std::pow(0.9, m->adam_t), bc2 = 1.0 - std::pow(0.999, m->adam_t);
    k_adam<<<(kNParams + 255) / 256, 256, 0, m->stream>>>(m->params, m->m, m->v, m->grads, kNParams, lr, (float)bc1,
                                                          (float)bc2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = pack(m);
    return e;
}

int g_num_sms = 0;

// Fused forward pass over n rows: from the BF16 input buffer X (outputs to O)
// or from the points [k0, k0 + n) of a context view (state written).
template <int SRC>
cudaError_t fused_forward(lskum_mlp *m, int n, const uint16_t *X, float *O, const lskum::MlpView *v, int k0)
{
    if (n <= 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_fused<SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    FusedArgs a{};
    for (int l = 0; l < kLayers; l++) {
        a.W[l] = m->W[l];
        a.off[l] = m->off[l];
    }
    a.params = m->params;
    a.n = n;
    a.X = X;
    a.O = O;
    if (v) a.v = *v;
    a.k0 = k0;
    a.fourier = m->fourier;
    a.err = m->err;
    a.wait_ns = m->wait_ns;
    a.skip_products = m->skip_products;
    const int tiles = (n + 127) / 128;
    k_mlp_fused<SRC><<<std::min(tiles, g_num_sms), kFusedThreads, kFusedSmem, m->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int32_t lskum_mlp_n_params(void)
{
    return kNParams;
}

lskum_status lskum_mlp_set_wait_test(lskum_mlp *m, int32_t skip_products, double wait_limit_s)
{
    if (!m) return LSKUM_ERR_ARG;
    if ((skip_products != 0 && skip_products != 1) || !(wait_limit_s >= 1e-4 && wait_limit_s <= 10.0))
        return mfail(m, LSKUM_ERR_ARG, "wait test: skip_products 0 or 1, wait_limit_s in [1e-4, 10]");
    m->skip_products = skip_products;
    m->wait_ns = (uint64_t)(wait_limit_s * 1e9);
    return LSKUM_OK;
}

const char *lskum_mlp_last_error(const lskum_mlp *m)
{
    return m ? m->msg.c_str() : g_mlp_create_error.c_str();
}

void lskum_mlp_destroy(lskum_mlp *m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    for (void *p : m->allocs) cudaFree(p);
    if (m->s_in) cudaFree(m->s_in);
    if (m->s_tgt) cudaFree(m->s_tgt);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

lskum_status lskum_mlp_create(uint64_t seed, int32_t max_batch, void *cuda_stream, lskum_mlp **out)
{
    if (!out) return mfail(nullptr, LSKUM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 24)) return mfail(nullptr, LSKUM_ERR_ARG, "max_batch out of range");
    lskum_mlp *m = new (std::nothrow) lskum_mlp();
    if (!m) return mfail(nullptr, LSKUM_ERR_OOM, "host allocation");
    cudaGetDevice(&m->device);
    cudaError_t e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete m;
        return mcuda(nullptr, e, "cudaStreamCreate");
    }
    if (cuda_stream) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, (cudaStream_t)cuda_stream);
            cudaStreamWaitEvent(m->stream, ev, 0);
            cudaEventDestroy(ev);
        }
    }
    m->P = round_rows(max_batch);
    const size_t P = m->P;
    int o = 0;
    for (int l = 0; l < kLayers; l++) {
        m->off[l] = o;
        o += kOutTrue[l] * kInTrue[l] + kOutTrue[l];
    }
    e = cudaSuccess;
    auto A = [&](auto **p, size_t count) {
        if (e == cudaSuccess) e = dalloc(m, p, count);
    };
    A(&m->params, kNParams);
    A(&m->m, kNParams);
    A(&m->v, kNParams);
    A(&m->grads, kNParams);
    A(&m->fourier, 3 * kFreq);
    for (int l = 0; l < kLayers; l++) {
        A(&m->W[l], (size_t)kOutP[l] * kInP[l]);
        A(&m->Wt[l], (size_t)kOutP[l] * kInP[l]);
    }
    A(&m->X, P * kInPad);
    A(&m->Xt, P * kInPad);
    for (int l = 0; l < 4; l++) {
        A(&m->H[l], P * kWidth);
        A(&m->Ht[l], P * kWidth);
        A(&m->G[l], P * kWidth);
        A(&m->Gt[l], P * kWidth);
        A(&m->GP[l], P * kWidth);
    }
    A(&m->G5, P * kOutPad);
    A(&m->G5t, P * kOutPad);
    A(&m->O, P * kOut);
    A(&m->part, (P / kSplitK) * (size_t)kWidth * kWidth);
    A(&m->Xf, P * kIn);
    A(&m->Tf, P * kOut);
    A(&m->loss, 1);
    A(&m->err, 1);
    A(&m->idx, P);
    if (e != cudaSuccess) {
        lskum_mlp_destroy(m);
        return mcuda(nullptr, e, "cudaMalloc");
    }
    // initial parameters and Fourier matrix
    uint64_t s = seed ^ 0x5DEECE66Dull;
    std::vector<float> h(kNParams), B(3 * kFreq);
    for (int l = 0; l < kLayers; l++) {
        const double k = 1.0 / std::sqrt((double)kInTrue[l]);
        const int cnt = kOutTrue[l] * kInTrue[l] + kOutTrue[l];
        for (int i = 0; i < cnt; i++) h[m->off[l] + i] = (float)((2.0 * uniform01(s) - 1.0) * k);
    }
    for (int i = 0; i < 3 * kFreq; i += 2) {  // Box-Muller
        const double u1 = 1.0 - uniform01(s), u2 = uniform01(s);
        const double r = std::sqrt(-2.0 * std::log(u1));
        B[i] = (float)(r * std::cos(2.0 * M_PI * u2));
        B[i + 1] = (float)(r * std::sin(2.0 * M_PI * u2));
    }
    lskum_status st = lskum_mlp_set_params(m, h.data(), B.data());
    if (st != LSKUM_OK) {
        g_mlp_create_error = m->msg;
        lskum_mlp_destroy(m);
        return st;
    }
    *out = m;
    return LSKUM_OK;
}

lskum_status lskum_mlp_get_params(lskum_mlp *m, float *params, float *fourier)
{
    if (!m) return LSKUM_ERR_ARG;
    cudaError_t e = cudaSuccess;
    if (params) e = cudaMemcpyAsync(params, m->params, kNParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (fourier && e == cudaSuccess)
        e = cudaMemcpyAsync(fourier, m->fourier, 3 * kFreq * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LSKUM_OK : mcuda(m, e, "reading the parameters");
}

lskum_status lskum_mlp_set_params(lskum_mlp *m, const float *params, const float *fourier)
{
    if (!m || !params) return m ? mfail(m, LSKUM_ERR_ARG, "params is NULL") : LSKUM_ERR_ARG;
    for (int i = 0; i < kNParams; i++)
        if (!std::isfinite(params[i])) return mfail(m, LSKUM_ERR_ARG, "non-finite parameter");
    cudaError_t e = cudaMemcpyAsync(m->params, params, kNParams * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (fourier && e == cudaSuccess)
        e = cudaMemcpyAsync(m->fourier, fourier, 3 * kFreq * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, kNParams * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, kNParams * sizeof(float), m->stream);
    if (e == cudaSuccess) e = pack(m);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    m->adam_t = 0;
    return e == cudaSuccess ? LSKUM_OK : mcuda(m, e, "writing the parameters");
}

lskum_status lskum_mlp_features(lskum_mlp *m, const float *in5, int32_t n, float *X)
{
    if (!m || n < 0 || (n > 0 && (!in5 || !X))) return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    for (int32_t k0 = 0; k0 < n; k0 += m->P) {
        const int nb = std::min(m->P, n - k0);
        cudaError_t e = cudaMemcpyAsync(m->Xf, in5 + (size_t)k0 * 5, (size_t)nb * 5 * sizeof(float),
                                        cudaMemcpyHostToDevice, m->stream);  // Xf holds >= 5 floats per row
        if (e == cudaSuccess) {
            k_features<<<(nb + 255) / 256, 256, 0, m->stream>>>(m->Xf, nullptr, nb, nb, m->fourier, m->X, nullptr, 0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_inputs_to_f32<<<(nb + 255) / 256, 256, 0, m->stream>>>(m->X, nb, m->Xf);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(X + (size_t)k0 * kIn, m->Xf, (size_t)nb * kIn * sizeof(float), cudaMemcpyDeviceToHost,
                                m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return mcuda(m, e, "features");
    }
    return LSKUM_OK;
}

lskum_status lskum_mlp_forward(lskum_mlp *m, const float *X, int32_t n, float *out)
{
    if (!m || n < 0 || (n > 0 && (!X || !out))) return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    for (int32_t k0 = 0; k0 < n; k0 += m->P) {
        const int nb = std::min(m->P, n - k0);
        const int rows = (nb + 127) / 128 * 128;
        cudaError_t e = cudaMemcpyAsync(m->Xf, X + (size_t)k0 * kIn, (size_t)nb * kIn * sizeof(float),
                                        cudaMemcpyHostToDevice, m->stream);
        if (e == cudaSuccess) {
            k_inputs_from_f32<<<(rows + 255) / 256, 256, 0, m->stream>>>(m->Xf, nb, rows, m->X, nullptr, 0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = fused_forward<kSrcBuffer>(m, nb, m->X, m->O, nullptr, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + (size_t)k0 * kOut, m->O, (size_t)nb * kOut * sizeof(float),
                                cudaMemcpyDeviceToHost, m->stream);
        if (e != cudaSuccess) return mcuda(m, e, "forward");
        lskum_status s = check_err(m);
        if (s != LSKUM_OK) return s;
    }
    return LSKUM_OK;
}

lskum_status lskum_mlp_loss_grads(lskum_mlp *m, const float *X, const float *T, int32_t n, float *loss, float *grads)
{
    if (!m || n < 1 || n > m->P || !X || !T) return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    const int rows = round_rows(n);
    cudaError_t e = cudaMemcpyAsync(m->Xf, X, (size_t)n * kIn * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->Tf, T, (size_t)n * kOut * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
    if (e == cudaSuccess) {
        k_inputs_from_f32<<<(rows + 255) / 256, 256, 0, m->stream>>>(m->Xf, n, rows, m->X, m->Xt, m->P);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = train_step(m, n, m->Tf, nullptr);
    double l = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    if (grads && e == cudaSuccess)
        e = cudaMemcpyAsync(grads, m->grads, kNParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e != cudaSuccess) return mcuda(m, e, "loss and gradients");
    lskum_status s = check_err(m);
    if (s != LSKUM_OK) return s;
    if (loss) *loss = (float)l;
    return LSKUM_OK;
}

lskum_status lskum_mlp_adam(lskum_mlp *m, const float *grads, float lr)
{
    if (!m || !grads || !(lr > 0.f)) return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(m->grads, grads, kNParams * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = adam(m, lr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LSKUM_OK : mcuda(m, e, "Adam step");
}

lskum_status lskum_mlp_time_forward(lskum_mlp *m, int32_t n, int32_t reps, double *ms)
{
    if (!m || n < 1 || reps < 1 || !ms) return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, m->stream);
    for (int r = 0; r < reps && e == cudaSuccess; r++)
        for (int32_t k0 = 0; k0 < n && e == cudaSuccess; k0 += m->P) {
            const int nb = std::min(m->P, n - k0);
            e = fused_forward<kSrcBuffer>(m, nb, m->X, m->O, nullptr, 0);
        }
    if (e == cudaSuccess) e = cudaEventRecord(e1, m->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return mcuda(m, e, "timing the forward pass");
    lskum_status st = check_err(m);
    if (st != LSKUM_OK) return st;
    *ms = (double)t / reps;
    return LSKUM_OK;
}

lskum_status lskum_mlp_n_samples(lskum_mlp *m, int32_t *n)
{
    if (!m || !n) return LSKUM_ERR_ARG;
    *n = m->n_samples;
    return LSKUM_OK;
}

lskum_status lskum_mlp_add_samples(lskum_mlp *m, lskum_ctx *ctx, int32_t per_case, uint64_t seed)
{
    if (!m || !ctx || per_case < 1) return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    lskum::MlpView v{};
    lskum_status st = lskum::ctx_mlp_view(ctx, &v);
    if (st != LSKUM_OK) return mfail(m, st, "context view: " + std::string(lskum_last_error(ctx)));
    std::vector<int32_t> status;
    st = lskum::ctx_case_status(ctx, status);
    if (st != LSKUM_OK) return mfail(m, st, "case status: " + std::string(lskum_last_error(ctx)));
    const lskum::CtxHost h = lskum::ctx_host(ctx);
    // per case, its wall and interior points (internal positions)
    std::vector<std::vector<int32_t>> cand(h.n_cases);
    for (int32_t p = 0; p < h.n; p++)
        if (h.flag[p] != LSKUM_OUTER) cand[h.case_of_caller[p]].push_back(h.inv[p]);
    std::vector<int32_t> pts;
    uint64_t s = seed ^ 0x2545F4914F6CDD1Dull;
    for (int32_t b = 0; b < h.n_cases; b++) {
        if (status[b] != LSKUM_OK) continue;
        auto &c = cand[b];
        const int take = std::min<int>(per_case, (int)c.size());
        for (int i = 0; i < take; i++) {  // partial Fisher-Yates
            const int j = i + (int)(splitmix64(s) % (uint64_t)(c.size() - i));
            std::swap(c[i], c[j]);
            pts.push_back(c[i]);
        }
    }
    if (pts.empty()) return LSKUM_OK;
    const int32_t add = (int32_t)pts.size();
    if ((int64_t)m->n_samples + add > (1 << 28)) return mfail(m, LSKUM_ERR_ARG, "too many samples");
    cudaError_t e = cudaSuccess;
    if (m->n_samples + add > m->cap_samples) {
        const int32_t cap = std::max(m->n_samples + add, 2 * m->cap_samples);
        float *in = nullptr, *tg = nullptr;
        e = cudaMalloc(&in, (size_t)cap * 5 * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&tg, (size_t)cap * 4 * sizeof(float));
        if (e == cudaSuccess && m->n_samples) {
            e = cudaMemcpyAsync(in, m->s_in, (size_t)m->n_samples * 5 * sizeof(float), cudaMemcpyDeviceToDevice,
                                m->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(tg, m->s_tgt, (size_t)m->n_samples * 4 * sizeof(float),
                                    cudaMemcpyDeviceToDevice, m->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) {
            cudaFree(in);
            cudaFree(tg);
            return mcuda(m, e, "sample store");
        }
        cudaFree(m->s_in);
        cudaFree(m->s_tgt);
        m->s_in = in;
        m->s_tgt = tg;
        m->cap_samples = cap;
    }
    int32_t *dpts = nullptr;
    e = cudaMalloc(&dpts, (size_t)add * sizeof(int32_t));
    // the context's stream wrote the state; order after it
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dpts, pts.data(), (size_t)add * sizeof(int32_t), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) {
        k_gather_samples<<<(add + 255) / 256, 256, 0, m->stream>>>(v, dpts, add, m->s_in + (size_t)m->n_samples * 5,
                                                                  m->s_tgt + (size_t)m->n_samples * 4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(dpts);
    if (e != cudaSuccess) return mcuda(m, e, "gathering samples");
    m->n_samples += add;
    return LSKUM_OK;
}

lskum_status lskum_mlp_train(lskum_mlp *m, int32_t epochs, int32_t batch, float lr, uint64_t seed, float *epoch_loss)
{
    if (!m || epochs < 0 || batch < 1 || batch > m->P || !(lr > 0.f))
        return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    if (m->n_samples < 1) return mfail(m, LSKUM_ERR_ARG, "no samples");
    const int32_t S = m->n_samples;
    std::vector<int32_t> perm(S);
    int32_t *dperm = nullptr;
    cudaError_t e = cudaMalloc(&dperm, (size_t)S * sizeof(int32_t));
    if (e != cudaSuccess) return mcuda(m, e, "cudaMalloc(permutation)");
    uint64_t s = seed ^ 0x9E3779B97F4A7C15ull;
    for (int32_t ep = 0; ep < epochs && e == cudaSuccess; ep++) {
        for (int32_t i = 0; i < S; i++) perm[i] = i;
        for (int32_t i = S - 1; i > 0; i--) std::swap(perm[i], perm[(int32_t)(splitmix64(s) % (uint64_t)(i + 1))]);
        e = cudaMemcpyAsync(dperm, perm.data(), (size_t)S * sizeof(int32_t), cudaMemcpyHostToDevice, m->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
        int steps = 0;
        for (int32_t b0 = 0; b0 < S && e == cudaSuccess; b0 += batch, steps++) {
            const int nb = std::min(batch, S - b0);
            const int rows = round_rows(nb);
            k_features<<<(rows + 255) / 256, 256, 0, m->stream>>>(m->s_in, dperm + b0, nb, rows, m->fourier, m->X,
                                                                  m->Xt, m->P);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = train_step(m, nb, m->s_tgt, dperm + b0);
            if (e == cudaSuccess) e = adam(m, lr);
        }
        double l = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (epoch_loss && e == cudaSuccess) epoch_loss[ep] = (float)(l / std::max(steps, 1));
        if (e == cudaSuccess) {
            lskum_status st = check_err(m);
            if (st != LSKUM_OK) {
                cudaFree(dperm);
                return st;
            }
        }
    }
    cudaFree(dperm);
    return e == cudaSuccess ? LSKUM_OK : mcuda(m, e, "training");
}

lskum_status lskum_mlp_predict(lskum_mlp *m, lskum_ctx *ctx, int32_t *warm)
{
    if (!m || !ctx) return m ? mfail(m, LSKUM_ERR_ARG, "bad argument") : LSKUM_ERR_ARG;
    lskum::MlpView v{};
    lskum_status st = lskum::ctx_mlp_view(ctx, &v);
    if (st != LSKUM_OK) return mfail(m, st, "context view: " + std::string(lskum_last_error(ctx)));
    cudaError_t e = cudaStreamSynchronize(v.stream);
    // 1. free stream everywhere, its first residual norm per case
    std::vector<double> n_free, n_warm;
    if (e == cudaSuccess) {
        k_free_stream<<<(v.n + 255) / 256, 256, 0, v.stream>>>(v, nullptr);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return mcuda(m, e, "free stream");
    st = lskum::ctx_state_written(ctx);
    if (st == LSKUM_OK) st = lskum::ctx_case_norms(ctx, n_free);
    if (st != LSKUM_OK) return mfail(m, st, "free-stream residual: " + std::string(lskum_last_error(ctx)));
    // 2. the prediction, chunk by chunk (the network's stream follows the context's)
    st = lskum::ctx_mlp_view(ctx, &v);  // the current state set may have changed
    if (st != LSKUM_OK) return mfail(m, st, "context view");
    e = cudaStreamSynchronize(v.stream);
    if (e == cudaSuccess) e = fused_forward<kSrcView>(m, v.n, nullptr, nullptr, &v, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return mcuda(m, e, "prediction");
    st = check_err(m);
    if (st != LSKUM_OK) return st;
    st = lskum::ctx_state_written(ctx);
    if (st == LSKUM_OK) st = lskum::ctx_case_norms(ctx, n_warm);
    if (st == LSKUM_ERR_NONPOSITIVE) {  // the prediction is not a physical state anywhere: free stream
        n_warm.assign(n_free.size(), INFINITY);
        st = LSKUM_OK;
    } else if (st != LSKUM_OK) {
        return mfail(m, st, "predicted residual: " + std::string(lskum_last_error(ctx)));
    }
    // 3. the residual judges, per case
    const int nc = (int)n_free.size();
    std::vector<uint8_t> keep(nc);
    bool all = true;
    for (int b = 0; b < nc; b++) {
        keep[b] = std::isfinite(n_warm[b]) && n_warm[b] < n_free[b];
        all = all && keep[b];
        if (warm) warm[b] = keep[b];
    }
    if (!all) {
        st = lskum::ctx_mlp_view(ctx, &v);
        if (st != LSKUM_OK) return mfail(m, st, "context view");
        uint8_t *dkeep = nullptr;
        e = cudaMalloc(&dkeep, nc);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dkeep, keep.data(), nc, cudaMemcpyHostToDevice, v.stream);
        if (e == cudaSuccess) {
            k_free_stream<<<(v.n + 255) / 256, 256, 0, v.stream>>>(v, dkeep);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
        cudaFree(dkeep);
        if (e != cudaSuccess) return mcuda(m, e, "fallback to the free stream");
    }
    st = lskum::ctx_state_written(ctx);
    return st == LSKUM_OK ? LSKUM_OK : mfail(m, st, "warm state: " + std::string(lskum_last_error(ctx)));
}

}  // extern "C"

namespace lskum {

cudaError_t launch_wall_distance(const float *x, const float *y, const int32_t *case_of, int32_t n,
                                 const float4 *seg, const int32_t *seg_off, float *dwall, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_wall_distance<<<(n + 255) / 256, 256, 0, s>>>(x, y, case_of, n, seg, seg_off, dwall);
    return cudaGetLastError();
}

}  // namespace lskum
