// Learned surrogate of the outer volume: a small MLP that predicts the empty
// fraction of a box from its parameters and an 8^3 occupancy patch sampled in
// the box's own frame.  The partition rounds of the Lloyd step use it to keep
// only the most promising candidate moves per cluster; the exact lattice count
// still decides every accepted move.
//
// Features (524 per box), from the quantised box alone, FP64 with a fixed
// operation order (so the patch bits are reproducible):
//   Lq, Hq = ceil(lo / 256), floor(hi / 256); M = n (3x3), M^-1 by cofactors;
//   sample s in {0..7}^3: v_a = Lq_a + (Hq_a - Lq_a) (2 s_a + 1) / 16,
//   p = M^-1 v, index = floor(p + 1/2), bit = occupancy (0 outside [0, N)^3);
//   box parameters: centre M^-1 (Lq + Hq) / 2 / N, axes n_0 / |n_0|, n_1 / |n_1|,
//   half widths (Hq_a - Lq_a) / (2 |n_a|) / N.
// Network: 524 -> 128 -> 128 -> 128 -> 1, ReLU, sigmoid output (the empty
// fraction); predicted outer volume = fraction x box volume in lattice cells
// (prod (Hq_a - Lq_a + 1) / |det M|).  Training: mean squared error on the
// fraction, Adam, FP32 master weights; inference reads an FP16 copy of the
// weights and accumulates in FP32.  The contraction is 100k multiply-adds per
// box on a few thousand boxes, so it runs on CUDA cores (tiled GEMM in shared
// memory), not tensor cores.
#include <cuda_fp16.h>

#include <cmath>
#include <random>
#include <vector>

#include "internal.h"

namespace obbv {
namespace {

constexpr int kIn = kSurrogateInputs;
constexpr int kH = 128;

// parameter offsets in the flat vector: W1 b1 W2 b2 W3 b3 W4 b4 (W row-major [in][out])
constexpr int64_t oW1 = 0, oB1 = oW1 + (int64_t)kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
                  oB3 = oW3 + kH * kH, oW4 = oB3 + kH, oB4 = oW4 + kH, kParams = oB4 + 1;

// ---------------------------------------------------------------- features

__global__ void k_features(const obb_qbox* __restrict__ boxes, const int32_t* __restrict__ d_K,
                           const uint64_t* __restrict__ words, int32_t N, int32_t W, float* __restrict__ feats)
{
    const int64_t b = blockIdx.x;
    if (b >= *d_K) return;
    // Per box, once: the exact adjugate A of the normals (n^-1 = A / det) in
    // int64 and det in 128 bits, then FP32 with one rounding per operation in
    // a fixed order (explicit _rn intrinsics: nothing is fused).  Integers
    // reach FP32 as two 32-bit halves joined by one fmaf.
    __shared__ float sh_c[3], sh_E[9];
    float* f = feats + b * (int64_t)kIn;
    if (threadIdx.x == 0) {
        const obb_qbox q = boxes[b];
        int64_t m[9], L[3], H[3];
        for (int i = 0; i < 9; ++i) m[i] = q.n[i];
        for (int a = 0; a < 3; ++a) {
            L[a] = -((-q.b[2 * a]) >> kS);
            H[a] = q.b[2 * a + 1] >> kS;
        }
        const int64_t A[9] = {m[4] * m[8] - m[5] * m[7], m[2] * m[7] - m[1] * m[8], m[1] * m[5] - m[2] * m[4],
                              m[5] * m[6] - m[3] * m[8], m[0] * m[8] - m[2] * m[6], m[2] * m[3] - m[0] * m[5],
                              m[3] * m[7] - m[4] * m[6], m[1] * m[6] - m[0] * m[7], m[0] * m[4] - m[1] * m[3]};
        const __int128 det = (__int128)m[0] * A[0] + (__int128)m[1] * A[3] + (__int128)m[2] * A[6];
        const float detf = i128_to_float(det);
        float Af[9], Sf[3], Df[3];
        for (int i = 0; i < 9; ++i) Af[i] = i64_to_float(A[i]);
        for (int a = 0; a < 3; ++a) {
            Sf[a] = i64_to_float(L[a] + H[a]);
            Df[a] = i64_to_float(H[a] - L[a]);
        }
        for (int r = 0; r < 3; ++r) {
            float c = 0.0f;
            if (det != 0) {
                // index-space centre: ((A_r0 S_0 + A_r1 S_1) + A_r2 S_2) / (2 det)
                const float t = __fadd_rn(__fadd_rn(__fmul_rn(Af[3 * r], Sf[0]), __fmul_rn(Af[3 * r + 1], Sf[1])),
                                          __fmul_rn(Af[3 * r + 2], Sf[2]));
                c = __fdiv_rn(t, __fmul_rn(2.0f, detf));
            }
            sh_c[r] = c;
            f[r] = __fdiv_rn(c, (float)N);
            // edge a of the box in index space: (A_ra D_a) / det
            for (int a = 0; a < 3; ++a)
                sh_E[3 * r + a] = det != 0 ? __fdiv_rn(__fmul_rn(Af[3 * r + a], Df[a]), detf) : 0.0f;
        }
        for (int a = 0; a < 3; ++a) {
            const float n0 = (float)q.n[3 * a], n1 = (float)q.n[3 * a + 1], n2 = (float)q.n[3 * a + 2];
            const float nn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(n0, n0), __fmul_rn(n1, n1)), __fmul_rn(n2, n2)));
            if (a < 2) {
                f[3 + 3 * a] = nn > 0.0f ? __fdiv_rn(n0, nn) : 0.0f;
                f[4 + 3 * a] = nn > 0.0f ? __fdiv_rn(n1, nn) : 0.0f;
                f[5 + 3 * a] = nn > 0.0f ? __fdiv_rn(n2, nn) : 0.0f;
            }
            f[9 + a] = nn > 0.0f ? __fdiv_rn(__fdiv_rn(__fmul_rn(Df[a], 0.5f), nn), (float)N) : 0.0f;
        }
    }
    __syncthreads();
    const float c0 = sh_c[0], c1 = sh_c[1], c2 = sh_c[2];
    float E[9];
    for (int i = 0; i < 9; ++i) E[i] = sh_E[i];
    // patch point s: the centre plus the edges times g_a = (2 s_a - 7) / 16,
    // ((c_r + E_r0 g_0) + E_r1 g_1) + E_r2 g_2, rounded to the nearest lattice
    // point (floor(p + 1/2)); the bit is 0 outside the lattice
    for (int s = threadIdx.x; s < 512; s += blockDim.x) {
        const float g0 = __fmul_rn((float)(2 * (s & 7) - 7), 0.0625f);
        const float g1 = __fmul_rn((float)(2 * ((s >> 3) & 7) - 7), 0.0625f);
        const float g2 = __fmul_rn((float)(2 * (s >> 6) - 7), 0.0625f);
        const float cr[3] = {c0, c1, c2};
        int32_t idx[3];
        for (int r = 0; r < 3; ++r) {
            const float p = __fadd_rn(__fadd_rn(__fadd_rn(cr[r], __fmul_rn(E[3 * r], g0)), __fmul_rn(E[3 * r + 1], g1)),
                                      __fmul_rn(E[3 * r + 2], g2));
            const float qf = floorf(__fadd_rn(p, 0.5f));
            idx[r] = fabsf(qf) < 1e9f ? (int32_t)qf : -1;
        }
        float bit = 0.f;
        if (idx[0] >= 0 && idx[0] < N && idx[1] >= 0 && idx[1] < N && idx[2] >= 0 && idx[2] < N) {
            const uint64_t w = words[((int64_t)idx[2] * N + idx[1]) * W + (idx[0] >> 6)];
            bit = (float)((w >> (idx[0] & 63)) & 1ull);
        }
        f[12 + s] = bit;
    }
}


// ------------------------------------------------------ tensor-core forward
//
// Inference of the screening network on the 5th-generation tensor cores: one
// CTA (4 warps) carries 128 boxes through all four layers.  Operands are FP16
// in shared memory in the canonical K-major layout without swizzle (8 x 8
// "core matrices" of 128 contiguous bytes: core (r / 8, c / 8) of a tile with
// C columns at ((r / 8) (C / 8) + c / 8) * 128 bytes, so the leading (K)
// byte offset is 128 and the stride (M/N) byte offset C * 16).  One thread
// issues tcgen05.mma (kind::f16, M = N = 128, K = 16 per instruction, FP32
// accumulator in 128 TMEM columns) and commits to an mbarrier; every thread
// then reads its own row of the accumulator (TMEM lane = box) with
// tcgen05.ld, adds the bias, applies ReLU and writes FP16 back as the next
// layer's A operand.  The 128 -> 1 output layer is a dot product per row in
// registers.  Every wait is bounded; a CTA that allocated TMEM frees it on
// every path.

constexpr int kTcRows = 128;                    // boxes per CTA (= TMEM lanes)
constexpr int kTcK1 = 576;                      // layer-1 K (524 features) padded to chunks of 64
constexpr int kTcChunk = 64;                    // layer-1 K per staged chunk
constexpr uint32_t kTcCols = 128;               // TMEM columns (one FP32 accumulator)
// instruction descriptor: D = FP32 (bits 4-5), A = B = FP16 (bits 7-12 zero),
// both K-major (bits 15, 16 zero), N / 8 at bits 17-22, M / 16 at bits 24-28
constexpr uint32_t kTcIdesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint64_t kTcWaitNs = 250000000ull;    // a wait gives up after 250 ms (device global timer)

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (>> 4), descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// byte offset of element (r, c) in a K-major no-swizzle tile of C columns
__device__ __forceinline__ uint32_t tc_off(int r, int c, int C)
{
    return (uint32_t)((((r >> 3) * (C >> 3) + (c >> 3)) << 7) + ((r & 7) << 4) + ((c & 7) << 1));
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// wait for the given phase of the mbarrier; false once kTcWaitNs have passed
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t phase)
{
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(phase)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kTcWaitNs) return false;
    }
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void tc_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }


// bulk copy (TMA, untiled) of `bytes` from global to shared memory, completing
// on `bar` (16-byte aligned addresses, a multiple of 16 bytes)
__device__ __forceinline__ void tc_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// FP16 weights, transposed (N x K, K-major) and laid out as the kernel's shared
// tiles: W1 as 9 chunks of 128 x 64 (K zero-padded to 576), then W2, W3 as
// 128 x 128 tiles
constexpr int64_t kTcW1Chunk = (int64_t)kH * kTcChunk;               // halves per W1 chunk
constexpr int64_t kTcPacked = (kTcK1 / kTcChunk) * kTcW1Chunk + 2 * (int64_t)kH * kH;

__global__ void k_pack_tc(const __half* __restrict__ wh, __half* __restrict__ wtc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n1 = (int64_t)kH * kTcK1;
    if (i < n1) {
        const int n = (int)(i % kH), k = (int)(i / kH);
        const int q = k / kTcChunk, c = k % kTcChunk;
        wtc[q * kTcW1Chunk + tc_off(n, c, kTcChunk) / 2] = k < kIn ? wh[oW1 + (int64_t)k * kH + n] : __float2half_rn(0.f);
    } else if (i < n1 + 2 * (int64_t)kH * kH) {
        const int64_t j = i - n1;
        const int layer = (int)(j / ((int64_t)kH * kH));
        const int e = (int)(j % ((int64_t)kH * kH));
        const int n = e % kH, c = e / kH;
        const int64_t base = (kTcK1 / kTcChunk) * kTcW1Chunk + layer * (int64_t)kH * kH;
        wtc[base + tc_off(n, c, kH) / 2] = wh[(layer == 0 ? oW2 : oW3) + (int64_t)c * kH + n];
    }
}

constexpr int kTcSmem = 65536 + (4 * kH + 4) * 4;   // A and B tiles, biases, w4, b4

// y = sigmoid(W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4) for rows
// [128 blockIdx.x, +128) of X (the live row count is *d_M when given)
__global__ void __launch_bounds__(kTcRows) k_mlp_tc(const float* __restrict__ X, int M, const int32_t* __restrict__ d_M,
                                                    const __half* __restrict__ wtc, const __half* __restrict__ wh,
                                                    const float* __restrict__ w, float* __restrict__ y,
                                                    int32_t* __restrict__ err, int32_t stall)
{
    // stall (test hook): the first MMA group is neither issued nor committed,
    // so its wait can only give up; nothing is left in flight
    if (d_M) M = min(M, *d_M);
    const int m0 = blockIdx.x * kTcRows;
    if (m0 >= M) return;   // uniform: the whole CTA leaves before any TMEM or barrier use
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sA = tc_smem;            // A operand: layer-1 chunk (128 x 64), then h (128 x 128)
    unsigned char* sB = tc_smem + 32768;    // B operand: W^T tile
    float* sBias = reinterpret_cast<float*>(tc_smem + 65536);   // b1, b2, b3, w4 (4 x 128), b4
    __shared__ __align__(8) uint64_t bar_mma, bar_ld;
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < kH; i += kTcRows) {
        sBias[i] = w[oB1 + i];
        sBias[kH + i] = w[oB2 + i];
        sBias[2 * kH + i] = w[oB3 + i];
        sBias[3 * kH + i] = __half2float(wh[oW4 + i]);
    }
    if (t == 0) {
        sBias[4 * kH] = w[oB4];
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_mma)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_ld)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t aS = smem_addr(sA), bS = smem_addr(sB);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 TMEM lanes
    uint32_t ph_mma = 0, ph_ld = 0;
    bool ok = true;

    // layer 1: the W1 chunk arrives by bulk copy while the threads convert
    // their rows' features to FP16 (16-byte stores of 8 consecutive K)
    for (int q = 0; q < kTcK1 / kTcChunk && ok; ++q) {
        const int k0 = q * kTcChunk;
        if (t == 0) tc_bulk_load(sB, wtc + q * kTcW1Chunk, (uint32_t)(kTcW1Chunk * 2), &bar_ld);
        for (int i = t; i < kTcRows * (kTcChunk / 8); i += kTcRows) {
            const int r = i / (kTcChunk / 8), g = i % (kTcChunk / 8);
            const int m = m0 + r, k = k0 + 8 * g;
            __align__(16) __half hv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                hv[e] = __float2half_rn((m < M && k + e < kIn) ? X[(int64_t)m * kIn + k + e] : 0.f);
            *reinterpret_cast<uint4*>(sA + tc_off(r, 8 * g, kTcChunk)) = *reinterpret_cast<const uint4*>(hv);
        }
        tc_fence_smem();
        const bool got = tc_wait(&bar_ld, ph_ld);
        ph_ld ^= 1;
        tc_fence_before();
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        if (t == 0 && !(stall && q == 0)) {
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < kTcChunk / 16; ++j)
                tc_mma(tmem, tc_desc(aS + 256 * j, 128, kTcChunk * 16), tc_desc(bS + 256 * j, 128, kTcChunk * 16),
                       (q > 0 || j > 0) ? 1u : 0u);
            tc_commit(&bar_mma);
        }
        ok = __syncthreads_and(tc_wait(&bar_mma, ph_mma));
        ph_mma ^= 1;
    }

    // layers 2 and 3: the accumulator row of this thread (TMEM lane = row)
    // becomes FP16 h in the A tile; W^T arrives by bulk copy
    for (int layer = 0; layer < 2 && ok; ++layer) {
        if (t == 0)
            tc_bulk_load(sB, wtc + (kTcK1 / kTcChunk) * kTcW1Chunk + layer * (int64_t)kH * kH,
                         (uint32_t)(kH * kH * 2), &bar_ld);
        tc_fence_after();
        for (int c = 0; c < kH / 32; ++c) {
            float v[32];
            tc_ld32(lane_base + 32 * c, v);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                __align__(16) __half hv[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) hv[e] = __float2half_rn(fmaxf(v[8 * g + e] + sBias[layer * kH + 32 * c + 8 * g + e], 0.f));
                *reinterpret_cast<uint4*>(sA + tc_off(t, 32 * c + 8 * g, kH)) = *reinterpret_cast<const uint4*>(hv);
            }
        }
        tc_fence_smem();
        const bool got = tc_wait(&bar_ld, ph_ld);
        ph_ld ^= 1;
        tc_fence_before();
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < kH / 16; ++j)
                tc_mma(tmem, tc_desc(aS + 256 * j, 128, kH * 16), tc_desc(bS + 256 * j, 128, kH * 16), j > 0 ? 1u : 0u);
            tc_commit(&bar_mma);
        }
        ok = __syncthreads_and(tc_wait(&bar_mma, ph_mma));
        ph_mma ^= 1;
    }

    if (ok) {
        // output layer: relu(h3) . w4 + b4 per row, then the sigmoid
        tc_fence_after();
        float acc = sBias[4 * kH];
        for (int c = 0; c < kH / 32; ++c) {
            float v[32];
            tc_ld32(lane_base + 32 * c, v);
#pragma unroll
            for (int e = 0; e < 32; ++e)
                acc = fmaf(fmaxf(v[e] + sBias[2 * kH + 32 * c + e], 0.f), sBias[3 * kH + 32 * c + e], acc);
        }
        const int m = m0 + t;
        if (m < M) y[m] = 1.f / (1.f + __expf(-acc));
    } else {
        // a wait gave up: report it, let in-flight tensor-core work and copies
        // finish (bounded), then free TMEM below
        if (t == 0) atomicOr(err, kErrTimeout);
        tc_wait(&bar_mma, ph_mma ^ 1);
        tc_wait(&bar_ld, ph_ld ^ 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// box volume in lattice cells: prod (Hq_a - Lq_a + 1) / |det n|
__device__ __forceinline__ float box_cells(const obb_qbox& q)
{
    double M[9];
    for (int i = 0; i < 9; ++i) M[i] = (double)q.n[i];
    const double det = M[0] * (M[4] * M[8] - M[5] * M[7]) + M[1] * (M[5] * M[6] - M[3] * M[8]) +
                       M[2] * (M[3] * M[7] - M[4] * M[6]);
    double v = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double w = (double)((q.b[2 * a + 1] >> kS) - (-((-q.b[2 * a]) >> kS)) + 1);
        v *= w > 0.0 ? w : 0.0;
    }
    return det != 0.0 ? (float)(v / fabs(det)) : 0.f;
}

// ---------------------------------------------------------------- GEMM

// C[m][n] = act(sum_k A(m, k) B(k, n) + bias[n]) (* (mask[m][n] > 0)), with
// A(m, k) = A[m sAm + k sAk], B(k, n) = B[k sBk + n sBn]; rows m >= *d_M
// (when given) are skipped.  act: 0 none, 1 ReLU, 2 sigmoid.  Tiles 64 x 64,
// 256 threads, 4 x 4 outputs per thread, K in steps of 16 through shared memory.
template <typename TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int64_t sAm,
                                              int64_t sAk, const TB* __restrict__ B, int64_t sBk, int64_t sBn,
                                              float* __restrict__ C, int64_t ldc, const float* __restrict__ bias,
                                              int act, const float* __restrict__ mask, int64_t ldm,
                                              const int32_t* __restrict__ d_M)
{
    if (d_M) M = min(M, *d_M);
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    if (m0 >= M) return;
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        // A is read along its contiguous index (k when sAk = 1, else m) and B
        // along n, so the loads coalesce; the padded rows of the shared tiles
        // keep the transposed stores free of bank conflicts
        if (sAk == 1) {
            for (int i = threadIdx.x; i < 16 * 64; i += 256) {
                const int mm = i >> 4, kk = i & 15;
                const int m = m0 + mm, k = k0 + kk;
                As[kk][mm] = (m < M && k < K) ? A[m * sAm + k] : 0.f;
            }
        } else {
            for (int i = threadIdx.x; i < 16 * 64; i += 256) {
                const int kk = i >> 6, mm = i & 63;
                const int m = m0 + mm, k = k0 + kk;
                As[kk][mm] = (m < M && k < K) ? A[m * sAm + k * sAk] : 0.f;
            }
        }
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = i >> 6, nn = i & 63;
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < K) ? (float)B[k * sBk + n * sBn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                bb[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j] + (bias ? bias[n] : 0.f);
            if (mask && !(mask[m * ldm + n] > 0.f)) v = 0.f;
            if (act == 1) v = fmaxf(v, 0.f);
            else if (act == 2) v = 1.f / (1.f + __expf(-v));
            C[m * ldc + n] = v;
        }
    }
}

// column sums: out[n] = sum_m X[m][n] (bias gradients)
__global__ void k_colsum(const float* __restrict__ X, int M, int N, float* __restrict__ out)
{
    const int n = blockIdx.x;
    float s = 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += X[(int64_t)m * N + n];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        out[n] = t;
    }
}

// dY = 2 (y - t) / B * y (1 - y); loss partial sums
__global__ void k_out_grad(const float* __restrict__ y, const float* __restrict__ t, int B, float* __restrict__ dy,
                           float* __restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < B) {
        const float e = y[i] - t[i];
        dy[i] = 2.f * e / (float)B * y[i] * (1.f - y[i]);
        l = e * e / (float)B;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __half* __restrict__ wh, int64_t n, float lr, float b1t, float b2t)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - b1t), vh = vi / (1.f - b2t);
    const float wi = w[i] - lr * mh / (sqrtf(vh) + eps);
    w[i] = wi;
    wh[i] = __float2half_rn(wi);
}

__global__ void k_to_half(const float* __restrict__ w, __half* __restrict__ wh, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) wh[i] = __float2half_rn(w[i]);
}

// predicted outer volume = fraction x cells
__global__ void k_pred_obv(const float* __restrict__ frac, const obb_qbox* __restrict__ boxes,
                           const int32_t* __restrict__ d_K, float* __restrict__ pred)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *d_K) return;
    pred[i] = frac[i] * box_cells(boxes[i]);
}

// training target = exact outer volume / the same cell volume the screen scales by, in [0, 1]
__global__ void k_targets(const uint64_t* __restrict__ counts, const obb_qbox* __restrict__ boxes, int64_t K,
                          float* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= K) return;
    const float cells = box_cells(boxes[i]);
    const float t = cells > 0.f ? (float)counts[i] / cells : 0.f;
    out[i] = fminf(fmaxf(t, 0.f), 1.f);
}

template <typename TB>
void gemm(obb_ctx* ctx, int M, int N, int K, const float* A, int64_t sAm, int64_t sAk, const TB* B, int64_t sBk,
          int64_t sBn, float* C, int64_t ldc, const float* bias, int act, const float* mask, int64_t ldm,
          const int32_t* d_M)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<TB><<<grid, 256, 0, ctx->stream>>>(M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc, bias, act, mask, ldm, d_M);
    note_launch(ctx);
}

}  // namespace

struct MlpImpl {
    float* w = nullptr;    // FP32 master weights
    __half* wh = nullptr;  // FP16 inference copy
    __half* wtc = nullptr; // the FP16 weights transposed into the tensor-core kernel's shared tiles
    float* g = nullptr;    // gradients
    float* m = nullptr;    // Adam moments
    float* v = nullptr;
    int64_t step = 0;
    int64_t cap = 0;       // batch capacity of the activation buffers
    float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *y = nullptr, *d1 = nullptr, *d2 = nullptr, *d3 = nullptr,
          *dy = nullptr, *loss = nullptr;
};

}  // namespace obbv

struct obb_mlp {
    obb_ctx* ctx = nullptr;
    obbv::MlpImpl* p = nullptr;
};

namespace obbv {

// the context a network was created in (the entry points of other units
// check ownership through this; the type is complete only here)
const obb_ctx* mlp_owner(const obb_mlp* m) { return m ? m->ctx : nullptr; }

static obb_status mlp_reserve(obb_ctx* ctx, MlpImpl* P, int64_t B)
{
    if (B <= P->cap) return OBB_OK;
    cudaStream_t s = ctx->stream;
    float** bufs[] = {&P->h1, &P->h2, &P->h3, &P->d1, &P->d2, &P->d3};
    for (float** b : bufs) {
        if (*b) cudaFreeAsync(*b, s);
        OBB_CK(ctx, pool_alloc((void**)b, sizeof(float) * kH * B, s));
    }
    if (P->y) cudaFreeAsync(P->y, s);
    if (P->dy) cudaFreeAsync(P->dy, s);
    OBB_CK(ctx, pool_alloc((void**)&P->y, sizeof(float) * B, s));
    OBB_CK(ctx, pool_alloc((void**)&P->dy, sizeof(float) * B, s));
    P->cap = B;
    return OBB_OK;
}

// forward pass into P->h1..h3, P->y (fraction); FP32 or FP16 weights
static void mlp_forward(obb_ctx* ctx, const MlpImpl* P, const float* X, int B, const int32_t* d_B, bool half)
{
    if (half) {
        // all four layers in one tensor-core kernel (FP16 operands, FP32 accumulators)
        cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        const int32_t stall = (ctx->inject & OBB_INJECT_TC_STALL) ? 1 : 0;
        ctx->inject &= ~OBB_INJECT_TC_STALL;   // one launch only
        k_mlp_tc<<<(unsigned)((B + kTcRows - 1) / kTcRows), kTcRows, kTcSmem, ctx->stream>>>(X, B, d_B, P->wtc, P->wh,
                                                                                           P->w, P->y, ctx->d_err, stall);
        note_launch(ctx);
    } else {
        const float* w = P->w;
        gemm<float>(ctx, B, kH, kIn, X, kIn, 1, w + oW1, kH, 1, P->h1, kH, w + oB1, 1, nullptr, 0, d_B);
        gemm<float>(ctx, B, kH, kH, P->h1, kH, 1, w + oW2, kH, 1, P->h2, kH, w + oB2, 1, nullptr, 0, d_B);
        gemm<float>(ctx, B, kH, kH, P->h2, kH, 1, w + oW3, kH, 1, P->h3, kH, w + oB3, 1, nullptr, 0, d_B);
        gemm<float>(ctx, B, 1, kH, P->h3, kH, 1, w + oW4, 1, 1, P->y, 1, w + oB4, 2, nullptr, 0, d_B);
    }
}

// loss and gradients (FP32 weights) into P->g; loss into P->loss (device)
static obb_status mlp_backward(obb_ctx* ctx, MlpImpl* P, const float* X, const float* T, int B)
{
    cudaStream_t s = ctx->stream;
    mlp_forward(ctx, P, X, B, nullptr, false);
    OBB_CK(ctx, cudaMemsetAsync(P->loss, 0, sizeof(float), s));
    k_out_grad<<<(B + 255) / 256, 256, 0, s>>>(P->y, T, B, P->dy, P->loss);
    note_launch(ctx);
    float* g = P->g;
    const float* w = P->w;
    // layer 4: dW4 = H3^T dY, db4 = sum dY, dH3 = dY W4^T * (H3 > 0)
    gemm<float>(ctx, kH, 1, B, P->h3, 1, kH, P->dy, 1, 1, g + oW4, 1, nullptr, 0, nullptr, 0, nullptr);
    k_colsum<<<1, 256, 0, s>>>(P->dy, B, 1, g + oB4);
    note_launch(ctx);
    gemm<float>(ctx, B, kH, 1, P->dy, 1, 1, w + oW4, 1, 1, P->d3, kH, nullptr, 0, P->h3, kH, nullptr);
    // layer 3
    gemm<float>(ctx, kH, kH, B, P->h2, 1, kH, P->d3, kH, 1, g + oW3, kH, nullptr, 0, nullptr, 0, nullptr);
    k_colsum<<<kH, 256, 0, s>>>(P->d3, B, kH, g + oB3);
    note_launch(ctx);
    gemm<float>(ctx, B, kH, kH, P->d3, kH, 1, w + oW3, 1, kH, P->d2, kH, nullptr, 0, P->h2, kH, nullptr);
    // layer 2
    gemm<float>(ctx, kH, kH, B, P->h1, 1, kH, P->d2, kH, 1, g + oW2, kH, nullptr, 0, nullptr, 0, nullptr);
    k_colsum<<<kH, 256, 0, s>>>(P->d2, B, kH, g + oB2);
    note_launch(ctx);
    gemm<float>(ctx, B, kH, kH, P->d2, kH, 1, w + oW2, 1, kH, P->d1, kH, nullptr, 0, P->h1, kH, nullptr);
    // layer 1
    gemm<float>(ctx, kIn, kH, B, X, 1, kIn, P->d1, kH, 1, g + oW1, kH, nullptr, 0, nullptr, 0, nullptr);
    k_colsum<<<kH, 256, 0, s>>>(P->d1, B, kH, g + oB1);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

obb_status surrogate_predict(obb_ctx* ctx, const obb_mlp* mlp, const obb_lattice* lat, const obb_qbox* d_boxes,
                             const int32_t* d_K, int64_t cap, float* d_feats, float* d_pred)
{
    MlpImpl* P = mlp->p;
    OBB_TRY(mlp_reserve(ctx, P, cap));
    k_features<<<(unsigned)cap, 128, 0, ctx->stream>>>(d_boxes, d_K, lat->d_words, lat->frame.N, lat->frame.W,
                                                       d_feats);
    note_launch(ctx);
    mlp_forward(ctx, P, d_feats, (int)cap, d_K, true);
    k_pred_obv<<<(unsigned)((cap + 255) / 256), 256, 0, ctx->stream>>>(P->y, d_boxes, d_K, d_pred);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

}  // namespace obbv

using namespace obbv;

namespace {
template <class T>
obb_status dev_in(obb_ctx* ctx, const T* src, size_t n, int on_device, void** hold, const T** out)
{
    if (on_device) {
        *out = src;
        return OBB_OK;
    }
    OBB_CK(ctx, pool_alloc(hold, sizeof(T) * n, ctx->stream));
    OBB_CK(ctx, cudaMemcpyAsync(*hold, src, sizeof(T) * n, cudaMemcpyHostToDevice, ctx->stream));
    *out = static_cast<const T*>(*hold);
    return OBB_OK;
}
}  // namespace

extern "C" {

obb_status obb_mlp_create(obb_ctx* ctx, uint64_t seed, obb_mlp** out)
{
    if (!ctx || !out) return fail(ctx, OBB_ERR_ARG, "null argument");
    *out = nullptr;
    // He-uniform initial weights from a seeded host generator, zero biases
    std::vector<float> w(kParams, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int64_t off, int fan_in, int64_t count) {
        std::uniform_real_distribution<float> U(-std::sqrt(6.f / fan_in), std::sqrt(6.f / fan_in));
        for (int64_t i = 0; i < count; ++i) w[off + i] = U(rng);
    };
    fill(oW1, kIn, (int64_t)kIn * kH);
    fill(oW2, kH, (int64_t)kH * kH);
    fill(oW3, kH, (int64_t)kH * kH);
    fill(oW4, kH, kH);
    obb_mlp* m = new obb_mlp();
    m->ctx = ctx;
    m->p = new MlpImpl();
    MlpImpl* P = m->p;
    cudaStream_t s = ctx->stream;
    cudaError_t e = pool_alloc((void**)&P->w, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&P->wh, sizeof(__half) * kParams, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&P->wtc, sizeof(__half) * kTcPacked, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&P->g, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&P->m, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&P->v, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&P->loss, sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->w, w.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->m, 0, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->v, 0, sizeof(float) * kParams, s);
    if (e == cudaSuccess) {
        k_to_half<<<(unsigned)((kParams + 255) / 256), 256, 0, s>>>(P->w, P->wh, kParams);
        k_pack_tc<<<(unsigned)((kTcPacked + 255) / 256), 256, 0, s>>>(P->wh, P->wtc);
        note_launch(ctx, 2);
        e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        obb_mlp_free(m);
        return cuda_fail(ctx, e, "surrogate allocation");
    }
    *out = m;
    return OBB_OK;
}

void obb_mlp_free(obb_mlp* m)
{
    if (!m) return;
    cudaStream_t s = m->ctx ? m->ctx->stream : nullptr;
    if (m->p) {
        MlpImpl* P = m->p;
        void* ptrs[] = {P->w, P->wh, P->wtc, P->g, P->m, P->v, P->h1, P->h2, P->h3, P->y, P->d1, P->d2, P->d3, P->dy, P->loss};
        for (void* q : ptrs)
            if (q) cudaFreeAsync(q, s);
        delete P;
    }
    delete m;
}

int64_t obb_mlp_num_params(void) { return kParams; }

obb_status obb_mlp_params(obb_ctx* ctx, const obb_mlp* m, float* out, int32_t on_device)
{
    if (!ctx || !m || !out) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (m->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "network belongs to another context");
    OBB_CK(ctx, cudaMemcpyAsync(out, m->p->w, sizeof(float) * kParams,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    return on_device ? OBB_OK : check_device_error(ctx);
}

obb_status obb_mlp_set_params(obb_ctx* ctx, obb_mlp* m, const float* in, int32_t on_device)
{
    if (!ctx || !m || !in) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (m->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "network belongs to another context");
    MlpImpl* P = m->p;
    OBB_CK(ctx, cudaMemcpyAsync(P->w, in, sizeof(float) * kParams,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    k_to_half<<<(unsigned)((kParams + 255) / 256), 256, 0, ctx->stream>>>(P->w, P->wh, kParams);
    k_pack_tc<<<(unsigned)((kTcPacked + 255) / 256), 256, 0, ctx->stream>>>(P->wh, P->wtc);
    note_launch(ctx);
    note_launch(ctx);
    OBB_CK(ctx, cudaMemsetAsync(P->m, 0, sizeof(float) * kParams, ctx->stream));
    OBB_CK(ctx, cudaMemsetAsync(P->v, 0, sizeof(float) * kParams, ctx->stream));
    P->step = 0;
    return check_device_error(ctx);
}

obb_status obb_surrogate_features(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* boxes, int64_t K, float* feats,
                                  int32_t on_device)
{
    if (!ctx || !lat || (K > 0 && (!boxes || !feats))) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    if (K <= 0) return OBB_OK;
    void* hb = nullptr;
    const obb_qbox* db;
    OBB_TRY(dev_in(ctx, boxes, (size_t)K, on_device, &hb, &db));
    float* df = feats;
    if (!on_device) OBB_CK(ctx, pool_alloc((void**)&df, sizeof(float) * kIn * K, ctx->stream));
    OBB_CK(ctx, ctx->kdev.reserve(sizeof(int32_t), ctx->stream));
    OBB_TRY(set_device_int(ctx, ctx->kdev.as<int32_t>(), (int32_t)K));
    k_features<<<(unsigned)K, 128, 0, ctx->stream>>>(db, ctx->kdev.as<int32_t>(), lat->d_words, lat->frame.N,
                                                     lat->frame.W, df);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    if (!on_device) {
        OBB_CK(ctx, cudaMemcpyAsync(feats, df, sizeof(float) * kIn * K, cudaMemcpyDeviceToHost, ctx->stream));
        cudaFreeAsync(df, ctx->stream);
    }
    if (hb) cudaFreeAsync(hb, ctx->stream);
    return on_device ? OBB_OK : check_device_error(ctx);
}

obb_status obb_surrogate_targets(obb_ctx* ctx, const obb_qbox* boxes, const uint64_t* counts, int64_t K, float* out,
                                 int32_t on_device)
{
    if (!ctx || (K > 0 && (!boxes || !counts || !out))) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (K <= 0) return OBB_OK;
    void *hb = nullptr, *hc = nullptr;
    const obb_qbox* db;
    const uint64_t* dc;
    OBB_TRY(dev_in(ctx, boxes, (size_t)K, on_device, &hb, &db));
    OBB_TRY(dev_in(ctx, counts, (size_t)K, on_device, &hc, &dc));
    float* dout = out;
    if (!on_device) OBB_CK(ctx, pool_alloc((void**)&dout, sizeof(float) * K, ctx->stream));
    k_targets<<<(unsigned)((K + 255) / 256), 256, 0, ctx->stream>>>(dc, db, K, dout);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    if (!on_device) {
        OBB_CK(ctx, cudaMemcpyAsync(out, dout, sizeof(float) * K, cudaMemcpyDeviceToHost, ctx->stream));
        cudaFreeAsync(dout, ctx->stream);
    }
    if (hb) cudaFreeAsync(hb, ctx->stream);
    if (hc) cudaFreeAsync(hc, ctx->stream);
    return on_device ? OBB_OK : check_device_error(ctx);
}

obb_status obb_mlp_forward(obb_ctx* ctx, const obb_mlp* m, const float* feats, int64_t B, float* out,
                           int32_t half_weights, int32_t on_device)
{
    if (!ctx || !m || (B > 0 && (!feats || !out))) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (m->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "network belongs to another context");
    if (B <= 0) return OBB_OK;
    if (B > (1 << 24)) return fail(ctx, OBB_ERR_RANGE, "batch too large");
    void* hx = nullptr;
    const float* dx;
    OBB_TRY(dev_in(ctx, feats, (size_t)B * kIn, on_device, &hx, &dx));
    OBB_TRY(mlp_reserve(ctx, m->p, B));
    mlp_forward(ctx, m->p, dx, (int)B, nullptr, half_weights != 0);
    OBB_CK(ctx, cudaGetLastError());
    OBB_CK(ctx, cudaMemcpyAsync(out, m->p->y, sizeof(float) * B,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (hx) cudaFreeAsync(hx, ctx->stream);
    return on_device ? OBB_OK : check_device_error(ctx);
}

obb_status obb_mlp_gradients(obb_ctx* ctx, obb_mlp* m, const float* feats, const float* target, int64_t B,
                             float* grads, float* loss, int32_t on_device)
{
    if (!ctx || !m || !feats || !target || B <= 0) return fail(ctx, OBB_ERR_ARG, "bad argument");
    if (m->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "network belongs to another context");
    if (B > (1 << 24)) return fail(ctx, OBB_ERR_RANGE, "batch too large");
    void *hx = nullptr, *ht = nullptr;
    const float *dx, *dt;
    OBB_TRY(dev_in(ctx, feats, (size_t)B * kIn, on_device, &hx, &dx));
    OBB_TRY(dev_in(ctx, target, (size_t)B, on_device, &ht, &dt));
    OBB_TRY(mlp_reserve(ctx, m->p, B));
    OBB_TRY(mlp_backward(ctx, m->p, dx, dt, (int)B));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (grads) OBB_CK(ctx, cudaMemcpyAsync(grads, m->p->g, sizeof(float) * kParams, kind, ctx->stream));
    if (loss) OBB_CK(ctx, cudaMemcpyAsync(loss, m->p->loss, sizeof(float), kind, ctx->stream));
    if (hx) cudaFreeAsync(hx, ctx->stream);
    if (ht) cudaFreeAsync(ht, ctx->stream);
    return on_device ? OBB_OK : check_device_error(ctx);
}

obb_status obb_mlp_train_step(obb_ctx* ctx, obb_mlp* m, const float* feats, const float* target, int64_t B, float lr,
                              float* loss, int32_t on_device)
{
    if (!ctx || !m || !feats || !target || B <= 0) return fail(ctx, OBB_ERR_ARG, "bad argument");
    if (m->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "network belongs to another context");
    if (B > (1 << 24)) return fail(ctx, OBB_ERR_RANGE, "batch too large");
    void *hx = nullptr, *ht = nullptr;
    const float *dx, *dt;
    OBB_TRY(dev_in(ctx, feats, (size_t)B * kIn, on_device, &hx, &dt));
    dx = dt;
    OBB_TRY(dev_in(ctx, target, (size_t)B, on_device, &ht, &dt));
    MlpImpl* P = m->p;
    OBB_TRY(mlp_reserve(ctx, P, B));
    OBB_TRY(mlp_backward(ctx, P, dx, dt, (int)B));
    P->step += 1;
    const float b1t = std::pow(0.9f, (float)P->step), b2t = std::pow(0.999f, (float)P->step);
    k_adam<<<(unsigned)((kParams + 255) / 256), 256, 0, ctx->stream>>>(P->w, P->g, P->m, P->v, P->wh, kParams, lr,
                                                                      b1t, b2t);
    k_pack_tc<<<(unsigned)((kTcPacked + 255) / 256), 256, 0, ctx->stream>>>(P->wh, P->wtc);
    note_launch(ctx, 2);
    OBB_CK(ctx, cudaGetLastError());
    if (loss)
        OBB_CK(ctx, cudaMemcpyAsync(loss, P->loss, sizeof(float),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (hx) cudaFreeAsync(hx, ctx->stream);
    if (ht) cudaFreeAsync(ht, ctx->stream);
    return (loss && !on_device) ? check_device_error(ctx) : OBB_OK;
}

}  // extern "C"
