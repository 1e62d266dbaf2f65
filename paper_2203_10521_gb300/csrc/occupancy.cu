// Solid occupancy of the lattice by per-column crossing parity.
//
// The paper's outer volume (Eq. 4) needs the solid Omega(X) of Sec. 3; here
// it is sampled at the N^3 cell-centred lattice points, exactly:
//   1. AABB of the vertices (ordered-integer atomics, order independent);
//   2. snap every vertex to fixed point U = rint(((x - lo)/h - 1/2) 2^8);
//   3. per triangle, per covered column: Simulation-of-Simplicity containment
//      of the column point in the (y, z) projection, exact int64 crossing
//      x* = num / den, flip bit i* = ceil(x* / 256) (clamped below at 0,
//      dropped at >= N) with atomicXor: every crossing toggles one bit;
//   4. prefix XOR along each row: bit i = parity of crossings with i* <= i.
// Row layout: row (j, k) at word (k N + j) W, W = 2 ceil(N / 128), bit i of
// word i >> 6; the scan clears padding bits >= N.
#include "internal.h"

namespace obbv {
namespace {

__device__ __forceinline__ uint32_t f2key(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_init_aabb(uint32_t* keys)
{
    if (threadIdx.x < 3) keys[threadIdx.x] = 0xffffffffu;
    else if (threadIdx.x < 6) keys[threadIdx.x] = 0u;
}

__global__ void k_aabb(const float* __restrict__ V, int64_t nv, uint32_t* keys)
{
    uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x)
        for (int b = 0; b < 3; ++b) {
            uint32_t k = f2key(V[3 * v + b]);
            mn[b] = min(mn[b], k);
            mx[b] = max(mx[b], k);
        }
    for (int b = 0; b < 3; ++b)
        for (int o = 16; o > 0; o >>= 1) {
            mn[b] = min(mn[b], __shfl_xor_sync(0xffffffffu, mn[b], o));
            mx[b] = max(mx[b], __shfl_xor_sync(0xffffffffu, mx[b], o));
        }
    // warp results through shared memory, then six atomics per block (atomics
    // from every warp to the same six words serialise in L2)
    __shared__ uint32_t sh[6][32];
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int b = 0; b < 3; ++b) {
            sh[b][w] = mn[b];
            sh[3 + b][w] = mx[b];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int b = threadIdx.x;
        uint32_t v = sh[b][0];
        for (int i = 1; i < nw; ++i) v = b < 3 ? min(v, sh[b][i]) : max(v, sh[b][i]);
        if (b < 3) atomicMin(&keys[b], v);
        else atomicMax(&keys[b], v);
    }
}

__global__ void k_frame(const uint32_t* keys, int32_t N, LatticeFrame* f, int32_t* err)
{
    if (threadIdx.x != 0) return;
    double hm = 0.0;
    for (int b = 0; b < 3; ++b) {
        double lo = (double)key2f(keys[b]);
        double hi = (double)key2f(keys[3 + b]);
        double h = __ddiv_rn(__dsub_rn(hi, lo), (double)N);
        f->lo[b] = lo;
        f->h[b] = h;
        if (!(h > 0.0)) atomicOr(err, kErrDegenerate);
        hm = fmax(hm, h);
    }
    f->hmax = hm;
    for (int b = 0; b < 3; ++b) {
        f->center[b] = __dadd_rn(f->lo[b], __dmul_rn(0.5 * N, f->h[b]));
        f->s256[b] = f->h[b] > 0.0 ? __dmul_rn(__drcp_rn(f->h[b]), 256.0) : 0.0;   // 256 rn(1/h), exact scaling
    }
    f->N = N;
    f->W = 2 * ((N + 127) / 128);
}

// U = rint(((x - lo) / h - 1/2) 256), each step a correctly rounded FP64 op
// (the definition: Q = 256 rn(rn(d / h) - 1/2), d = x - lo).  With
// X = d / h <= 2^12 (|Q| < 2^20; a vertex of the lattice's own frame has
// X <= N + 1 <= 2049), Q lies within 2^-32 of 256 (X - 1/2), and so does the
// fast value q = rn(d s256 - 128), s256 = 256 rn(1/h): one fused
// multiply-add, within 2^-31 of Q.  Whenever q lies farther than 2^-29 from
// a half-integer, rint(q) = rint(Q); otherwise, or out of that range, the
// defining sequence, with the division, decides.
__global__ void k_snap(const float* __restrict__ V, int64_t nv, const LatticeFrame* __restrict__ f,
                       int32_t* __restrict__ U)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * nv) return;
    int b = (int)(i % 3);
    const double d = __dsub_rn((double)V[i], f->lo[b]);
    double q = __fma_rn(d, f->s256[b], -128.0);
    double r = rint(q);
    if (!(fabs(q - r) < 0.5 - 0x1p-29) || !(fabs(q) < 0x1p20)) {
        q = __ddiv_rn(d, f->h[b]);
        q = __dsub_rn(q, 0.5);
        q = __dmul_rn(q, 256.0);
        r = rint(q);
    }
    U[i] = (int32_t)r;
}

// orient2d in the (y, z) plane; coordinates are |U| <= 2^19, so every factor
// fits in 32 bits and each product in 64 (one wide multiply-add).
__device__ __forceinline__ int64_t orient_yz(int32_t ay, int32_t az, int32_t by, int32_t bz, int32_t py,
                                             int32_t pz)
{
    return (int64_t)(by - ay) * (pz - az) - (int64_t)(bz - az) * (py - ay);
}

// sign of orient2d((a, b), p + (eps, eps^2)) for eps -> 0+
__device__ __forceinline__ int sos_side(int32_t ay, int32_t az, int32_t by, int32_t bz, int32_t py, int32_t pz,
                                        int64_t* o)
{
    *o = orient_yz(ay, az, by, bz, py, pz);
    if (*o != 0) return *o > 0 ? 1 : -1;
    if (bz != az) return bz > az ? -1 : 1;
    if (by != ay) return by > ay ? 1 : -1;
    return 0;
}

// ceil(num / (256 den)) for den > 0, clamped to [-1, N]: a float estimate
// (through 32-bit conversions, which stay off the FP64 pipe) corrected by
// exact int64 products (the quotient is a lattice index).
__device__ __forceinline__ int32_t first_index_at_or_after(int64_t num, int64_t den, int32_t N)
{
    const int64_t D = den << kS;
    float e = i64_to_float(num) / i64_to_float(D);
    e = fminf(fmaxf(e, -2.0f), (float)N + 1.0f);
    int32_t q = (int32_t)ceilf(e);
    // smallest q with q * D >= num, searched within [-1, N]
    while (q > -1 && (int64_t)(q - 1) * D >= num) --q;
    while (q < N && (int64_t)q * D < num) ++q;
    return q;
}

// Column-crossing flips (one atomicXor per crossing), with the work balanced
// inside each warp: a warp holds 32 triangles, and their (triangle, column) checks -- 1 to 64 per triangle on
// the benchmark's mesh, 27% lane utilisation when each lane walks its own
// triangle -- are dealt out as equal contiguous runs, one per lane.  A lane
// walks its run column by column and moves to the next triangle (its data
// staged in shared memory) when one is exhausted.
constexpr int kFlipWarps = 4;

__global__ void __launch_bounds__(32 * kFlipWarps) k_flip_balanced(const int32_t* __restrict__ U,
                                                                   const int32_t* __restrict__ F, int64_t nt,
                                                                   int32_t N, int32_t W,
                                                                   unsigned long long* __restrict__ words)
{
    __shared__ int32_t s_tri[kFlipWarps][32][13];   // x, y, z of A, B, C; j0, j1, k0, k1
    __shared__ int32_t s_pre[kFlipWarps][33];       // exclusive prefix of the check counts
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * kFlipWarps + w) * 32 + lane;
    int32_t cnt = 0;
    if (t < nt) {
        const int32_t* A = U + 3 * (int64_t)F[3 * t];
        const int32_t* B = U + 3 * (int64_t)F[3 * t + 1];
        const int32_t* C = U + 3 * (int64_t)F[3 * t + 2];
        int32_t* d = s_tri[w][lane];
        for (int q = 0; q < 3; ++q) {
            d[q] = A[q];
            d[3 + q] = B[q];
            d[6 + q] = C[q];
        }
        const int32_t ymin = min(d[1], min(d[4], d[7])), ymax = max(d[1], max(d[4], d[7]));
        const int32_t zmin = min(d[2], min(d[5], d[8])), zmax = max(d[2], max(d[5], d[8]));
        d[9] = max(-((-ymin) >> kS), 0);
        d[10] = min(ymax >> kS, N - 1);
        d[11] = max(-((-zmin) >> kS), 0);
        d[12] = min(zmax >> kS, N - 1);
        cnt = max(d[10] - d[9] + 1, 0) * max(d[12] - d[11] + 1, 0);
    }
    int32_t inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    s_pre[w][lane + 1] = inc;
    if (lane == 0) s_pre[w][0] = 0;
    const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
    __syncwarp();
    const int32_t b = (int32_t)((int64_t)total * lane / 32), e = (int32_t)((int64_t)total * (lane + 1) / 32);
    if (b >= e) return;
    // the triangle holding check b: the last tt with s_pre[tt] <= b (its count is > b - s_pre[tt])
    int32_t lo = 0, hi = 31;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (s_pre[w][mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    int32_t tt = lo;
    const int32_t* d = s_tri[w][tt];
    int32_t c = b - s_pre[w][tt];
    int32_t nj = d[10] - d[9] + 1;
    int32_t k = d[11] + c / nj, j = d[9] + c % nj;
    for (int32_t i = b;; ) {
        const int32_t pz = k << kS, py = j << kS;
        int64_t wa, wb, wc;
        const int sa = sos_side(d[4], d[5], d[7], d[8], py, pz, &wa);
        const int sb = sos_side(d[7], d[8], d[1], d[2], py, pz, &wb);
        const int sc = sos_side(d[1], d[2], d[4], d[5], py, pz, &wc);
        if (sa != 0 && sa == sb && sb == sc) {
            int64_t den = wa + wb + wc;
            int64_t num = wa * (int64_t)d[0] + wb * (int64_t)d[3] + wc * (int64_t)d[6];
            if (den < 0) {
                den = -den;
                num = -num;
            }
            // first index with 256 i >= num / den; below 0 every point counts the crossing
            int32_t istar = first_index_at_or_after(num, den, N);
            if (istar < 0) istar = 0;
            if (istar < N) atomicXor(&words[((int64_t)k * N + j) * W + (istar >> 6)], 1ull << (istar & 63));
        }
        if (++i == e) break;
        if (++j > d[10]) {
            j = d[9];
            if (++k > d[12]) {
                // next triangle with checks (one exists: checks remain in this run)
                do {
                    ++tt;
                } while (s_pre[w][tt + 1] == s_pre[w][tt]);
                d = s_tri[w][tt];
                j = d[9];
                k = d[11];
            }
        }
    }
}

// 64 x 64 bit transpose across a warp: lane l holds rows l (a) and l + 32 (b);
// afterwards row c holds at bit r what row r held at bit c.  Six rounds swap
// the off-diagonal halves of 32-, 16-, ..., 1-bit blocks; below 32 the
// partner row sits in lane l ^ j.
__device__ __forceinline__ void transpose64(uint64_t& a, uint64_t& b, int lane)
{
    const uint64_t t = ((a >> 32) ^ b) & 0x00000000FFFFFFFFull;
    b ^= t;
    a ^= t << 32;
    const uint64_t masks[5] = {0x0000FFFF0000FFFFull, 0x00FF00FF00FF00FFull, 0x0F0F0F0F0F0F0F0Full,
                               0x3333333333333333ull, 0x5555555555555555ull};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int j = 16 >> q;
        const uint64_t m = masks[q];
        const uint64_t oa = __shfl_xor_sync(0xffffffffu, a, j), ob = __shfl_xor_sync(0xffffffffu, b, j);
        if (lane & j) {
            a ^= ((oa >> j) ^ a) & m;
            b ^= ((ob >> j) ^ b) & m;
        } else {
            a ^= (((a >> j) ^ oa) & m) << j;
            b ^= (((b >> j) ^ ob) & m) << j;
        }
    }
}

// The occupancy with rows along y (mode 0: slice k, row (k, i), bit j) or
// along z (mode 1: slice j, row (j, i), bit k), from the rows along x (row
// (k, j), bit i): one warp per (slice, 64 x 64 block).  The copies are for
// counting and interleave a slice's rows by column: word w of row (slice s,
// column c) at (s W + w) N + c.  Bits of rows past N read as 0; words past
// ceil(N / 64) are never read by the counting kernel.
__global__ void k_transpose_rows(const uint64_t* __restrict__ xw, uint64_t* __restrict__ dst, int32_t N, int32_t W,
                                 int mode)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int32_t nb = (N + 63) >> 6;
    if (warp >= (int64_t)N * nb * nb) return;
    const int32_t sl = (int32_t)(warp / ((int64_t)nb * nb));
    const int32_t rem = (int32_t)(warp % ((int64_t)nb * nb));
    const int32_t R = rem / nb, C = rem % nb;   // source rows 64 R.., source word C
    const int32_t r0 = 64 * R + lane, r1 = r0 + 32;
    auto src_row = [&](int32_t r) -> int64_t {
        return mode == 0 ? ((int64_t)sl * N + r) * W : ((int64_t)r * N + sl) * W;
    };
    uint64_t a = r0 < N ? __ldg(xw + src_row(r0) + C) : 0ull;
    uint64_t b = r1 < N ? __ldg(xw + src_row(r1) + C) : 0ull;
    transpose64(a, b, lane);
    const int32_t c0 = 64 * C + lane, c1 = c0 + 32;
    if (c0 < N) dst[((int64_t)sl * W + R) * N + c0] = a;
    if (c1 < N) dst[((int64_t)sl * W + R) * N + c1] = b;
}

__device__ __forceinline__ uint64_t prefix_xor(uint64_t x)
{
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    x ^= x << 16;
    x ^= x << 32;
    return x;
}

// Exclusive prefix of v over the G lanes of a row (lanes lr G .. lr G + G - 1;
// c = the lane's place in the row); every lane of the warp takes part.
__device__ __forceinline__ uint32_t row_exclusive_sum(uint32_t v, int c, int G)
{
    uint32_t x = v;
    for (int off = 1; off < G; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (c >= off) x += y;
    }
    return x - v;
}

// One lane per 128-bit chunk; a row's G = W / 2 chunks sit on consecutive
// lanes.  The prefix XOR along the row turns the crossing flips into
// occupancy; the same pass writes the counting copy of the words and the
// rank table (occupied bits before each 64-bit word), both interleaved by
// column: word w of row (k, j) at (k W + w) N + j.
__global__ void k_row_scan(uint64_t* __restrict__ words, uint64_t* __restrict__ cwords,
                           uint16_t* __restrict__ rank, int32_t N, int32_t W)
{
    const int G = W >> 1;
    const int rpw = 32 / G;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lr = lane / G, c = lane - lr * G;
    const int64_t row = warp * rpw + lr;
    const bool active = lr < rpw && row < (int64_t)N * N;
    uint64_t w0 = 0, w1 = 0;
    uint4* p = reinterpret_cast<uint4*>(words + row * W + 2 * c);
    if (active) {
        uint4 v = *p;
        w0 = ((uint64_t)v.y << 32) | v.x;
        w1 = ((uint64_t)v.w << 32) | v.z;
    }
    int par0 = __popcll(w0) & 1;
    uint64_t p0 = prefix_xor(w0);
    uint64_t p1 = prefix_xor(w1) ^ (par0 ? ~0ull : 0ull);
    int x = (__popcll(w0) + __popcll(w1)) & 1;
    const int mine = x;
    for (int off = 1; off < G; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, off);
        if (c >= off) x ^= y;
    }
    if (x ^ mine) {
        p0 = ~p0;
        p1 = ~p1;
    }
    const int base = 128 * c;
    uint64_t m0 = (base + 64 <= N) ? ~0ull : (base >= N ? 0ull : ((1ull << (N - base)) - 1));
    uint64_t m1 = (base + 128 <= N) ? ~0ull : (base + 64 >= N ? 0ull : ((1ull << (N - base - 64)) - 1));
    p0 &= m0;
    p1 &= m1;
    const uint32_t n0 = (uint32_t)__popcll(p0);
    const uint32_t before = row_exclusive_sum(n0 + (uint32_t)__popcll(p1), c, G);
    if (active) {
        *p = make_uint4((uint32_t)p0, (uint32_t)(p0 >> 32), (uint32_t)p1, (uint32_t)(p1 >> 32));
        const int64_t k = row / N, j = row - k * N;
        const int64_t i0 = (k * W + 2 * c) * N + j;
        cwords[i0] = p0;
        cwords[i0 + N] = p1;
        rank[i0] = (uint16_t)before;
        rank[i0 + N] = (uint16_t)(before + n0);
    }
}

// The rank table of finished interleaved rows (the y- and z-row copies): one
// thread per row (slice s, column c), columns on consecutive threads.
__global__ void k_row_rank(const uint64_t* __restrict__ words, uint16_t* __restrict__ rank, int32_t N, int32_t W)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * N) return;
    const int64_t sl = t / N, c = t - sl * N;
    const int64_t base = sl * W * N + c;
    uint32_t run = 0;
    for (int32_t w = 0; w < W; ++w) {
        rank[base + (int64_t)w * N] = (uint16_t)run;
        run += (uint32_t)__popcll(__ldg(words + base + (int64_t)w * N));
    }
}

}  // namespace

obb_status rebuild_occupancy(obb_ctx* ctx, obb_lattice* lat)
{
    cudaStream_t s = ctx->stream;
    const obb_mesh* mesh = lat->mesh;
    const int32_t N = lat->frame.N;
    const int32_t W = 2 * ((N + 127) / 128);
    OBB_CK(ctx, ctx->tmp_d.reserve(64, s));
    uint32_t* keys = ctx->tmp_d.as<uint32_t>();
    k_init_aabb<<<1, 32, 0, s>>>(keys);
    note_launch(ctx);
    int64_t nb64 = (mesh->nv + 255) / 256;
    int nb = (int)(nb64 < 4 * ctx->num_sms ? nb64 : 4 * ctx->num_sms);
    k_aabb<<<max(nb, 1), 256, 0, s>>>(mesh->d_verts, mesh->nv, keys);
    note_launch(ctx);
    k_frame<<<1, 32, 0, s>>>(keys, N, lat->d_frame, ctx->d_err);
    note_launch(ctx);
    k_snap<<<(unsigned)((3 * mesh->nv + 255) / 256), 256, 0, s>>>(mesh->d_verts, mesh->nv, lat->d_frame,
                                                                 lat->d_fixed);
    note_launch(ctx);
    OBB_CK(ctx, cudaMemsetAsync(lat->d_words, 0, sizeof(uint64_t) * lat->n_words, s));
    k_flip_balanced<<<(unsigned)((mesh->nt + 32 * kFlipWarps - 1) / (32 * kFlipWarps)), 32 * kFlipWarps, 0, s>>>(
        lat->d_fixed, mesh->d_tris, mesh->nt, N, W, reinterpret_cast<unsigned long long*>(lat->d_words));
    note_launch(ctx);
    const int G = W / 2, rpw = 32 / G;
    int64_t warps = ((int64_t)N * N + rpw - 1) / rpw;
    k_row_scan<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(lat->d_words, lat->d_cwords, lat->d_rank, N, W);
    note_launch(ctx);
    // rows along y and z: kept once a context counts along them, then refreshed
    // by every rebuild
    if (ctx->count_axis != 0 && !lat->d_words_y) {
        OBB_CK(ctx, pool_alloc((void**)&lat->d_words_y, sizeof(uint64_t) * lat->n_words, s));
        OBB_CK(ctx, pool_alloc((void**)&lat->d_words_z, sizeof(uint64_t) * lat->n_words, s));
        OBB_CK(ctx, pool_alloc((void**)&lat->d_rank_y, sizeof(uint16_t) * lat->n_words, s));
        OBB_CK(ctx, pool_alloc((void**)&lat->d_rank_z, sizeof(uint16_t) * lat->n_words, s));
        // the transposes never write the padding words past ceil(N / 64): zero them once
        OBB_CK(ctx, cudaMemsetAsync(lat->d_words_y, 0, sizeof(uint64_t) * lat->n_words, s));
        OBB_CK(ctx, cudaMemsetAsync(lat->d_words_z, 0, sizeof(uint64_t) * lat->n_words, s));
        lat->ref.words_y = lat->d_words_y;
        lat->ref.words_z = lat->d_words_z;
        lat->ref.rank_y = lat->d_rank_y;
        lat->ref.rank_z = lat->d_rank_z;
        OBB_CK(ctx, cudaMemcpyAsync(lat->d_ref, &lat->ref, sizeof(LatRef), cudaMemcpyHostToDevice, s));
    }
    if (lat->d_words_y) {
        const int64_t tb = (N + 63) / 64, tw = (int64_t)N * tb * tb;
        k_transpose_rows<<<(unsigned)((tw + 7) / 8), 256, 0, s>>>(lat->d_words, lat->d_words_y, N, W, 0);
        k_transpose_rows<<<(unsigned)((tw + 7) / 8), 256, 0, s>>>(lat->d_words, lat->d_words_z, N, W, 1);
        const unsigned rb = (unsigned)(((int64_t)N * N + 255) / 256);
        k_row_rank<<<rb, 256, 0, s>>>(lat->d_words_y, lat->d_rank_y, N, W);
        k_row_rank<<<rb, 256, 0, s>>>(lat->d_words_z, lat->d_rank_z, N, W);
        note_launch(ctx, 4);
    }
    OBB_CK(ctx, cudaGetLastError());
    lat->frame_stale = true;   // the host copy is refreshed when a host reader needs it
    return OBB_OK;
}

obb_status build_occupancy(obb_ctx* ctx, const obb_mesh* mesh, int32_t N, obb_lattice* lat)
{
    cudaStream_t s = ctx->stream;
    if (N < 1 || N > kMaxN) return fail(ctx, OBB_ERR_RANGE, "lattice size N must be in [1, 2048]");
    const int32_t W = 2 * ((N + 127) / 128);
    lat->ctx = ctx;
    lat->mesh = mesh;
    lat->n_words = (size_t)N * N * W;
    lat->frame.N = N;
    lat->frame.W = W;
    OBB_CK(ctx, pool_alloc((void**)&lat->d_frame, sizeof(LatticeFrame), s));
    OBB_CK(ctx, pool_alloc((void**)&lat->d_fixed, sizeof(int32_t) * 3 * mesh->nv, s));
    OBB_CK(ctx, pool_alloc((void**)&lat->d_words, sizeof(uint64_t) * lat->n_words, s));
    OBB_CK(ctx, pool_alloc((void**)&lat->d_cwords, sizeof(uint64_t) * lat->n_words, s));
    OBB_CK(ctx, pool_alloc((void**)&lat->d_rank, sizeof(uint16_t) * lat->n_words, s));
    OBB_CK(ctx, pool_alloc((void**)&lat->d_ref, sizeof(LatRef), s));
    lat->ref = LatRef{lat->d_cwords, nullptr, nullptr, lat->d_rank, nullptr, nullptr, N, W};
    OBB_CK(ctx, cudaMemcpyAsync(lat->d_ref, &lat->ref, sizeof(LatRef), cudaMemcpyHostToDevice, s));
    OBB_TRY(rebuild_occupancy(ctx, lat));
    OBB_TRY(lattice_frame_host(lat));
    return check_device_error(ctx);
}

}  // namespace obbv
