// Lloyd iteration on one layer of boxes (Sec. 4.2.1, Eq. 11-13), data parallel.
//
// Layer state lives on the device: triangle -> cluster map, per-cluster
// frame (FP64), quantised box, exact outer volume, and the member list of
// every cluster (triangles sorted by cluster, stable).
//
// Partition round (all exact integers):
//   extents     block per cluster: for each of the six slab sides the extreme
//               projection of the members, the smallest triangle attaining
//               it, and the extreme over the other members;
//   candidates  thread per triangle: a triangle that alone attains a side of
//               its cluster s (size >= 2) shrinks s's box when it leaves; for
//               each sibling cluster k of its edge neighbours the grown box of
//               k is formed; every box that differs from the current one is
//               appended to an evaluation list;
//   count       the outer-volume kernel on the evaluation list;
//   gains       gain = [OBV(s) - OBV(s - t)] - [OBV(k + t) - OBV(k)]; best k per
//               triangle (ties -> smaller k); a positive proposal posts its key
//               (gain << 24 | (2^24 - 1 - t)) with atomicMax at both clusters;
//   accept      a proposal holding the maximum key at both of its clusters is
//               applied; accepted moves touch disjoint clusters.
// Refit: area-weighted covariance with compensated FP32 sums (TwoProduct +
// TwoSum), cyclic Jacobi in FP64, quantised normals, tight bounds, exact count;
// the new box is kept iff its outer volume is strictly smaller.
// Member lists: a stable least-significant-digit radix sort of the triangles
// by cluster (per-tile digit counts, their exclusive scan, a stable scatter
// that ranks equal digits with warp matches in triangle order).
#include <algorithm>

#include "internal.h"

namespace obbv {
namespace {

constexpr int kNT = 128;   // threads of the block-per-cluster kernels

enum { kCtrCand = 0, kCtrEval, kCtrCount };

constexpr int kMaxTopk = 16;   // candidates a surrogate may keep per source cluster

struct Cand {
    int32_t t, s;
    int32_t k[3];
    int32_t nk;
    int32_t e_shr;
    int32_t e_gro[3];
    int32_t best;
    int32_t pad;
    int64_t gain;
    unsigned long long key;
};

__device__ __forceinline__ void proj3(const int32_t* __restrict__ U, const int32_t* __restrict__ F, int32_t t,
                                      const int32_t* n, int64_t* dmin, int64_t* dmax)
{
    int32_t v[3] = {F[3 * t], F[3 * t + 1], F[3 * t + 2]};
    for (int a = 0; a < 3; ++a) {
        dmin[a] = INT64_MAX;
        dmax[a] = INT64_MIN;
    }
    for (int q = 0; q < 3; ++q) {
        const int32_t* P = U + 3 * (int64_t)v[q];
        int64_t x = P[0], y = P[1], z = P[2];
        for (int a = 0; a < 3; ++a) {
            int64_t d = (int64_t)n[3 * a] * x + (int64_t)n[3 * a + 1] * y + (int64_t)n[3 * a + 2] * z;
            dmin[a] = min(dmin[a], d);
            dmax[a] = max(dmax[a], d);
        }
    }
}

// ------------------------------------------------------- membership

__global__ void k_check_nonempty(const int32_t* __restrict__ size, int32_t K, int32_t* err)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K && size[k] == 0) atomicOr(err, kErrEmpty);
}

// Member lists: triangles sorted by cluster, ascending triangle index within
// a cluster.  Each pass of the radix sort orders the (cluster, triangle) pairs
// stably by one digit of the cluster (at most 10 bits, lowest digit first),
// over tiles of kSortTile consecutive positions:
//   k_sort_count    digit counts of every tile, cnt[digit * ntiles + tile];
//                   for a small table its last block (an atomic ticket,
//                   nothing waits) also scans them;
//   k_sort_sums /   otherwise the exclusive scan of cnt in that order, in two
//   k_sort_offsets  passes: where each tile's items of each digit start;
//   k_sort_scatter  the tile's items in order, rounds of 256: equal digits of
//                   a warp ranked by __match_any_sync, warps after one another
//                   per digit, rounds after one another.
// The first pass takes the triangle index as its value; the last writes only
// the values (the member list).  With one pass the digit is the cluster, so
// the offsets of the first tile are the cluster starts.
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kSortMaxBits = 10;
constexpr int kSortScanPer = 8;
constexpr int kSortScanBlock = kSortThreads * kSortScanPer;
constexpr int64_t kSortFusedScanMax = 8192;   // largest table the count kernel's last block scans

__device__ __forceinline__ int sort_digit(int32_t key, int shift, int bins)
{
    return (int)(((uint32_t)key >> shift) & (uint32_t)(bins - 1));
}

// exclusive scan of in[0..n) into out by one block, chunks of kSortScanBlock
// (a thread's eight consecutive values in registers), with a running carry
__device__ void block_scan_i32(const int32_t* in, int64_t n, int32_t* out, int32_t* ws)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t carry = 0;
    for (int64_t c = 0; c < n; c += kSortScanBlock) {
        const int64_t base = c + threadIdx.x * kSortScanPer;
        int32_t v[kSortScanPer];
        int32_t sum = 0;
#pragma unroll
        for (int q = 0; q < kSortScanPer; ++q) {
            v[q] = base + q < n ? __ldcg(in + base + q) : 0;
            sum += v[q];
        }
        int32_t x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        int32_t run = carry + x - sum, tot = 0;
        for (int i = 0; i < kSortThreads / 32; ++i) {
            if (i < w) run += ws[i];
            tot += ws[i];
        }
#pragma unroll
        for (int q = 0; q < kSortScanPer; ++q) {
            if (base + q < n) out[base + q] = run;
            run += v[q];
        }
        carry += tot;
        __syncthreads();   // ws is reused
    }
}

// K > 0: keys outside [0, K) raise kErrArg.  size != nullptr: the cluster
// sizes are added up as well (keys = clusters; size zeroed beforehand).
// scan_out != nullptr: the last block to finish scans the counts into
// scan_out.
__global__ void __launch_bounds__(kSortThreads) k_sort_count(const int32_t* __restrict__ keys, int64_t n, int shift,
                                                             int bins, int32_t ntiles, int32_t K,
                                                             int32_t* __restrict__ size,
                                                             int32_t* __restrict__ cnt, int32_t* __restrict__ scan_out,
                                                             unsigned int* __restrict__ ticket, int32_t* err)
{
    extern __shared__ int32_t h[];   // [bins]
    __shared__ int32_t ws[kSortThreads / 32];
    __shared__ bool last;
    for (int i = threadIdx.x; i < bins; i += kSortThreads) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int lane = threadIdx.x & 31;
    int32_t kr[kSortRounds];   // every load issued before the first is used
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        kr[r] = i < n ? keys[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        // the digit of every key, valid or not, as k_sort_scatter takes it;
        // a key outside [0, K) is reported and left out of the sizes
        int d = -1;
        int32_t cl = -1;
        if (i < n) {
            const int32_t key = kr[r];
            if (K > 0 && (key < 0 || key >= K)) atomicOr(err, kErrArg);
            else cl = key;
            d = sort_digit(key, shift, bins);
        }
        if (size) {
            const unsigned same = __match_any_sync(0xffffffffu, cl);
            if (cl >= 0 && lane == __ffs(same) - 1) atomicAdd(&size[cl], __popc(same));
        }
        // equal digits of a warp (neighbouring triangles mostly share a
        // cluster) add once
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < bins; i += kSortThreads) cnt[(int64_t)i * ntiles + blockIdx.x] = h[i];
    if (!scan_out) return;
    // the block's writes, then one gpu-scope fence before its ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    if (!last) return;
    block_scan_i32(cnt, (int64_t)bins * ntiles, scan_out, ws);
    if (threadIdx.x == 0) *ticket = 0;   // ready for the next launch
}

// bsum[b] = sum of in[b * kSortScanBlock .. (b + 1) * kSortScanBlock)
__global__ void __launch_bounds__(kSortThreads) k_sort_sums(const int32_t* __restrict__ in, int64_t n,
                                                            int32_t* __restrict__ bsum)
{
    __shared__ int32_t ws[kSortThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kSortScanBlock + threadIdx.x * kSortScanPer;
    int32_t v = 0;
#pragma unroll
    for (int q = 0; q < kSortScanPer; ++q) v += base + q < n ? in[base + q] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) t += ws[w];
        bsum[blockIdx.x] = t;
    }
}

// out = exclusive scan of in (the block totals before this block, then the
// block's own positions)
__global__ void __launch_bounds__(kSortThreads) k_sort_offsets(const int32_t* __restrict__ in, int64_t n,
                                                               const int32_t* __restrict__ bsum,
                                                               int32_t* __restrict__ out)
{
    __shared__ int32_t ws[kSortThreads / 32];
    __shared__ int32_t before;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t p = 0;
    for (int32_t b = threadIdx.x; b < (int32_t)blockIdx.x; b += kSortThreads) p += bsum[b];
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0) ws[w] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int i = 0; i < kSortThreads / 32; ++i) t += ws[i];
        before = t;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortScanBlock + threadIdx.x * kSortScanPer;
    int32_t v[kSortScanPer];
    int32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kSortScanPer; ++q) {
        v[q] = base + q < n ? in[base + q] : 0;
        sum += v[q];
    }
    int32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();   // ws is reused
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int32_t run = before + x - sum;
    for (int i = 0; i < w; ++i) run += ws[i];
#pragma unroll
    for (int q = 0; q < kSortScanPer; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
}

// dynamic shared memory of k_sort_scatter for 2^bits digits
static size_t sort_scatter_smem(int bins)
{
    return sizeof(int32_t) * (size_t)(kSortThreads / 32) * bins;
}

// One pass's stable scatter of a tile.  Each warp owns kSortTile / 8
// consecutive positions of the tile: it counts their digits into its own
// row of shared memory, the rows become per-digit starts (the tile's offset
// plus the items of the warps before), and the warp places its items in
// order, ranking equal digits within a round by __match_any_sync.
// vals == nullptr: the value is the position (the triangle index);
// keys_out == nullptr: keys are not written.  start != nullptr (one pass,
// digit = cluster): block 0 also writes the cluster starts start[0..K] and
// sizes size[0..K).
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_scatter(const int32_t* __restrict__ keys,
                                                               const int32_t* __restrict__ vals, int64_t n,
                                                               int shift, int bins, int32_t ntiles,
                                                               const int32_t* __restrict__ off,
                                                               int32_t* __restrict__ keys_out,
                                                               int32_t* __restrict__ vals_out, int32_t K,
                                                               int32_t* __restrict__ start,
                                                               int32_t* __restrict__ size)
{
    constexpr int kW = kSortThreads / 32;
    constexpr int kSub = kSortTile / kW;
    extern __shared__ int32_t wb[];   // [kW][bins]: a warp's count of each digit, then where the next one goes
    for (int i = threadIdx.x; i < kW * bins; i += kSortThreads) wb[i] = 0;
    if (start && blockIdx.x == 0)
        for (int k = threadIdx.x; k <= K; k += kSortThreads) {
            const int32_t a = k < bins ? off[(int64_t)k * ntiles] : (int32_t)n;
            start[k] = a;
            if (k < K) size[k] = (k + 1 < bins ? off[(int64_t)(k + 1) * ntiles] : (int32_t)n) - a;
        }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + w * kSub;
    int32_t* mine = wb + w * bins;
    // the warp's items in registers, every load issued before the first is used
    constexpr int kR = kSub / 32;
    int32_t kr[kR], vr[kR];
    const int32_t left = (int32_t)min((int64_t)kSub, max(n - base, (int64_t)0));   // the warp's items
    const int32_t* kp = keys + base;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int32_t o = r * 32 + lane;
        kr[r] = o < left ? kp[o] : 0;
        vr[r] = o < left ? (vals ? vals[base + o] : (int32_t)(base + o)) : 0;
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int d = r * 32 + lane < left ? sort_digit(kr[r], shift, bins) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d >= 0 && lane == __ffs(peers) - 1) mine[d] += __popc(peers);   // distinct digits: distinct words
        __syncwarp();
    }
    __syncthreads();
    for (int q = threadIdx.x; q < bins; q += kSortThreads) {
        int32_t x = off[(int64_t)q * ntiles + blockIdx.x];
        for (int v = 0; v < kW; ++v) {
            const int32_t c = wb[v * bins + q];
            wb[v * bins + q] = x;
            x += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const bool ok = r * 32 + lane < left;
        const int32_t key = kr[r], val = vr[r];
        const int d = ok ? sort_digit(key, shift, bins) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int32_t pos = ok ? mine[d] + rank : 0;
        __syncwarp();
        if (ok && rank == 0) mine[d] += __popc(peers);
        __syncwarp();
        if (ok) {
            if (keys_out) keys_out[pos] = key;
            vals_out[pos] = val;
        }
    }
}

// Member lists after one round's accepted moves (each cluster lost at most
// one triangle, mv[c], or gained at most one, mv[K + c]; -1 = none): a warp
// per cluster copies its old segment to its new start, dropping the leaver
// and opening the place of the joiner, which keeps every segment ascending
// -- the stable sort of the new assignment.  Consumes the records (-1).
__global__ void k_members_update(const int32_t* __restrict__ old_members, const int32_t* __restrict__ old_start,
                                 const int32_t* __restrict__ new_start, int32_t* __restrict__ mv, int32_t K,
                                 int32_t* __restrict__ out)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t c = (int32_t)(g >> 5);
    const int lane = (int)(g & 31);
    if (c >= K) return;   // warp-uniform
    const int32_t so = old_start[c], n = old_start[c + 1] - so, sn = new_start[c];
    const int32_t t_out = mv[c], t_in = mv[K + c];
    int32_t below = 0;   // old members below the joiner, the leaver excepted
    for (int32_t b = 0; b < n; b += 32) {
        const int32_t i = b + lane;
        if (i >= n) break;
        const int32_t x = old_members[so + i];
        if (x == t_out) continue;
        const int32_t dst = i - (t_out >= 0 && x > t_out ? 1 : 0) + (t_in >= 0 && x > t_in ? 1 : 0);
        out[sn + dst] = x;
        below += t_in >= 0 && x < t_in ? 1 : 0;
    }
    if (t_in >= 0) {
        for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
        if (lane == 0) out[sn + below] = t_in;
    }
    if (lane == 0) {
        mv[c] = -1;
        mv[K + c] = -1;
    }
}

// ------------------------------------------------------- extents (a6)

// Per slab side of a cluster, in one pass over its members: the extreme
// projection v1 with the smallest triangle t1 attaining it, and v2, the
// extreme over every member but t1.  A member (v, t) that beats (v1, t1)
// demotes v1 into v2; any other only updates v2.  Two partial states merge
// the same way: the better best wins, and v2 is the extreme of both v2 and
// the loser's v1.  Low sides minimise, high sides maximise.
struct Top2 {
    int64_t v1, v2;
    int32_t t1;
};

__device__ __forceinline__ bool beats(int64_t v, int32_t t, const Top2& b, bool lowside)
{
    if (v != b.v1) return lowside ? (v < b.v1) : (v > b.v1);
    return t < b.t1;
}

__device__ __forceinline__ int64_t extreme(int64_t a, int64_t b, bool lowside) { return lowside ? min(a, b) : max(a, b); }

__device__ __forceinline__ void top2_add(Top2& b, int64_t v, int32_t t, bool lowside)
{
    if (beats(v, t, b, lowside)) {
        b.v2 = extreme(b.v2, b.v1, lowside);
        b.v1 = v;
        b.t1 = t;
    } else {
        b.v2 = extreme(b.v2, v, lowside);
    }
}

__device__ __forceinline__ void top2_merge(Top2& a, const Top2& b, bool lowside)
{
    if (beats(b.v1, b.t1, a, lowside)) {
        a.v2 = extreme(extreme(a.v2, b.v2, lowside), a.v1, lowside);
        a.v1 = b.v1;
        a.t1 = b.t1;
    } else {
        a.v2 = extreme(extreme(a.v2, b.v2, lowside), b.v1, lowside);
    }
}

__device__ __forceinline__ Top2 top2_shfl(const Top2& x, int o)
{
    Top2 y;
    y.v1 = (int64_t)__shfl_xor_sync(0xffffffffu, (long long)x.v1, o);
    y.v2 = (int64_t)__shfl_xor_sync(0xffffffffu, (long long)x.v2, o);
    y.t1 = __shfl_xor_sync(0xffffffffu, x.t1, o);
    return y;
}

__device__ __forceinline__ void top2_init(Top2 (&b)[6])
{
    for (int s = 0; s < 6; ++s) {
        const int64_t e = (s & 1) ? INT64_MIN : INT64_MAX;
        b[s] = Top2{e, e, INT32_MAX};
    }
}

// one thread's members [i0, b1) with stride st into its six states
__device__ __forceinline__ void top2_members(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                                             const int32_t* __restrict__ members, const int32_t (&n)[9], int32_t i0,
                                             int32_t b1, int32_t st, Top2 (&b)[6])
{
    for (int32_t i = i0; i < b1; i += st) {
        const int32_t t = members[i];
        int64_t dmin[3], dmax[3];
        proj3(U, F, t, n, dmin, dmax);
        for (int a = 0; a < 3; ++a) {
            top2_add(b[2 * a], dmin[a], t, true);
            top2_add(b[2 * a + 1], dmax[a], t, false);
        }
    }
}

// Large clusters: a block of NT threads per cluster.
template <int NT>
__global__ void __launch_bounds__(NT) k_extents(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                                                const int32_t* __restrict__ members,
                                                const int32_t* __restrict__ start,
                                                const obb_qbox* __restrict__ q, ClusterExt* __restrict__ ext)
{
    const int32_t k = blockIdx.x;
    int32_t n[9];
    for (int i = 0; i < 9; ++i) n[i] = q[k].n[i];
    Top2 b[6];
    top2_init(b);
    top2_members(U, F, members, n, start[k] + threadIdx.x, start[k + 1], NT, b);
    __shared__ Top2 sh[6][NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int s = 0; s < 6; ++s) {
        for (int o = 16; o > 0; o >>= 1) top2_merge(b[s], top2_shfl(b[s], o), (s & 1) == 0);
        if (lane == 0) sh[s][w] = b[s];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int s = threadIdx.x;
        Top2 x = sh[s][0];
        for (int i = 1; i < NT / 32; ++i) top2_merge(x, sh[s][i], (s & 1) == 0);
        ext[k].v1[s] = x.v1;
        ext[k].arg[s] = x.t1;
        ext[k].v2[s] = x.v2;
    }
}

// the three vertices of triangle t projected on the box's axes: per axis the
// smallest and the largest of the three (the coordinates already loaded)
__device__ __forceinline__ void proj_loaded(const int32_t (&P)[9], const int32_t (&n)[9], int64_t (&dmin)[3],
                                            int64_t (&dmax)[3])
{
    for (int a = 0; a < 3; ++a) {
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        for (int q = 0; q < 3; ++q) {
            const int64_t d = (int64_t)n[3 * a] * P[3 * q] + (int64_t)n[3 * a + 1] * P[3 * q + 1] +
                              (int64_t)n[3 * a + 2] * P[3 * q + 2];
            lo = min(lo, d);
            hi = max(hi, d);
        }
        dmin[a] = lo;
        dmax[a] = hi;
    }
}

__device__ __forceinline__ void load_tri(const int32_t* __restrict__ U, const int32_t* __restrict__ F, int32_t t,
                                         int32_t (&P)[9])
{
    const int32_t v0 = __ldg(F + 3 * (int64_t)t), v1 = __ldg(F + 3 * (int64_t)t + 1),
                  v2 = __ldg(F + 3 * (int64_t)t + 2);
    const int32_t v[3] = {v0, v1, v2};
    for (int q = 0; q < 3; ++q)
        for (int c = 0; c < 3; ++c) P[3 * q + c] = __ldg(U + 3 * (int64_t)v[q] + c);
}

__device__ __forceinline__ void top2_add6(Top2 (&b)[8], const int64_t (&dmin)[3], const int64_t (&dmax)[3], int32_t t)
{
    for (int a = 0; a < 3; ++a) {
        top2_add(b[2 * a], dmin[a], t, true);
        top2_add(b[2 * a + 1], dmax[a], t, false);
    }
}

// Small clusters: a warp per cluster, no block barrier.  Each lane takes
// every 32nd member, two at a time with both triangles' loads issued before
// either is projected.  The six states (padded to eight) are then reduced
// and scattered over the warp: at lane offsets 16, 8 and 4 a lane keeps half
// of its states, hands the other half to its partner and merges what it
// receives (4 + 2 + 1 merges instead of 6 a level), so lane l ends with
// state (l >> 2) & 7 over eight lanes; offsets 2 and 1 finish it.  Every
// order of merges gives the same state (the extreme, its smallest triangle,
// the extreme of the rest), so the result is that of a sequential pass.
__global__ void __launch_bounds__(128) k_extents_small(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                                                       const int32_t* __restrict__ members,
                                                       const int32_t* __restrict__ start, int32_t K,
                                                       const obb_qbox* __restrict__ q, ClusterExt* __restrict__ ext)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t k = (int32_t)(g >> 5);
    const int l = (int)(g & 31);
    const bool live = k < K;   // every lane of the warp takes part in the shuffles
    Top2 b[8];
    for (int s = 0; s < 8; ++s) {
        const int64_t e = (s & 1) ? INT64_MIN : INT64_MAX;
        b[s] = Top2{e, e, INT32_MAX};
    }
    if (live) {
        int32_t n[9];
        for (int i = 0; i < 9; ++i) n[i] = q[k].n[i];
        const int32_t b1 = start[k + 1];
        int32_t i = start[k] + l;
        for (; i + 32 < b1; i += 64) {
            const int32_t ta = __ldg(members + i), tb = __ldg(members + i + 32);
            int32_t Pa[9], Pb[9];
            load_tri(U, F, ta, Pa);
            load_tri(U, F, tb, Pb);
            int64_t dmin[3], dmax[3];
            proj_loaded(Pa, n, dmin, dmax);
            top2_add6(b, dmin, dmax, ta);
            proj_loaded(Pb, n, dmin, dmax);
            top2_add6(b, dmin, dmax, tb);
        }
        if (i < b1) {
            const int32_t ta = __ldg(members + i);
            int32_t Pa[9];
            load_tri(U, F, ta, Pa);
            int64_t dmin[3], dmax[3];
            proj_loaded(Pa, n, dmin, dmax);
            top2_add6(b, dmin, dmax, ta);
        }
    }
    // offset 16: keep states 0-3 (lanes 0-15) or 4-7; state parity (low or
    // high side) is that of j
    const bool u16 = (l >> 4) & 1, u8 = (l >> 3) & 1, u4 = (l >> 2) & 1;
    Top2 t4[4];
    for (int j = 0; j < 4; ++j) {
        Top2 keep = u16 ? b[4 + j] : b[j];
        top2_merge(keep, top2_shfl(u16 ? b[j] : b[4 + j], 16), (j & 1) == 0);
        t4[j] = keep;
    }
    Top2 t2[2];
    for (int j = 0; j < 2; ++j) {
        Top2 keep = u8 ? t4[2 + j] : t4[j];
        top2_merge(keep, top2_shfl(u8 ? t4[j] : t4[2 + j], 8), (j & 1) == 0);
        t2[j] = keep;
    }
    Top2 w = u4 ? t2[1] : t2[0];
    const bool low = !u4;
    top2_merge(w, top2_shfl(u4 ? t2[0] : t2[1], 4), low);
    top2_merge(w, top2_shfl(w, 2), low);
    top2_merge(w, top2_shfl(w, 1), low);
    const int s = (l >> 2) & 7;
    if (live && (l & 3) == 0 && s < 6) {
        ext[k].v1[s] = w.v1;
        ext[k].arg[s] = w.t1;
        ext[k].v2[s] = w.v2;
    }
}

// the extents of a layer's clusters, by their average size: a warp a
// cluster up to 1,024 triangles, else a block
void launch_extents(obb_ctx* ctx, const obb_layer* L, cudaStream_t s)
{
    const obb_lattice* lat = L->lat;
    const int32_t K = L->K;
    if (L->T <= (int64_t)1024 * K) {
        const int64_t th = (int64_t)K * 32;
        k_extents_small<<<(unsigned)((th + 127) / 128), 128, 0, s>>>(lat->d_fixed, lat->mesh->d_tris, L->d_members,
                                                                      L->d_start, K, L->d_q, L->d_ext);
    } else {
        k_extents<kNT><<<K, kNT, 0, s>>>(lat->d_fixed, lat->mesh->d_tris, L->d_members, L->d_start, L->d_q,
                                         L->d_ext);
    }
    note_launch(ctx);
}

// ------------------------------------------------------- candidates (a7)

// One thread per (cluster s, slab side): only a triangle that alone attains
// a side of its cluster's box shrinks the box when it leaves, so the
// candidates are the clusters' side extremes.  A triangle extreme on several
// sides is taken by the thread of the first of them, and its shrunk box moves
// all those sides.
__global__ void k_candidates(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                             const int32_t* __restrict__ adj, int32_t K, const int32_t* __restrict__ assign,
                             const int32_t* __restrict__ parent, const int32_t* __restrict__ size,
                             const ClusterExt* __restrict__ ext, const obb_qbox* __restrict__ q,
                             Cand* __restrict__ cand, obb_qbox* __restrict__ evals, int32_t* __restrict__ ctr,
                             int32_t cand_cap, int32_t eval_cap, int32_t* err)
{
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= 6 * (int64_t)K) return;
    const int32_t s = (int32_t)(id / 6);
    const int my_side = (int)(id - 6 * (int64_t)s);
    if (size[s] < 2) return;
    const ClusterExt& e = ext[s];
    const int32_t t = e.arg[my_side];
    if (e.v2[my_side] == e.v1[my_side]) return;
    obb_qbox shr = q[s];
    for (int side = 0; side < 6; ++side)
        if (e.arg[side] == t && e.v2[side] != e.v1[side]) {
            if (side < my_side) return;   // the first such side's thread takes t
            shr.b[side] = e.v2[side];
        }
    int32_t ks[3];
    int nk = 0;
    const int32_t ps = parent[s];
    for (int i = 0; i < 3; ++i) {
        int32_t k = assign[adj[3 * t + i]];
        if (k == s || parent[k] != ps) continue;
        bool dup = false;
        for (int j = 0; j < nk; ++j) dup |= ks[j] == k;
        if (!dup) ks[nk++] = k;
    }
    if (nk == 0) return;
    const int32_t r = atomicAdd(&ctr[kCtrCand], 1);
    if (r >= cand_cap) {
        atomicOr(err, kErrOverflow);
        return;
    }
    Cand c;
    c.t = t;
    c.s = s;
    c.nk = nk;
    c.best = -1;
    c.pad = 0;
    c.gain = 0;
    c.key = 0;
    for (int i = 0; i < 3; ++i) {
        c.k[i] = i < nk ? ks[i] : -1;
        c.e_gro[i] = -1;
    }
    c.e_shr = atomicAdd(&ctr[kCtrEval], 1);
    if (c.e_shr >= eval_cap) {
        atomicOr(err, kErrOverflow);
        return;
    }
    evals[c.e_shr] = shr;
    for (int i = 0; i < nk; ++i) {
        const obb_qbox& qk = q[ks[i]];
        int64_t dmin[3], dmax[3];
        proj3(U, F, t, qk.n, dmin, dmax);
        obb_qbox g = qk;
        bool grew = false;
        for (int a = 0; a < 3; ++a) {
            if (dmin[a] < g.b[2 * a]) {
                g.b[2 * a] = dmin[a];
                grew = true;
            }
            if (dmax[a] > g.b[2 * a + 1]) {
                g.b[2 * a + 1] = dmax[a];
                grew = true;
            }
        }
        if (grew) {
            int32_t ei = atomicAdd(&ctr[kCtrEval], 1);
            if (ei >= eval_cap) {
                atomicOr(err, kErrOverflow);
                return;
            }
            evals[ei] = g;
            c.e_gro[i] = ei;
        }
    }
    cand[r] = c;
}

// ------------------------------------------------------- gains + matching (a8)

__global__ void k_gains(Cand* __restrict__ cand, const int32_t* __restrict__ ctr,
                        const uint64_t* __restrict__ obv, const uint64_t* __restrict__ ecount,
                        unsigned long long* __restrict__ best, int64_t* __restrict__ stats)
{
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ctr[kCtrCand]) return;
    Cand c = cand[r];
    const int64_t rem = (int64_t)obv[c.s] - (int64_t)ecount[c.e_shr];
    int bi = -1;
    int64_t bg = 0;
    for (int i = 0; i < c.nk; ++i) {
        int64_t add = c.e_gro[i] >= 0 ? (int64_t)ecount[c.e_gro[i]] - (int64_t)obv[c.k[i]] : 0;
        int64_t g = rem - add;
        if (g > 0 && (bi < 0 || g > bg || (g == bg && c.k[i] < c.k[bi]))) {
            bi = i;
            bg = g;
        }
    }
    cand[r].best = bi;
    if (bi < 0) return;
    const unsigned long long key = ((unsigned long long)bg << 24) | (unsigned long long)(0xffffff - c.t);
    cand[r].gain = bg;
    cand[r].key = key;
    atomicMax(&best[c.s], key);
    atomicMax(&best[c.k[bi]], key);
    atomicAdd((unsigned long long*)&stats[kStProposals], 1ull);
}

__global__ void k_accept(const Cand* __restrict__ cand, const int32_t* __restrict__ ctr,
                         const unsigned long long* __restrict__ best, const obb_qbox* __restrict__ evals,
                         const uint64_t* __restrict__ ecount, int32_t* __restrict__ assign,
                         obb_qbox* __restrict__ q, uint64_t* __restrict__ obv, int32_t* __restrict__ size,
                         int64_t* __restrict__ stats, uint8_t* __restrict__ dirty, int32_t* __restrict__ level,
                         int32_t K, int32_t* __restrict__ mv)
{
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ctr[kCtrCand]) return;
    const Cand c = cand[r];
    if (c.best < 0) return;
    const int32_t k = c.k[c.best];
    if (best[c.s] != c.key || best[k] != c.key) return;
    assign[c.t] = k;
    // accepted moves touch disjoint clusters: one leaver or one joiner each
    mv[c.s] = c.t;
    mv[K + k] = c.t;
    for (int i = 0; i < 6; ++i) q[c.s].b[i] = evals[c.e_shr].b[i];
    obv[c.s] = ecount[c.e_shr];
    const int32_t eg = c.e_gro[c.best];
    if (eg >= 0) {
        for (int i = 0; i < 6; ++i) q[k].b[i] = evals[eg].b[i];
        obv[k] = ecount[eg];
    }
    size[c.s] -= 1;
    size[k] += 1;
    dirty[c.s] = 1;
    dirty[k] = 1;
    level[c.s] = 0;   // a new member set restarts the box-parameter search
    level[k] = 0;
    atomicAdd((unsigned long long*)&stats[kStAccepted], 1ull);
    atomicAdd((unsigned long long*)&stats[kStGain], (unsigned long long)c.gain);
}

__global__ void k_sum_points(const uint64_t* __restrict__ pts, const int32_t* __restrict__ d_n,
                             int64_t* __restrict__ stats)
{
    const int32_t n = *d_n;
    unsigned long long s = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += pts[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd((unsigned long long*)&stats[kStPoints], s);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd((unsigned long long*)&stats[kStEvals], (unsigned long long)n);
}

// ------------------------------------------------------- refit (a9-a11)

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

struct Comp {
    float s, c;
};

// s += x * y with the product error (FMA) and the addition error (TwoSum) kept in c
__device__ __forceinline__ void comp_fma(Comp& A, float x, float y)
{
    float p = __fmul_rn(x, y);
    float pe = fmaf(x, y, -p);
    float s, e;
    two_sum(A.s, p, s, e);
    A.s = s;
    A.c = __fadd_rn(A.c, __fadd_rn(e, pe));
}

__device__ __forceinline__ Comp comp_merge(Comp a, Comp b)
{
    float s, e;
    two_sum(a.s, b.s, s, e);
    return Comp{s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
}

// kComp = false: the same sums in plain FP32 (one rounding per fused
// multiply-add, no error terms) -- kept only to measure what compensation buys
template <int NT, bool kComp = true>
__global__ void __launch_bounds__(NT) k_moments(const float* __restrict__ V, const int32_t* __restrict__ F,
                                                const int32_t* __restrict__ members,
                                                const int32_t* __restrict__ start,
                                                const LatticeFrame* __restrict__ f, double* __restrict__ mom,
                                                const uint8_t* __restrict__ dirty)
{
    const int32_t k = blockIdx.x;
    if (dirty && !dirty[k]) return;
    const int32_t b0 = start[k], b1 = start[k + 1];
    // coordinates relative to the cluster's own origin (the first vertex of
    // its first member), subtracted exactly in FP64 and rounded once to FP32:
    // small clusters far from the lattice centre keep their spread instead of
    // losing it to cancellation in sum M / sum A - mu mu^T (the covariance
    // does not depend on the origin)
    double cx = 0.0, cy = 0.0, cz = 0.0;
    if (b1 > b0) {
        const float* O0 = V + 3 * (int64_t)F[3 * (int64_t)members[b0]];
        cx = (double)O0[0];
        cy = (double)O0[1];
        cz = (double)O0[2];
    }
    Comp acc[10];
    for (int i = 0; i < 10; ++i) acc[i] = Comp{0.f, 0.f};
    for (int32_t i = b0 + threadIdx.x; i < b1; i += NT) {
        const int32_t t = members[i];
        float P[3][3];
        for (int v = 0; v < 3; ++v) {
            const float* X = V + 3 * (int64_t)F[3 * t + v];
            P[v][0] = (float)__dsub_rn((double)X[0], cx);
            P[v][1] = (float)__dsub_rn((double)X[1], cy);
            P[v][2] = (float)__dsub_rn((double)X[2], cz);
        }
        float e1[3], e2[3];
        for (int b = 0; b < 3; ++b) {
            e1[b] = P[1][b] - P[0][b];
            e2[b] = P[2][b] - P[0][b];
        }
        float nx = fmaf(e1[1], e2[2], -e1[2] * e2[1]);
        float ny = fmaf(e1[2], e2[0], -e1[0] * e2[2]);
        float nz = fmaf(e1[0], e2[1], -e1[1] * e2[0]);
        float A = 0.5f * sqrtf(nx * nx + ny * ny + nz * nz);
        float m[3];
        for (int b = 0; b < 3; ++b) m[b] = (P[0][b] + P[1][b] + P[2][b]) / 3.0f;
        auto add = [&](Comp& a, float x, float y) {
            if constexpr (kComp) comp_fma(a, x, y);
            else a.s = __fmaf_rn(x, y, a.s);
        };
        add(acc[0], A, 1.0f);
        for (int b = 0; b < 3; ++b) add(acc[1 + b], A, m[b]);
        const float a12 = A / 12.0f;
        const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int qd = 0; qd < 6; ++qd) {
            const int x = ia[qd], y = ib[qd];
            float sxy = 9.0f * m[x] * m[y] + P[0][x] * P[0][y] + P[1][x] * P[1][y] + P[2][x] * P[2][y];
            add(acc[4 + qd], a12, sxy);
        }
    }
    __shared__ Comp sh[10][NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = 0; i < 10; ++i) {
        Comp x = acc[i];
        for (int o = 16; o > 0; o >>= 1) {
            Comp y{__shfl_xor_sync(0xffffffffu, x.s, o), __shfl_xor_sync(0xffffffffu, x.c, o)};
            // combine in lane order so every lane holds the same bits
            if constexpr (kComp) x = (lane & o) ? comp_merge(y, x) : comp_merge(x, y);
            else x = Comp{(lane & o) ? __fadd_rn(y.s, x.s) : __fadd_rn(x.s, y.s), 0.f};
        }
        if (lane == 0) sh[i][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        Comp x = sh[threadIdx.x][0];
        for (int i = 1; i < NT / 32; ++i) {
            if constexpr (kComp) x = comp_merge(x, sh[threadIdx.x][i]);
            else x.s = __fadd_rn(x.s, sh[threadIdx.x][i].s);
        }
        mom[10 * (int64_t)k + threadIdx.x] = (double)x.s + (double)x.c;
    }
}

// Cyclic Jacobi on the symmetric 3x3 covariance, FP64; frame rows = eigenvectors
// sorted by decreasing eigenvalue, rows 0 and 1 with a positive largest-magnitude
// component, row 2 = row 0 x row 1.
__device__ void jacobi3(const double c6[6], double R[9])
{
    double A[3][3] = {{c6[0], c6[3], c6[4]}, {c6[3], c6[1], c6[5]}, {c6[4], c6[5], c6[2]}};
    double Vm[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double fro = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) fro += A[i][j] * A[i][j];
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = 2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]);
        if (off <= 1e-30 * fro) break;
        for (int r = 0; r < 3; ++r) {
            const int p = r == 2 ? 1 : 0, qq = r == 0 ? 1 : 2;
            if (A[p][qq] == 0.0) continue;
            double theta = (A[qq][qq] - A[p][p]) / (2.0 * A[p][qq]);
            double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0);
            double s = t * c;
            for (int k = 0; k < 3; ++k) {
                double akp = A[k][p], akq = A[k][qq];
                A[k][p] = c * akp - s * akq;
                A[k][qq] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                double apk = A[p][k], aqk = A[qq][k];
                A[p][k] = c * apk - s * aqk;
                A[qq][k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                double vkp = Vm[k][p], vkq = Vm[k][qq];
                Vm[k][p] = c * vkp - s * vkq;
                Vm[k][qq] = s * vkp + c * vkq;
            }
        }
    }
    double ev[3] = {A[0][0], A[1][1], A[2][2]};
    int o[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (ev[o[j]] > ev[o[i]]) {
                int tmp = o[i];
                o[i] = o[j];
                o[j] = tmp;
            }
    for (int a = 0; a < 2; ++a) {
        double row[3] = {Vm[0][o[a]], Vm[1][o[a]], Vm[2][o[a]]};
        int big = 0;
        for (int b = 1; b < 3; ++b)
            if (fabs(row[b]) > fabs(row[big])) big = b;
        double sg = row[big] < 0.0 ? -1.0 : 1.0;
        for (int b = 0; b < 3; ++b) R[3 * a + b] = sg * row[b];
    }
    R[6] = R[1] * R[5] - R[2] * R[4];
    R[7] = R[2] * R[3] - R[0] * R[5];
    R[8] = R[0] * R[4] - R[1] * R[3];
}

__global__ void k_frames_from_moments(const double* __restrict__ mom, const double* __restrict__ fallback,
                                      int32_t K, double* __restrict__ out, const uint8_t* __restrict__ dirty)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K || (dirty && !dirty[k])) return;
    const double* m = mom + 10 * (int64_t)k;
    double* R = out + 9 * (int64_t)k;
    const double A = m[0];
    if (!(A > 0.0)) {
        for (int i = 0; i < 9; ++i) R[i] = fallback ? fallback[9 * (int64_t)k + i] : (i % 4 == 0 ? 1.0 : 0.0);
        return;
    }
    const double mu[3] = {m[1] / A, m[2] / A, m[3] / A};
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    double c6[6];
    for (int q = 0; q < 6; ++q) c6[q] = m[4 + q] / A - mu[ia[q]] * mu[ib[q]];
    jacobi3(c6, R);
}

// n_ab = rint(2^24 ((R_ab h_b) / h_max)), each step correctly rounded
__global__ void k_normals(const double* __restrict__ frames, int32_t K, const LatticeFrame* __restrict__ f,
                          obb_qbox* __restrict__ q, const uint8_t* __restrict__ active)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K || (active && !active[k])) return;
    const double hm = f->hmax;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double t = __dmul_rn(frames[9 * (int64_t)k + 3 * a + b], f->h[b]);
            t = __ddiv_rn(t, hm);
            t = __dmul_rn(t, 16777216.0);
            q[k].n[3 * a + b] = (int32_t)rint(t);
        }
    q[k].reserved = 0;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_tight(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                                              const int32_t* __restrict__ members,
                                              const int32_t* __restrict__ start, obb_qbox* __restrict__ q,
                                              int32_t per_cluster, const uint8_t* __restrict__ active)
{
    // box blockIdx.x belongs to cluster blockIdx.x / per_cluster
    const int32_t bx = blockIdx.x;
    if (active && !active[bx]) return;
    const int32_t cl = bx / per_cluster;
    const int32_t b0 = start[cl], b1 = start[cl + 1];
    const int32_t k = bx;
    int32_t n[9];
    for (int i = 0; i < 9; ++i) n[i] = q[k].n[i];
    int64_t v[6];
    for (int s = 0; s < 6; ++s) v[s] = (s & 1) ? INT64_MIN : INT64_MAX;
    for (int32_t i = b0 + threadIdx.x; i < b1; i += NT) {
        int64_t dmin[3], dmax[3];
        proj3(U, F, members[i], n, dmin, dmax);
        for (int a = 0; a < 3; ++a) {
            v[2 * a] = min(v[2 * a], dmin[a]);
            v[2 * a + 1] = max(v[2 * a + 1], dmax[a]);
        }
    }
    __shared__ int64_t sh[6][NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int s = 0; s < 6; ++s) {
        int64_t x = v[s];
        for (int o = 16; o > 0; o >>= 1) {
            int64_t y = (int64_t)__shfl_xor_sync(0xffffffffu, (long long)x, o);
            x = (s & 1) ? max(x, y) : min(x, y);
        }
        if (lane == 0) sh[s][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int s = threadIdx.x;
        int64_t x = sh[s][0];
        for (int i = 1; i < NT / 32; ++i) x = (s & 1) ? max(x, sh[s][i]) : min(x, sh[s][i]);
        q[k].b[s] = x;
    }
}

// The same with a warp per box (clusters of up to about a thousand
// triangles): no block barrier; min / max are exact, so the bounds are those
// of k_tight.
__global__ void __launch_bounds__(256) k_tight_warp(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                                                    const int32_t* __restrict__ members,
                                                    const int32_t* __restrict__ start, obb_qbox* __restrict__ q,
                                                    int32_t per_cluster, int32_t nbox,
                                                    const uint8_t* __restrict__ active)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t k = (int32_t)(g >> 5);
    const int lane = (int)(g & 31);
    if (k >= nbox) return;                 // warp-uniform
    if (active && !active[k]) return;      // warp-uniform
    const int32_t cl = k / per_cluster;
    const int32_t b0 = start[cl], b1 = start[cl + 1];
    int32_t n[9];
    for (int i = 0; i < 9; ++i) n[i] = q[k].n[i];
    int64_t v[6];
    for (int s = 0; s < 6; ++s) v[s] = (s & 1) ? INT64_MIN : INT64_MAX;
    for (int32_t i = b0 + lane; i < b1; i += 32) {
        int64_t dmin[3], dmax[3];
        proj3(U, F, members[i], n, dmin, dmax);
        for (int a = 0; a < 3; ++a) {
            v[2 * a] = min(v[2 * a], dmin[a]);
            v[2 * a + 1] = max(v[2 * a + 1], dmax[a]);
        }
    }
    for (int s = 0; s < 6; ++s) {
        int64_t x = v[s];
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t y = (int64_t)__shfl_xor_sync(0xffffffffu, (long long)x, o);
            x = (s & 1) ? max(x, y) : min(x, y);
        }
        if (lane == 0) q[k].b[s] = x;
    }
}

// Tight bounds of the layer's boxes q (per_cluster a cluster, active = null
// for all): a warp per box when clusters average up to 1,024 triangles,
// else a block.
void launch_tight(obb_ctx* ctx, const obb_layer* L, obb_qbox* q, int32_t per_cluster, const uint8_t* active,
                  cudaStream_t s)
{
    const obb_lattice* lat = L->lat;
    const int32_t nbox = L->K * per_cluster;
    if (L->T <= (int64_t)1024 * L->K)
        k_tight_warp<<<(unsigned)(((int64_t)nbox * 32 + 255) / 256), 256, 0, s>>>(
            lat->d_fixed, lat->mesh->d_tris, L->d_members, L->d_start, q, per_cluster, nbox, active);
    else
        k_tight<128><<<nbox, 128, 0, s>>>(lat->d_fixed, lat->mesh->d_tris, L->d_members, L->d_start, q, per_cluster,
                                          active);
}

__global__ void k_total(const uint64_t* __restrict__ obv, int32_t K, int64_t* __restrict__ out)
{
    unsigned long long s = 0;
    for (int32_t i = threadIdx.x; i < K; i += blockDim.x) s += obv[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ unsigned long long sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        *out = (int64_t)t;
    }
}

// End of a partition round inside a captured step: rounds run, moves so far,
// and the two conditions of the graph (run another round; rebuild the member
// lists first).  loop: [0] rounds run, [1] moves accepted before this round,
// [2] member-list rebuilds.
__global__ void k_round_end(const int64_t* __restrict__ stats, int64_t* __restrict__ loop, int32_t rounds,
                            cudaGraphConditionalHandle again, cudaGraphConditionalHandle rebuild)
{
    const int64_t acc = stats[kStAccepted];
    const int64_t moved = acc - loop[1];
    loop[1] = acc;
    loop[0] += 1;
    if (moved > 0) loop[2] += 1;
    cudaGraphSetConditional(again, (moved > 0 && loop[0] < rounds) ? 1u : 0u);
    cudaGraphSetConditional(rebuild, moved > 0 ? 1u : 0u);
}

// ------------------------------------------------------- surrogate screening

__device__ __forceinline__ uint32_t float_key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// predicted gain of each candidate record from predicted outer volumes of its boxes
__global__ void k_screen_score(const Cand* __restrict__ cand, const int32_t* __restrict__ ctr,
                               const uint64_t* __restrict__ obv, const float* __restrict__ pred,
                               unsigned long long* __restrict__ key)
{
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ctr[kCtrCand]) return;
    const Cand c = cand[r];
    const float rem = (float)obv[c.s] - pred[c.e_shr];
    float best = -3.0e38f;
    for (int i = 0; i < c.nk; ++i) {
        const float add = c.e_gro[i] >= 0 ? pred[c.e_gro[i]] - (float)obv[c.k[i]] : 0.f;
        best = fmaxf(best, rem - add);
    }
    key[r] = ((unsigned long long)float_key(best) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)c.t);
}

// Top-k of each source cluster in one pass: a record's key is inserted into
// its cluster's k slots (kept in descending order) by a chain of atomicMax
// operations, each slot keeping the larger of its value and the carried one
// and passing the smaller on; after every record has gone through, the slots
// hold the k largest keys of the cluster (keys are distinct: they end with the
// record's triangle).
__global__ void k_screen_insert(const Cand* __restrict__ cand, const int32_t* __restrict__ ctr,
                                const unsigned long long* __restrict__ key, int32_t topk,
                                unsigned long long* __restrict__ slot)
{
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ctr[kCtrCand]) return;
    unsigned long long v = key[r];
    unsigned long long* sl = slot + (int64_t)cand[r].s * kMaxTopk;
    for (int i = 0; i < topk && v; ++i) {
        const unsigned long long old = atomicMax(&sl[i], v);
        v = old < v ? old : v;
    }
}

// keep the records among their source cluster's top k (key at least the k-th
// slot) with their boxes in a new evaluation list; the others propose nothing
__global__ void k_screen_compact(Cand* __restrict__ cand, const int32_t* __restrict__ ctr,
                                 const unsigned long long* __restrict__ key, const unsigned long long* __restrict__ slot,
                                 int32_t topk, const obb_qbox* __restrict__ evals, obb_qbox* __restrict__ evals2,
                                 int32_t* __restrict__ n2)
{
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ctr[kCtrCand]) return;
    Cand c = cand[r];
    if (key[r] < slot[(int64_t)c.s * kMaxTopk + topk - 1]) {
        cand[r].nk = 0;
        return;
    }
    int need = 1;
    for (int i = 0; i < c.nk; ++i) need += c.e_gro[i] >= 0;
    int32_t base = atomicAdd(n2, need);
    evals2[base] = evals[c.e_shr];
    c.e_shr = base++;
    for (int i = 0; i < c.nk; ++i)
        if (c.e_gro[i] >= 0) {
            evals2[base] = evals[c.e_gro[i]];
            c.e_gro[i] = base++;
        }
    cand[r] = c;
}

__global__ void k_refit_accept_mapped(const double* __restrict__ newframe, const obb_qbox* __restrict__ newq,
                                      const uint64_t* __restrict__ cnt, const int32_t* __restrict__ map,
                                      const int32_t* __restrict__ n2, double* __restrict__ frames,
                                      obb_qbox* __restrict__ q, uint64_t* __restrict__ obv,
                                      int64_t* __restrict__ stats)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n2) return;
    const int32_t k = map[i];
    if (cnt[i] < obv[k]) {
        for (int t = 0; t < 9; ++t) frames[9 * (int64_t)k + t] = newframe[9 * (int64_t)k + t];
        q[k] = newq[k];
        obv[k] = cnt[i];
        atomicAdd((unsigned long long*)&stats[kStRefits], 1ull);
    }
}

// clusters whose membership changed since their last covariance refit
__global__ void k_dirty_compact(const uint8_t* __restrict__ dirty, const uint8_t* __restrict__ screen, int32_t K,
                                const obb_qbox* __restrict__ newq, obb_qbox* __restrict__ evals2,
                                int32_t* __restrict__ map, int32_t* __restrict__ n2)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K || !dirty[k] || (screen && !screen[k])) return;
    const int32_t i = atomicAdd(n2, 1);
    evals2[i] = newq[k];
    map[i] = k;
}

// surrogate screen of the covariance refit: keep predicted improvements (5% slack)
__global__ void k_refit_keep(const float* __restrict__ pred, const uint64_t* __restrict__ obv, int32_t K,
                             uint8_t* __restrict__ keep)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    keep[k] = pred[k] < (float)obv[k] * 1.05f;
}

// ---- box-parameter descent (the perturbation search of the box update) ----
//
// Probe p of cluster k rotates k's frame about its own axis a = p / 2 by
// +-theta with the rational rotation cos = (1 - t^2) / (1 + t^2),
// sin = 2 t / (1 + t^2), t = 2^-(5 + level_k): every probe frame is a fixed
// sequence of correctly rounded FP64 operations.
constexpr int kProbes = 6;
constexpr int kDescentMaxLevel = 8;

__global__ void k_probe_frames(const double* __restrict__ frames, const int32_t* __restrict__ level, int32_t K,
                               double* __restrict__ pf, uint8_t* __restrict__ active)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * kProbes) return;
    const int32_t k = i / kProbes, p = i % kProbes;
    const bool on = level[k] < kDescentMaxLevel;
    active[i] = on;
    if (!on) return;
    const double t = ldexp(1.0, -(5 + level[k]));
    const double t2 = __dmul_rn(t, t);
    const double den = __dadd_rn(1.0, t2);
    const double c = __ddiv_rn(__dsub_rn(1.0, t2), den);
    const double sn = __ddiv_rn(__dmul_rn(2.0, t), den);
    const double ss = (p & 1) ? -sn : sn;
    const int a = p >> 1, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    const double* R = frames + 9 * (int64_t)k;
    double* O = pf + 9 * (int64_t)i;
    for (int j = 0; j < 3; ++j) {
        O[3 * a + j] = R[3 * a + j];
        O[3 * b1 + j] = __dadd_rn(__dmul_rn(c, R[3 * b1 + j]), __dmul_rn(ss, R[3 * b2 + j]));
        O[3 * b2 + j] = __dsub_rn(__dmul_rn(c, R[3 * b2 + j]), __dmul_rn(ss, R[3 * b1 + j]));
    }
}

// surrogate screen of the probes: keep the m lowest predicted outer volumes of each cluster
__global__ void k_probe_keep(const float* __restrict__ pred, int32_t K, int32_t m, uint8_t* __restrict__ active)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    float v[kProbes];
    for (int p = 0; p < kProbes; ++p) v[p] = active[k * kProbes + p] ? pred[k * kProbes + p] : 3.0e38f;
    for (int p = 0; p < kProbes; ++p) {
        if (!active[k * kProbes + p]) continue;
        int rank = 0;
        for (int o = 0; o < kProbes; ++o) rank += (v[o] < v[p]) || (v[o] == v[p] && o < p);
        if (rank >= m) active[k * kProbes + p] = 0;
    }
}

__global__ void k_probe_compact(const uint8_t* __restrict__ active, int32_t n, const obb_qbox* __restrict__ pq,
                                obb_qbox* __restrict__ evals2, int32_t* __restrict__ map, int32_t* __restrict__ n2)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !active[i]) return;
    const int32_t j = atomicAdd(n2, 1);
    evals2[j] = pq[i];
    map[j] = i;
}

__global__ void k_probe_best(const uint64_t* __restrict__ cnt, const int32_t* __restrict__ map,
                             const int32_t* __restrict__ n2, unsigned long long* __restrict__ best)
{
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *n2) return;
    const int32_t i = map[j];
    atomicMin(&best[i / kProbes], ((unsigned long long)cnt[j] << 3) | (unsigned long long)(i % kProbes));
}

// keep the best probe when its exact outer volume is strictly smaller, else halve theta
__global__ void k_probe_apply(const unsigned long long* __restrict__ best, const double* __restrict__ pf,
                              const obb_qbox* __restrict__ pq, int32_t K, int32_t* __restrict__ level,
                              double* __restrict__ frames, obb_qbox* __restrict__ q, uint64_t* __restrict__ obv,
                              int64_t* __restrict__ stats)
{
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K || level[k] >= kDescentMaxLevel) return;
    const unsigned long long b = best[k];
    const uint64_t c = b >> 3;
    if (b != ~0ull && c < obv[k]) {
        const int32_t i = k * kProbes + (int32_t)(b & 7);
        for (int t = 0; t < 9; ++t) frames[9 * (int64_t)k + t] = pf[9 * (int64_t)i + t];
        q[k] = pq[i];
        obv[k] = c;
        atomicAdd((unsigned long long*)&stats[kStRefits], 1ull);
    } else {
        level[k] += 1;
    }
}

}  // namespace

// -------------------------------------------------------------- host side

// Per-layer scratch that is not part of the layer's state, allocated with it.
struct LayerMem {
    int32_t* skeys[2] = {nullptr, nullptr};   // radix sort: keys and values between passes
    int32_t* svals[2] = {nullptr, nullptr};
    int32_t* scnt = nullptr;                   // [bins * tiles] digit counts, then offsets
    int32_t* soff = nullptr;
    int32_t* sbsum = nullptr;
    unsigned int* sticket = nullptr;           // zero between launches (the fused scan's ticket)
    int sort_passes = 1, sort_bits = 0;
    int32_t* ctr = nullptr;
    Cand* cand = nullptr;
    obb_qbox* evals = nullptr;
    uint64_t* ecount = nullptr;
    uint64_t* epoints = nullptr;
    double* mom = nullptr;
    double* newframe = nullptr;
    obb_qbox* newq = nullptr;
    uint64_t* ncount = nullptr;
    uint64_t* pcount = nullptr;     // [K * 6] exact counts of the probes
    int32_t* dK = nullptr;          // device copy of K
    // surrogate screening scratch (allocated when a surrogate is attached)
    float* feats = nullptr;
    float* pred = nullptr;
    unsigned long long* skey = nullptr;
    unsigned long long* slot = nullptr;
    obb_qbox* evals2 = nullptr;
    int32_t* n2 = nullptr;
    int32_t* map = nullptr;
    uint8_t* dirty = nullptr;       // [K] membership changed since the last covariance refit
    uint8_t* keep = nullptr;        // [K * 6] refit / probe activity
    int32_t* level = nullptr;       // [K] descent step level (theta = 2^-(5 + level))
    double* pframes = nullptr;      // [K * 6][9] probe frames
    obb_qbox* pq = nullptr;         // [K * 6] probe boxes
    unsigned long long* pbest = nullptr;  // [K]
    int32_t cand_cap = 0, eval_cap = 0;
    // a whole Lloyd iteration captured as one CUDA graph (see lloyd_step_graph)
    cudaGraphExec_t gexec = nullptr;
    int gkey[4] = {-1, -1, -1, -1};   // rounds, refit mode, descent steps, counting-tile generation
    int64_t* loop = nullptr;          // [0] rounds run, [1] moves before the round, [2] rebuilds, [3] total
    CountScratch cscr{};              // the graph's own counting scratch (fixed addresses)
    void* cscr_mem = nullptr;
    int64_t g_round = 0, g_rebuild = 0, g_post = 0;   // kernel launches per round, per rebuild, after the loop
    bool members_valid = false;
    // incremental member lists: mv [2K] the last round's leavers and joiners
    // per cluster (-1 = none), the new list and starts built beside the old
    int32_t* mv = nullptr;
    int32_t* mnew = nullptr;   // [T]
    int32_t* snew = nullptr;   // [K + 1]
    bool incr_ok = false;      // the lists were valid before the moves mv records (and nothing else moved)
};

static LayerMem* mem_of(const obb_layer* L) { return static_cast<LayerMem*>(L->aux); }

template <class T>
static cudaError_t dalloc(T** p, size_t n, cudaStream_t s)
{
    return pool_alloc(reinterpret_cast<void**>(p), sizeof(T) * (n > 0 ? n : 1), s);
}

static obb_status sort_members(obb_ctx* ctx, obb_layer* L);

// The member lists after the moves of one round (mv), from the lists
// before them: new starts from the sizes k_accept kept, the segments moved
// into place by k_members_update, copied back (the lists' addresses are
// fixed: captured graphs read them).
static obb_status update_members(obb_ctx* ctx, obb_layer* L)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    const int32_t K = L->K;
    launch_scan_i32(ctx, L->d_size, M->snew, M->dK);
    k_members_update<<<(unsigned)(((int64_t)K * 32 + 255) / 256), 256, 0, s>>>(L->d_members, L->d_start, M->snew,
                                                                               M->mv, K, M->mnew);
    note_launch(ctx);
    OBB_CK(ctx, cudaMemcpyAsync(L->d_members, M->mnew, sizeof(int32_t) * L->T, cudaMemcpyDeviceToDevice, s));
    OBB_CK(ctx, cudaMemcpyAsync(L->d_start, M->snew, sizeof(int32_t) * (K + 1), cudaMemcpyDeviceToDevice, s));
    OBB_CK(ctx, cudaGetLastError());
    M->members_valid = true;
    return OBB_OK;
}

obb_status rebuild_members(obb_ctx* ctx, obb_layer* L)
{
    LayerMem* M = mem_of(L);
    if (M->incr_ok) return update_members(ctx, L);
    return sort_members(ctx, L);
}

// The member lists from scratch: a stable radix sort of the triangles by
// cluster; the move records are cleared.
static obb_status sort_members(obb_ctx* ctx, obb_layer* L)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    const int64_t T = L->T;
    const bool one_pass = M->sort_passes == 1;
    OBB_CK(ctx, cudaMemsetAsync(M->mv, 0xff, sizeof(int32_t) * 2 * L->K, s));
    // cluster sizes: added up by the first pass's counts (with one pass the
    // sort's own offsets give sizes and starts)
    if (!one_pass) OBB_CK(ctx, cudaMemsetAsync(L->d_size, 0, sizeof(int32_t) * L->K, s));
    // the member list: a stable radix sort of the triangles by cluster
    const int32_t ntiles = (int32_t)((T + kSortTile - 1) / kSortTile);
    const int bins = 1 << M->sort_bits;
    const int64_t nc = (int64_t)bins * ntiles;
    const bool fused = nc <= kSortFusedScanMax;
    const unsigned nsb = (unsigned)((nc + kSortScanBlock - 1) / kSortScanBlock);
    const int32_t* kin = L->d_assign;
    const int32_t* vin = nullptr;
    for (int p = 0; p < M->sort_passes; ++p) {
        const bool last = p + 1 == M->sort_passes;
        const int shift = p * M->sort_bits;
        int32_t* kout = last ? nullptr : M->skeys[p & 1];
        int32_t* vout = last ? L->d_members : M->svals[p & 1];
        k_sort_count<<<ntiles, kSortThreads, sizeof(int32_t) * bins, s>>>(
            kin, T, shift, bins, ntiles, p == 0 ? L->K : 0, p == 0 && !one_pass ? L->d_size : nullptr, M->scnt,
            fused ? M->soff : nullptr, M->sticket, ctx->d_err);
        if (!fused) {
            k_sort_sums<<<nsb, kSortThreads, 0, s>>>(M->scnt, nc, M->sbsum);
            k_sort_offsets<<<nsb, kSortThreads, 0, s>>>(M->scnt, nc, M->sbsum, M->soff);
        }
        k_sort_scatter<<<ntiles, kSortThreads, sort_scatter_smem(bins), s>>>(
            kin, vin, T, shift, bins, ntiles, M->soff, kout, vout, L->K, one_pass ? L->d_start : nullptr,
            one_pass ? L->d_size : nullptr);
        note_launch(ctx, fused ? 2 : 4);
        if (p == 0 && !one_pass) launch_scan_i32(ctx, L->d_size, L->d_start, M->dK);   // cluster starts
        kin = kout;
        vin = vout;
    }
    OBB_CK(ctx, cudaGetLastError());
    M->members_valid = true;
    M->incr_ok = true;
    return OBB_OK;
}

void layer_destroy(obb_layer* L)
{
    if (!L) return;
    cudaStream_t s = L->ctx ? L->ctx->stream : nullptr;
    LayerMem* M = mem_of(L);
    void* ptrs[] = {L->d_assign, L->d_parent, L->d_frames, L->d_q, L->d_obv, L->d_size, L->d_start,
                    L->d_members, L->d_ext, L->d_best, L->d_stats};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, s);
    if (M) {
        if (M->gexec) cudaGraphExecDestroy(M->gexec);
        if (M->loop) cudaFreeAsync(M->loop, s);
        if (M->cscr_mem) cudaFreeAsync(M->cscr_mem, s);
        void* mp[] = {M->skeys[0], M->skeys[1], M->svals[0], M->svals[1], M->scnt, M->soff, M->sbsum, M->sticket, M->ctr, M->cand, M->evals, M->ecount, M->epoints, M->mom,
                      M->newframe, M->newq, M->ncount, M->dK, M->feats, M->pred, M->skey,
                      M->slot, M->evals2, M->n2, M->map, M->dirty, M->keep, M->level,
                      M->pframes, M->pq, M->pbest, M->pcount, M->mv, M->mnew, M->snew};
        for (void* p : mp)
            if (p) cudaFreeAsync(p, s);
        delete M;
    }
    delete L;
}

// Frames (given, or from the covariance), normals, tight bounds, exact OBV.
static obb_status init_boxes(obb_ctx* ctx, obb_layer* L, const double* d_frames, const double* d_fallback)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    const obb_lattice* lat = L->lat;
    const int K = L->K;
    if (d_frames) {
        OBB_CK(ctx, cudaMemcpyAsync(L->d_frames, d_frames, sizeof(double) * 9 * K, cudaMemcpyDeviceToDevice, s));
    } else {
        k_moments<kNT><<<K, kNT, 0, s>>>(lat->mesh->d_verts, lat->mesh->d_tris, L->d_members, L->d_start,
                                         lat->d_frame, M->mom, nullptr);
        note_launch(ctx);
        k_frames_from_moments<<<(K + 31) / 32, 32, 0, s>>>(M->mom, d_fallback, K, L->d_frames, nullptr);
        note_launch(ctx);
    }
    k_normals<<<(K + 31) / 32, 32, 0, s>>>(L->d_frames, K, lat->d_frame, L->d_q, nullptr);
    note_launch(ctx);
    launch_tight(ctx, L, L->d_q, 1, nullptr, s);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return count_boxes(ctx, lat, L->d_q, M->dK, K, L->d_obv, nullptr);
}

obb_status layer_create(obb_ctx* ctx, const obb_lattice* lat, const int32_t* d_assign, const int32_t* d_parent,
                        int32_t K, const double* d_frames, const double* d_fallback, obb_layer** out)
{
    cudaStream_t s = ctx->stream;
    const int64_t T = lat->mesh->nt;
    if (K < 1) return fail(ctx, OBB_ERR_ARG, "K must be >= 1");
    if (T >= (int64_t(1) << 24)) return fail(ctx, OBB_ERR_RANGE, "at most 2^24 - 1 triangles");
    if (K > T) return fail(ctx, OBB_ERR_EMPTY_CLUSTER, "more clusters than triangles");
    obb_layer* L = new obb_layer();
    LayerMem* M = new LayerMem();
    L->aux = M;
    L->ctx = ctx;
    L->lat = lat;
    L->K = K;
    L->T = T;
    M->cand_cap = 6 * K + 32;
    M->eval_cap = 4 * M->cand_cap;
    {
        int end_bit = 0;   // cluster indices < 2^end_bit
        while ((1 << end_bit) < K) ++end_bit;
        M->sort_passes = std::max(1, (end_bit + kSortMaxBits - 1) / kSortMaxBits);
        M->sort_bits = (end_bit + M->sort_passes - 1) / M->sort_passes;
    }
    const int64_t sort_tiles = (T + kSortTile - 1) / kSortTile;
    const int64_t sort_nc = ((int64_t)1 << M->sort_bits) * sort_tiles;
    cudaError_t e = cudaSuccess;
#define A_(x)                        \
    if (e == cudaSuccess) e = (x);
    A_(dalloc(&L->d_assign, T, s));
    A_(dalloc(&L->d_parent, K, s));
    A_(dalloc(&L->d_frames, 9 * (size_t)K, s));
    A_(dalloc(&L->d_q, K, s));
    A_(dalloc(&L->d_obv, K, s));
    A_(dalloc(&L->d_size, K, s));
    A_(dalloc(&L->d_start, (size_t)K + 1, s));
    A_(dalloc(&L->d_members, T, s));
    A_(dalloc(&L->d_ext, K, s));
    A_(dalloc(&L->d_best, K, s));
    A_(dalloc(&L->d_stats, kStCount, s));
    for (int p = 0; p + 1 < M->sort_passes; ++p) {
        A_(dalloc(&M->skeys[p], T, s));
        A_(dalloc(&M->svals[p], T, s));
    }
    A_(dalloc(&M->scnt, sort_nc, s));
    A_(dalloc(&M->soff, sort_nc, s));
    A_(dalloc(&M->sbsum, (sort_nc + kSortScanBlock - 1) / kSortScanBlock, s));
    A_(dalloc(&M->sticket, 1, s));
    if (e == cudaSuccess) e = cudaMemsetAsync(M->sticket, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sort_scatter_smem(1 << kSortMaxBits));
    A_(dalloc(&M->ctr, kCtrCount, s));
    A_(dalloc(&M->cand, M->cand_cap, s));
    A_(dalloc(&M->evals, M->eval_cap, s));
    A_(dalloc(&M->ecount, M->eval_cap, s));
    A_(dalloc(&M->epoints, std::max<int64_t>(M->eval_cap, (int64_t)kProbes * K), s));
    A_(dalloc(&M->mom, 10 * (size_t)K, s));
    A_(dalloc(&M->newframe, 9 * (size_t)K, s));
    A_(dalloc(&M->newq, K, s));
    A_(dalloc(&M->ncount, K, s));
    A_(dalloc(&M->dK, 1, s));
    const size_t cap2 = (size_t)std::max<int64_t>(M->eval_cap, (int64_t)kProbes * K);
    A_(dalloc(&M->evals2, cap2, s));
    A_(dalloc(&M->map, cap2, s));
    A_(dalloc(&M->n2, 1, s));
    A_(dalloc(&M->dirty, K, s));
    A_(dalloc(&M->keep, (size_t)kProbes * K, s));
    A_(dalloc(&M->level, K, s));
    A_(dalloc(&M->pframes, (size_t)9 * kProbes * K, s));
    A_(dalloc(&M->pq, (size_t)kProbes * K, s));
    A_(dalloc(&M->pbest, K, s));
    A_(dalloc(&M->pcount, (size_t)kProbes * K, s));
    A_(dalloc(&M->mv, 2 * (size_t)K, s));
    A_(dalloc(&M->mnew, T, s));
    A_(dalloc(&M->snew, (size_t)K + 1, s));
#undef A_
    if (e != cudaSuccess) {
        layer_destroy(L);
        return cuda_fail(ctx, e, "layer allocation");
    }
    OBB_CK(ctx, cudaMemcpyAsync(L->d_assign, d_assign, sizeof(int32_t) * T, cudaMemcpyDeviceToDevice, s));
    OBB_CK(ctx, cudaMemcpyAsync(L->d_parent, d_parent, sizeof(int32_t) * K, cudaMemcpyDeviceToDevice, s));
    OBB_CK(ctx, cudaMemsetAsync(L->d_best, 0, sizeof(unsigned long long) * K, s));
    OBB_CK(ctx, cudaMemsetAsync(L->d_stats, 0, sizeof(int64_t) * kStCount, s));
    OBB_CK(ctx, cudaMemsetAsync(M->dirty, 1, K, s));
    OBB_CK(ctx, cudaMemsetAsync(M->level, 0, sizeof(int32_t) * K, s));
    obb_status st = set_device_int(ctx, M->dK, K);
    if (st == OBB_OK) st = rebuild_members(ctx, L);
    if (st == OBB_OK) {
        k_check_nonempty<<<(K + 255) / 256, 256, 0, s>>>(L->d_size, K, ctx->d_err);
        note_launch(ctx);
        st = check_device_error(ctx);   // assignment range / empty clusters before any box work
    }
    if (st == OBB_OK) st = init_boxes(ctx, L, d_frames, d_fallback);
    if (st == OBB_OK) st = check_device_error(ctx);
    if (st != OBB_OK) {
        layer_destroy(L);
        return st;
    }
    *out = L;
    return OBB_OK;
}

// Phases of a step around its exact counts: a batched step runs every
// layer's kPre part (which records its counting request), counts all the
// requests in one launch, then runs every layer's kPost part.
enum { kPre = 1, kPost = 2, kWhole = 3 };

// One partition round (a6-a8) on ctx->stream, without host synchronisation.
static obb_status round_body(obb_ctx* ctx, obb_layer* L, int phase = kWhole)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    const obb_lattice* lat = L->lat;
    const obb_mesh* mesh = lat->mesh;
    const int K = L->K;
    const bool screened = L->mlp && L->topk > 0;
    const obb_qbox* evals = screened ? M->evals2 : M->evals;
    const int32_t* n_eval = screened ? M->n2 : M->ctr + kCtrEval;
    if (phase & kPre) {
        launch_extents(ctx, L, s);
        OBB_CK(ctx, cudaMemsetAsync(M->ctr, 0, sizeof(int32_t) * kCtrCount, s));
        OBB_CK(ctx, cudaMemsetAsync(L->d_best, 0, sizeof(unsigned long long) * K, s));
        k_candidates<<<(unsigned)((6 * (int64_t)K + 127) / 128), 128, 0, s>>>(
            lat->d_fixed, mesh->d_tris, mesh->d_adj, K, L->d_assign, L->d_parent, L->d_size, L->d_ext, L->d_q,
            M->cand, M->evals, M->ctr, M->cand_cap, M->eval_cap, ctx->d_err);
        note_launch(ctx);
        if (screened) {
            // surrogate screening: predicted gains keep the top-k candidates of each
            // source cluster; only their boxes are counted exactly
            OBB_TRY(surrogate_predict(ctx, L->mlp, lat, M->evals, M->ctr + kCtrEval, M->eval_cap, M->feats, M->pred));
            const unsigned cb0 = (unsigned)((M->cand_cap + 127) / 128);
            k_screen_score<<<cb0, 128, 0, s>>>(M->cand, M->ctr, L->d_obv, M->pred, M->skey);
            OBB_CK(ctx, cudaMemsetAsync(M->slot, 0, sizeof(unsigned long long) * kMaxTopk * K, s));
            k_screen_insert<<<cb0, 128, 0, s>>>(M->cand, M->ctr, M->skey, L->topk, M->slot);
            OBB_CK(ctx, cudaMemsetAsync(M->n2, 0, sizeof(int32_t), s));
            k_screen_compact<<<cb0, 128, 0, s>>>(M->cand, M->ctr, M->skey, M->slot, L->topk, M->evals, M->evals2,
                                                 M->n2);
            note_launch(ctx, 3);
        }
        OBB_TRY(count_boxes(ctx, lat, evals, n_eval, M->eval_cap, M->ecount, M->epoints));
    }
    if (phase & kPost) {
        k_sum_points<<<32, 256, 0, s>>>(M->epoints, n_eval, L->d_stats);
        note_launch(ctx);
        const unsigned cb = (unsigned)((M->cand_cap + 127) / 128);
        k_gains<<<cb, 128, 0, s>>>(M->cand, M->ctr, L->d_obv, M->ecount, L->d_best, L->d_stats);
        note_launch(ctx);
        k_accept<<<cb, 128, 0, s>>>(M->cand, M->ctr, L->d_best, evals, M->ecount, L->d_assign, L->d_q, L->d_obv,
                                    L->d_size, L->d_stats, M->dirty, M->level, K, M->mv);
        note_launch(ctx);
    }
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

static obb_status lloyd_step_graph(obb_ctx* ctx, obb_layer* L, int rounds, int refit_mode, int dsteps,
                                   obb_step_stats* st);

obb_status lloyd_step(obb_ctx* ctx, obb_layer* L, const obb_step_opts* opts, obb_step_stats* st)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    const int rounds = (opts && opts->rounds > 0) ? opts->rounds : 16;
    const int refit_mode = opts ? opts->refit : 1;
    const int dsteps = (opts && opts->descent_steps > 0) ? opts->descent_steps : 2;
    if (opts && opts->graph && !L->mlp) return lloyd_step_graph(ctx, L, rounds, refit_mode, dsteps, st);
    OBB_CK(ctx, cudaMemsetAsync(L->d_stats, 0, sizeof(int64_t) * kStCount, s));
    int64_t* h = host_stats(ctx);
    int ran = 0;
    int64_t before = 0;
    for (int r = 0; r < rounds; ++r) {
        if (!M->members_valid) OBB_TRY(rebuild_members(ctx, L));
        OBB_TRY(round_body(ctx, L));
        OBB_CK(ctx, cudaMemcpyAsync(h, L->d_stats, sizeof(int64_t) * kStCount, cudaMemcpyDeviceToHost, s));
        OBB_CK(ctx, cudaStreamSynchronize(s));
        ++ran;
        const int64_t moved = h[kStAccepted] - before;
        before = h[kStAccepted];
        if (moved > 0) M->members_valid = false;
        if (moved == 0) break;
    }
    OBB_TRY(layer_box_update(ctx, L, refit_mode, dsteps));
    return layer_finish_stats(ctx, L, ran, st);
}

// The Lloyd iteration as one CUDA graph: the partition rounds run in a
// device-side WHILE loop (a conditional node whose condition the last kernel of
// each round sets), the member lists are rebuilt inside an IF node after a
// round that moved triangles, and the box update follows.  The graph is
// captured once per (rounds, refit, descent steps, counting tile) and
// relaunched; it runs the same kernels in the same order as the host loop, so
// results are identical, without a host round trip per round.  Its counting
// launches use scratch of their own (fixed addresses) and are not profiled one
// by one.
static obb_status lloyd_step_graph(obb_ctx* ctx, obb_layer* L, int rounds, int refit_mode, int dsteps,
                                   obb_step_stats* st)
{
    LayerMem* M = mem_of(L);
    const int K = L->K;
    cudaStream_t s = ctx->stream;
    if (!M->members_valid) OBB_TRY(rebuild_members(ctx, L));
    if (!M->gexec || M->gkey[0] != rounds || M->gkey[1] != refit_mode || M->gkey[2] != dsteps ||
        M->gkey[3] != ctx->tile_gen) {
        if (M->gexec) {
            OBB_CK(ctx, cudaGraphExecDestroy(M->gexec));
            M->gexec = nullptr;
        }
        if (!M->loop) OBB_CK(ctx, pool_alloc((void**)&M->loop, sizeof(int64_t) * 4, s));
        if (!M->cscr_mem) {
            const int64_t cap = std::max<int64_t>({(int64_t)M->eval_cap, (int64_t)kProbes * K, (int64_t)K});
            const size_t pb = (sizeof(BoxPrep) * cap + 255) / 256 * 256;
            const size_t tb = sizeof(int64_t) * (2 * cap + 2 + cap / kScanBlock + 1);
            OBB_CK(ctx, pool_alloc(&M->cscr_mem, pb + tb, s));
            char* b = static_cast<char*>(M->cscr_mem);
            M->cscr.prep = reinterpret_cast<BoxPrep*>(b);
            M->cscr.tiles = reinterpret_cast<int64_t*>(b + pb);
            M->cscr.bsum = M->cscr.tiles + 2 * cap + 2;
            M->cscr.cap = cap;
        }
        OBB_CK(ctx, cudaStreamSynchronize(s));
        cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
        for (auto& c : cs) OBB_CK(ctx, cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
        const cudaStream_t saved_stream = ctx->stream;
        const int32_t saved_prof = ctx->prof;
        const int64_t saved_launches = ctx->launches;
        ctx->prof = 0;
        ctx->count_scratch = &M->cscr;
        M->members_valid = true;   // valid on entry; the graph rebuilds them after moving rounds
        cudaGraph_t g = nullptr;
        obb_status rc = OBB_OK;
        cudaError_t e = cudaSuccess;
        int depth = 0;   // captures still open
        auto ck = [&](cudaError_t x) {
            if (e == cudaSuccess && x != cudaSuccess) e = x;
            return e == cudaSuccess;
        };
        do {
            ctx->stream = cs[0];
            if (!ck(cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeThreadLocal))) break;
            depth = 1;
            ck(cudaMemsetAsync(L->d_stats, 0, sizeof(int64_t) * kStCount, cs[0]));
            ck(cudaMemsetAsync(M->loop, 0, sizeof(int64_t) * 4, cs[0]));
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            if (!ck(cudaStreamGetCaptureInfo(cs[0], &cst, nullptr, &g, &deps, nullptr, &nd))) break;
            cudaGraphConditionalHandle again, rebuild;
            if (!ck(cudaGraphConditionalHandleCreate(&again, g, 1, cudaGraphCondAssignDefault))) break;
            cudaGraphNodeParams wp = {};
            wp.type = cudaGraphNodeTypeConditional;
            wp.conditional.handle = again;
            wp.conditional.type = cudaGraphCondTypeWhile;
            wp.conditional.size = 1;
            cudaGraphNode_t wn;
            if (!ck(cudaGraphAddNode(&wn, g, deps, nullptr, nd, &wp))) break;
            cudaGraph_t body = wp.conditional.phGraph_out[0];
            if (!ck(cudaStreamUpdateCaptureDependencies(cs[0], &wn, nullptr, 1, cudaStreamSetCaptureDependencies)))
                break;
            if (!ck(cudaGraphConditionalHandleCreate(&rebuild, body, 0, cudaGraphCondAssignDefault))) break;
            // the round
            ctx->stream = cs[1];
            if (!ck(cudaStreamBeginCaptureToGraph(cs[1], body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
                break;
            depth = 2;
            const int64_t l0 = ctx->launches;
            rc = round_body(ctx, L);
            if (rc != OBB_OK) break;
            k_round_end<<<1, 1, 0, cs[1]>>>(L->d_stats, M->loop, rounds, again, rebuild);
            note_launch(ctx);
            if (!ck(cudaGetLastError())) break;
            M->g_round = ctx->launches - l0;
            cudaGraph_t bg = nullptr;
            if (!ck(cudaStreamGetCaptureInfo(cs[1], &cst, nullptr, &bg, &deps, nullptr, &nd))) break;
            cudaGraphNodeParams ip = {};
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = rebuild;
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            cudaGraphNode_t in;
            if (!ck(cudaGraphAddNode(&in, bg, deps, nullptr, nd, &ip))) break;
            cudaGraph_t ibody = ip.conditional.phGraph_out[0];
            if (!ck(cudaStreamUpdateCaptureDependencies(cs[1], &in, nullptr, 1, cudaStreamSetCaptureDependencies)))
                break;
            // the member lists after a round that moved triangles
            ctx->stream = cs[2];
            if (!ck(cudaStreamBeginCaptureToGraph(cs[2], ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
                break;
            depth = 3;
            const int64_t l1 = ctx->launches;
            rc = rebuild_members(ctx, L);
            if (rc != OBB_OK) break;
            M->g_rebuild = ctx->launches - l1;
            if (!ck(cudaStreamEndCapture(cs[2], &ibody))) break;
            depth = 2;
            if (!ck(cudaStreamEndCapture(cs[1], &bg))) break;
            depth = 1;
            // the box update and the layer total
            ctx->stream = cs[0];
            const int64_t l2 = ctx->launches;
            rc = layer_box_update(ctx, L, refit_mode, dsteps);
            if (rc != OBB_OK) break;
            k_total<<<1, 1024, 0, cs[0]>>>(L->d_obv, K, M->loop + 3);
            note_launch(ctx);
            M->g_post = ctx->launches - l2;
            if (!ck(cudaGetLastError())) break;
            if (!ck(cudaStreamEndCapture(cs[0], &g))) break;
            depth = 0;
            if (!ck(cudaGraphInstantiate(&M->gexec, g, 0))) break;
        } while (false);
        // close whatever capture is still open, innermost first
        for (int d = depth; d >= 1; --d) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs[d - 1], &junk);
            if (junk && d == 1) cudaGraphDestroy(junk);
        }
        if (g && depth == 0) cudaGraphDestroy(g);
        ctx->stream = saved_stream;
        ctx->prof = saved_prof;
        ctx->count_scratch = nullptr;
        ctx->launches = saved_launches;
        for (auto& c : cs) cudaStreamDestroy(c);
        if (rc != OBB_OK) return rc;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "capture of the Lloyd iteration");
        M->gkey[0] = rounds;
        M->gkey[1] = refit_mode;
        M->gkey[2] = dsteps;
        M->gkey[3] = ctx->tile_gen;
    }
    OBB_CK(ctx, cudaGraphLaunch(M->gexec, s));
    int64_t* h = host_stats(ctx);
    OBB_CK(ctx, cudaMemcpyAsync(h, L->d_stats, sizeof(int64_t) * kStCount, cudaMemcpyDeviceToHost, s));
    OBB_CK(ctx, cudaMemcpyAsync(h + kStCount, M->loop, sizeof(int64_t) * 4, cudaMemcpyDeviceToHost, s));
    OBB_TRY(check_device_error(ctx));
    M->members_valid = true;
    const int64_t ran = h[kStCount], rebuilds = h[kStCount + 2];
    note_launch(ctx, (int)(M->g_round * ran + M->g_rebuild * rebuilds + M->g_post));
    if (st) {
        st->rounds_run = (int32_t)ran;
        st->refits_accepted = (int32_t)h[kStRefits];
        st->proposals = h[kStProposals];
        st->moves = h[kStAccepted];
        st->gain = h[kStGain];
        st->box_evals = h[kStEvals];
        st->points_counted = (uint64_t)h[kStPoints];
        st->total_obv = (uint64_t)h[kStCount + 3];
    }
    return OBB_OK;
}

// Covariance refit (a9-a11) of the clusters whose membership changed (the
// others would rebuild the frame they already tried and keep their box), in
// the phases of a batched step.
static obb_status refit_covariance(obb_ctx* ctx, obb_layer* L, int phase)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    const obb_lattice* lat = L->lat;
    const obb_mesh* mesh = lat->mesh;
    const int K = L->K;
    if (phase & kPre) {
        if (!M->members_valid) OBB_TRY(rebuild_members(ctx, L));
        k_moments<kNT><<<K, kNT, 0, s>>>(mesh->d_verts, mesh->d_tris, L->d_members, L->d_start, lat->d_frame,
                                         M->mom, M->dirty);
        k_frames_from_moments<<<(K + 31) / 32, 32, 0, s>>>(M->mom, L->d_frames, K, M->newframe, M->dirty);
        k_normals<<<(K + 31) / 32, 32, 0, s>>>(M->newframe, K, lat->d_frame, M->newq, M->dirty);
        launch_tight(ctx, L, M->newq, 1, M->dirty, s);
        note_launch(ctx, 4);
        const uint8_t* screen = nullptr;
        if (L->mlp) {
            // surrogate screen: exact counts only for the boxes predicted to improve
            OBB_TRY(surrogate_predict(ctx, L->mlp, lat, M->newq, M->dK, K, M->feats, M->pred));
            k_refit_keep<<<(K + 127) / 128, 128, 0, s>>>(M->pred, L->d_obv, K, M->keep);
            note_launch(ctx);
            screen = M->keep;
        }
        OBB_CK(ctx, cudaMemsetAsync(M->n2, 0, sizeof(int32_t), s));
        k_dirty_compact<<<(K + 127) / 128, 128, 0, s>>>(M->dirty, screen, K, M->newq, M->evals2, M->map, M->n2);
        note_launch(ctx);
        OBB_TRY(count_boxes(ctx, lat, M->evals2, M->n2, K, M->ncount, M->epoints));
    }
    if (phase & kPost) {
        k_sum_points<<<32, 256, 0, s>>>(M->epoints, M->n2, L->d_stats);
        k_refit_accept_mapped<<<(K + 127) / 128, 128, 0, s>>>(M->newframe, M->newq, M->ncount, M->map, M->n2,
                                                              L->d_frames, L->d_q, L->d_obv, L->d_stats);
        note_launch(ctx, 2);
        OBB_CK(ctx, cudaMemsetAsync(M->dirty, 0, K, s));
    }
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

// Box update of a layer after its partition rounds (Sec. 4.2.1 step 2):
// refit_mode bit 0 the covariance refit of the clusters whose membership
// changed, bit 1 `dsteps` rotation-descent steps.  Adds to the layer's
// device counters.
obb_status layer_box_update(obb_ctx* ctx, obb_layer* L, int refit_mode, int dsteps)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    const obb_lattice* lat = L->lat;
    const int K = L->K;
    if (refit_mode & 1) OBB_TRY(refit_covariance(ctx, L, kWhole));
    if (refit_mode & 2) {
        // box-parameter descent: six rotation probes per cluster per step, the
        // best kept when its exact outer volume is strictly smaller
        if (!M->members_valid) OBB_TRY(rebuild_members(ctx, L));
        const int32_t KP = kProbes * K;
        for (int step = 0; step < dsteps; ++step) {
            k_probe_frames<<<(KP + 127) / 128, 128, 0, s>>>(L->d_frames, M->level, K, M->pframes, M->keep);
            k_normals<<<(KP + 31) / 32, 32, 0, s>>>(M->pframes, KP, lat->d_frame, M->pq, M->keep);
            launch_tight(ctx, L, M->pq, kProbes, M->keep, s);
            note_launch(ctx, 3);
            if (L->mlp) {
                OBB_CK(ctx, ctx->kdev.reserve(sizeof(int32_t), s));
                OBB_TRY(set_device_int(ctx, ctx->kdev.as<int32_t>(), KP));
                OBB_TRY(surrogate_predict(ctx, L->mlp, lat, M->pq, ctx->kdev.as<int32_t>(), KP, M->feats, M->pred));
                k_probe_keep<<<(K + 127) / 128, 128, 0, s>>>(M->pred, K, L->topk > 0 ? L->topk : 2, M->keep);
                note_launch(ctx);
            }
            OBB_CK(ctx, cudaMemsetAsync(M->n2, 0, sizeof(int32_t), s));
            k_probe_compact<<<(KP + 127) / 128, 128, 0, s>>>(M->keep, KP, M->pq, M->evals2, M->map, M->n2);
            note_launch(ctx);
            OBB_TRY(count_boxes(ctx, lat, M->evals2, M->n2, KP, M->pcount, M->epoints));
            OBB_CK(ctx, cudaMemsetAsync(M->pbest, 0xff, sizeof(unsigned long long) * K, s));
            k_sum_points<<<32, 256, 0, s>>>(M->epoints, M->n2, L->d_stats);
            k_probe_best<<<(KP + 127) / 128, 128, 0, s>>>(M->pcount, M->map, M->n2, M->pbest);
            k_probe_apply<<<(K + 127) / 128, 128, 0, s>>>(M->pbest, M->pframes, M->pq, K, M->level, L->d_frames, L->d_q,
                                                          L->d_obv, L->d_stats);
            note_launch(ctx, 3);
        }
        OBB_CK(ctx, cudaGetLastError());
    }
    return OBB_OK;
}

// ------------------------------------------------------- batched layers

namespace {
__global__ void k_gather_accepted(int64_t* const* __restrict__ stats, int32_t n, int64_t* __restrict__ out)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = stats[i][kStAccepted];
}

// Block per layer of a batch: its device counters and its total outer
// volume (as k_total sums it) into out[i][0..kStCount], one copy for all.
__global__ void k_batch_totals(int64_t* const* __restrict__ stats, const uint64_t* const* __restrict__ obv,
                               const int32_t* __restrict__ Ks, int64_t* __restrict__ out)
{
    const int32_t i = blockIdx.x;
    const uint64_t* o = obv[i];
    const int32_t K = Ks[i];
    unsigned long long s = 0;
    for (int32_t k = threadIdx.x; k < K; k += blockDim.x) s += o[k];
    for (int q = 16; q > 0; q >>= 1) s += __shfl_xor_sync(0xffffffffu, s, q);
    __shared__ unsigned long long sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    int64_t* row = out + (int64_t)i * (kStCount + 1);
    if (threadIdx.x < kStCount) row[threadIdx.x] = stats[i][threadIdx.x];
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        row[kStCount] = (int64_t)t;
    }
}

// resets the context's request list on every path out of a collecting phase
struct DeferGuard {
    obb_ctx* ctx;
    DeferGuard(obb_ctx* c, std::vector<CountReq>* reqs) : ctx(c) { ctx->count_defer = reqs; }
    ~DeferGuard() { ctx->count_defer = nullptr; }
};
}  // namespace

obb_status batch_create(obb_ctx* ctx, obb_layer* const* layers, int32_t n, obb_batch* B)
{
    cudaStream_t s = ctx->stream;
    B->ctx = ctx;
    B->layers.assign(layers, layers + n);
    std::vector<int64_t*> ptrs(n);
    for (int32_t i = 0; i < n; ++i) ptrs[i] = layers[i]->d_stats;
    OBB_CK(ctx, B->stat_ptrs.reserve(sizeof(int64_t*) * n + sizeof(int64_t) * n, s));
    OBB_CK(ctx, cudaMemcpyAsync(B->stat_ptrs.p, ptrs.data(), sizeof(int64_t*) * n, cudaMemcpyHostToDevice, s));
    OBB_CK(ctx, cudaMallocHost((void**)&B->h_acc, sizeof(int64_t) * n));
    // the totals of all layers in one launch: outer-volume pointers, K, then [n][kStCount + 1] results
    std::vector<const uint64_t*> obv(n);
    std::vector<int32_t> Ks(n);
    for (int32_t i = 0; i < n; ++i) {
        obv[i] = layers[i]->d_obv;
        Ks[i] = layers[i]->K;
    }
    const size_t fo = (sizeof(uint64_t*) * n + sizeof(int32_t) * n + 255) / 256 * 256;
    OBB_CK(ctx, B->fin.reserve(fo + sizeof(int64_t) * (kStCount + 1) * n, s));
    OBB_CK(ctx, cudaMemcpyAsync(B->fin.p, obv.data(), sizeof(uint64_t*) * n, cudaMemcpyHostToDevice, s));
    OBB_CK(ctx, cudaMemcpyAsync(B->fin.as<char>() + sizeof(uint64_t*) * n, Ks.data(), sizeof(int32_t) * n,
                                cudaMemcpyHostToDevice, s));
    OBB_CK(ctx, cudaMallocHost((void**)&B->h_fin, sizeof(int64_t) * (kStCount + 1) * n));
    OBB_CK(ctx, cudaStreamSynchronize(s));
    return OBB_OK;
}

// Captures every layer's partition-round phases as CUDA graphs (nothing
// runs): round_body's phase before the counting launch, once with the
// member-list update after a moving round in front, and its phase after the
// counting launch.
// Each layer's counting request is recorded by the capture (the counting
// itself stays deferred to the batch's one counting launch per round).
// The same six kinds are also captured for the whole batch at once, each
// layer on one of the batch's streams, for the phases in which every layer
// runs with its list in the same state: one graph launch instead of n.
static obb_status batch_capture(obb_ctx* ctx, obb_batch* B)
{
    const int32_t n = (int32_t)B->layers.size();
    // entries 0..n-1 of each kind's vector are the layers' graphs, entry n
    // the whole batch's
    for (auto* v : {&B->g_pre, &B->g_pre_rebuild, &B->g_post, &B->g_rpre, &B->g_rpre_rebuild, &B->g_rpost})
        v->assign(n + 1, nullptr);
    for (auto* v : {&B->k_pre, &B->k_pre_rebuild, &B->k_post, &B->k_rpre, &B->k_rpre_rebuild, &B->k_rpost})
        v->assign(n + 1, 0);
    B->req.assign(n, CountReq{});
    B->rreq.assign(n, CountReq{});
    for (int p = 0; p < obb_batch::kBatchStreams; ++p)
        if (!B->par[p]) OBB_CK(ctx, cudaStreamCreateWithFlags(&B->par[p], cudaStreamNonBlocking));
    for (auto& e : B->ev)
        if (!e) OBB_CK(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    OBB_CK(ctx, cudaStreamSynchronize(ctx->stream));
    cudaStream_t cs = nullptr;
    OBB_CK(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const cudaStream_t saved_stream = ctx->stream;
    const int32_t saved_prof = ctx->prof;
    const int64_t saved_launches = ctx->launches;
    ctx->prof = 0;
    ctx->stream = cs;
    obb_status rc = OBB_OK;
    cudaError_t e = cudaSuccess;
    for (int32_t i = 0; i < n && rc == OBB_OK && e == cudaSuccess; ++i) {
        obb_layer* L = B->layers[i];
        LayerMem* M = mem_of(L);
        const bool valid = M->members_valid;
        // kinds: 0 round before the count, 1 the same after the member-list
        // update, 2 round after the count; 3, 4, 5 the same for the covariance
        // refit
        cudaGraphExec_t* gx[6] = {&B->g_pre[i], &B->g_pre_rebuild[i], &B->g_post[i],
                                  &B->g_rpre[i], &B->g_rpre_rebuild[i], &B->g_rpost[i]};
        int32_t* kx[6] = {&B->k_pre[i], &B->k_pre_rebuild[i], &B->k_post[i],
                          &B->k_rpre[i], &B->k_rpre_rebuild[i], &B->k_rpost[i]};
        for (int kind = 0; kind < 6 && rc == OBB_OK && e == cudaSuccess; ++kind) {
            const bool before_count = kind % 3 < 2, refit = kind >= 3;
            std::vector<CountReq> rq;
            ctx->count_defer = before_count ? &rq : nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) break;
            const int64_t l0 = ctx->launches;
            M->members_valid = kind % 3 != 1;   // updated first in kinds 1 and 4 (after a moving round)
            if (kind % 3 == 1) rc = update_members(ctx, L);
            if (rc == OBB_OK)
                rc = refit ? refit_covariance(ctx, L, before_count ? kPre : kPost)
                           : round_body(ctx, L, before_count ? kPre : kPost);
            cudaGraph_t g = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (e == cudaSuccess) e = e2;
            cudaGraphExec_t x = nullptr;
            if (rc == OBB_OK && e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
            if (g) cudaGraphDestroy(g);
            *gx[kind] = x;
            *kx[kind] = (int32_t)(ctx->launches - l0);
            if (kind % 3 == 0 && rc == OBB_OK) {
                if (rq.size() == 1) (refit ? B->rreq : B->req)[i] = rq[0];
                else rc = fail(ctx, OBB_ERR_STATE, "a batched phase made other than one count");
            }
        }
        M->members_valid = valid;   // the captures ran nothing
    }
    // the whole-batch graphs: every layer's phase on the batch's streams,
    // forked from and joined to the capture origin inside the graph
    constexpr int P = obb_batch::kBatchStreams;
    for (int kind = 0; kind < 6 && rc == OBB_OK && e == cudaSuccess; ++kind) {
        const bool before_count = kind % 3 < 2, refit = kind >= 3;
        std::vector<CountReq> rq;
        ctx->count_defer = before_count ? &rq : nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        const int64_t l0 = ctx->launches;
        cudaError_t x = cudaEventRecord(B->ev[P], cs);
        for (int p = 0; p < P && x == cudaSuccess; ++p) x = cudaStreamWaitEvent(B->par[p], B->ev[P], 0);
        for (int32_t i = 0; i < n && rc == OBB_OK && x == cudaSuccess; ++i) {
            obb_layer* L = B->layers[i];
            LayerMem* M = mem_of(L);
            const bool valid = M->members_valid;
            M->members_valid = kind % 3 != 1;
            ctx->stream = B->par[i % P];
            if (kind % 3 == 1) rc = update_members(ctx, L);
            if (rc == OBB_OK)
                rc = refit ? refit_covariance(ctx, L, before_count ? kPre : kPost)
                           : round_body(ctx, L, before_count ? kPre : kPost);
            M->members_valid = valid;
        }
        for (int p = 0; p < P && x == cudaSuccess; ++p) {
            x = cudaEventRecord(B->ev[p], B->par[p]);
            if (x == cudaSuccess) x = cudaStreamWaitEvent(cs, B->ev[p], 0);
        }
        ctx->stream = cs;
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        e = x != cudaSuccess ? x : e2;
        cudaGraphExec_t* gx[6] = {&B->g_pre[n], &B->g_pre_rebuild[n], &B->g_post[n],
                                  &B->g_rpre[n], &B->g_rpre_rebuild[n], &B->g_rpost[n]};
        int32_t* kx[6] = {&B->k_pre[n], &B->k_pre_rebuild[n], &B->k_post[n],
                          &B->k_rpre[n], &B->k_rpre_rebuild[n], &B->k_rpost[n]};
        if (rc == OBB_OK && e == cudaSuccess) e = cudaGraphInstantiate(gx[kind], g, 0);
        if (g) cudaGraphDestroy(g);
        *kx[kind] = (int32_t)(ctx->launches - l0);
        if (before_count && rc == OBB_OK && (int32_t)rq.size() != n)
            rc = fail(ctx, OBB_ERR_STATE, "a whole-batch phase made other than one count per layer");
    }
    ctx->count_defer = nullptr;
    ctx->stream = saved_stream;
    ctx->prof = saved_prof;
    ctx->launches = saved_launches;
    cudaStreamDestroy(cs);
    if (rc != OBB_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture of the batched rounds");
    B->graphs = true;
    return OBB_OK;
}

void batch_destroy(obb_batch* B)
{
    if (!B) return;
    cudaStream_t s = B->ctx ? B->ctx->stream : nullptr;
    for (auto* v : {&B->g_pre, &B->g_pre_rebuild, &B->g_post, &B->g_rpre, &B->g_rpre_rebuild, &B->g_rpost})
        for (cudaGraphExec_t x : *v)
            if (x) cudaGraphExecDestroy(x);
    B->fin.release(s);
    if (B->h_fin) cudaFreeHost(B->h_fin);
    for (cudaStream_t p : B->par)
        if (p) cudaStreamDestroy(p);
    for (cudaEvent_t e : B->ev)
        if (e) cudaEventDestroy(e);
    B->tables.release(s);
    B->scratch.release(s);
    B->stat_ptrs.release(s);
    if (B->h_acc) cudaFreeHost(B->h_acc);
    delete B;
}

// One Lloyd iteration of every layer of the batch: the partition rounds of
// all layers still moving run together, each round's exact counts of all of
// them in one counting launch (count_flush); then the covariance refit of all
// layers, again with one counting launch; the rotation descent, when asked
// for, runs layer by layer.  Each layer runs the same kernels in the same
// order as obb_lloyd_step, so its state and statistics are the same.
obb_status batch_lloyd_step(obb_ctx* ctx, obb_batch* B, const obb_step_opts* opts, obb_step_stats* stats)
{
    cudaStream_t s = ctx->stream;
    const int32_t n = (int32_t)B->layers.size();
    const int rounds = (opts && opts->rounds > 0) ? opts->rounds : 16;
    const int refit_mode = opts ? opts->refit : 1;
    const int dsteps = (opts && opts->descent_steps > 0) ? opts->descent_steps : 2;
    std::vector<int64_t> before(n, 0);
    std::vector<int> ran(n, 0);
    std::vector<char> active(n, 1);
    for (obb_layer* L : B->layers) OBB_CK(ctx, cudaMemsetAsync(L->d_stats, 0, sizeof(int64_t) * kStCount, s));
    std::vector<CountReq> reqs;
    int64_t* const* d_ptrs = B->stat_ptrs.as<int64_t*>();
    int64_t* d_acc = reinterpret_cast<int64_t*>(B->stat_ptrs.as<char>() + sizeof(int64_t*) * n);
    // rounds as per-layer graphs (not with surrogate screening, whose
    // prediction allocates on first use)
    bool use_graphs = true;
    for (obb_layer* L : B->layers) use_graphs = use_graphs && !L->mlp;
    if (use_graphs && !B->graphs) OBB_TRY(batch_capture(ctx, B));
    constexpr int P = obb_batch::kBatchStreams;
    // the parallel streams start after everything on the context stream, and it waits for them
    auto fork = [&]() -> cudaError_t {
        cudaError_t x = cudaEventRecord(B->ev[P], s);
        for (int p = 0; p < P && x == cudaSuccess; ++p) x = cudaStreamWaitEvent(B->par[p], B->ev[P], 0);
        return x;
    };
    auto join = [&]() -> cudaError_t {
        cudaError_t x = cudaSuccess;
        for (int p = 0; p < P && x == cudaSuccess; ++p) {
            x = cudaEventRecord(B->ev[p], B->par[p]);
            if (x == cudaSuccess) x = cudaStreamWaitEvent(s, B->ev[p], 0);
        }
        return x;
    };
    // lists moved by something other than Lloyd moves are sorted from scratch
    // on the context stream, before the graphs (whose rebuild is the update)
    auto sort_stale = [&]() -> obb_status {
        for (obb_layer* L : B->layers) {
            LayerMem* M = mem_of(L);
            if (!M->members_valid && !M->incr_ok) OBB_TRY(sort_members(ctx, L));
        }
        return OBB_OK;
    };
    // a phase where every layer runs and every list is in the same state
    // (all valid, or all to be updated) is one whole-batch graph launch:
    // -1 none, else the per-layer kind offset (0 valid, 1 update first)
    auto uniform = [&](bool all_active) -> int {
        if (!all_active || n == 0) return -1;
        const bool v0 = mem_of(B->layers[0])->members_valid;
        for (obb_layer* L : B->layers)
            if (mem_of(L)->members_valid != v0) return -1;
        return v0 ? 0 : 1;
    };
    auto launch_all = [&](int kind) -> cudaError_t {
        const cudaGraphExec_t gx[6] = {B->g_pre[n], B->g_pre_rebuild[n], B->g_post[n],
                                       B->g_rpre[n], B->g_rpre_rebuild[n], B->g_rpost[n]};
        const int32_t kx[6] = {B->k_pre[n], B->k_pre_rebuild[n], B->k_post[n],
                               B->k_rpre[n], B->k_rpre_rebuild[n], B->k_rpost[n]};
        note_launch(ctx, kx[kind]);
        return cudaGraphLaunch(gx[kind], s);
    };
    int32_t n_active = n;
    for (int r = 0; r < rounds; ++r) {
        reqs.clear();
        if (use_graphs) OBB_TRY(sort_stale());
        const int u = use_graphs ? uniform(n_active == n) : -1;
        if (u >= 0) {
            OBB_CK(ctx, launch_all(u));
            for (int32_t i = 0; i < n; ++i) {
                mem_of(B->layers[i])->members_valid = true;
                reqs.push_back(B->req[i]);
            }
        } else if (use_graphs) {
            OBB_CK(ctx, fork());
            int j = 0;
            for (int32_t i = 0; i < n; ++i) {
                if (!active[i]) continue;
                LayerMem* M = mem_of(B->layers[i]);
                const bool rb = !M->members_valid;
                OBB_CK(ctx, cudaGraphLaunch(rb ? B->g_pre_rebuild[i] : B->g_pre[i], B->par[j++ % P]));
                note_launch(ctx, rb ? B->k_pre_rebuild[i] : B->k_pre[i]);
                M->members_valid = true;
                reqs.push_back(B->req[i]);
            }
            OBB_CK(ctx, join());
        } else {
            DeferGuard guard(ctx, &reqs);
            for (int32_t i = 0; i < n; ++i) {
                if (!active[i]) continue;
                obb_layer* L = B->layers[i];
                if (!mem_of(L)->members_valid) OBB_TRY(rebuild_members(ctx, L));
                OBB_TRY(round_body(ctx, L, kPre));
            }
        }
        OBB_TRY(count_flush(ctx, reqs, B->tables, B->scratch));
        const bool post_all = use_graphs && n_active == n;
        if (post_all) OBB_CK(ctx, launch_all(2));
        else if (use_graphs) OBB_CK(ctx, fork());
        for (int32_t i = 0, j = 0; i < n; ++i) {
            if (!active[i]) continue;
            if (post_all) {
                // launched above
            } else if (use_graphs) {
                OBB_CK(ctx, cudaGraphLaunch(B->g_post[i], B->par[j++ % P]));
                note_launch(ctx, B->k_post[i]);
            } else {
                OBB_TRY(round_body(ctx, B->layers[i], kPost));
            }
            ++ran[i];
        }
        if (use_graphs && !post_all) OBB_CK(ctx, join());
        k_gather_accepted<<<(n + 127) / 128, 128, 0, s>>>(d_ptrs, n, d_acc);
        note_launch(ctx);
        OBB_CK(ctx, cudaMemcpyAsync(B->h_acc, d_acc, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
        OBB_CK(ctx, cudaStreamSynchronize(s));
        bool any = false;
        for (int32_t i = 0; i < n; ++i) {
            if (!active[i]) continue;
            const int64_t moved = B->h_acc[i] - before[i];
            before[i] = B->h_acc[i];
            if (moved > 0) {
                mem_of(B->layers[i])->members_valid = false;
                any = true;
            } else {
                active[i] = 0;
                --n_active;
            }
        }
        if (!any) break;
    }
    if (refit_mode & 1) {
        reqs.clear();
        if (use_graphs) OBB_TRY(sort_stale());
        const int u = use_graphs ? uniform(true) : -1;
        if (u >= 0) {
            OBB_CK(ctx, launch_all(3 + u));
            for (int32_t i = 0; i < n; ++i) {
                mem_of(B->layers[i])->members_valid = true;
                reqs.push_back(B->rreq[i]);
            }
        } else if (use_graphs) {
            OBB_CK(ctx, fork());
            for (int32_t i = 0; i < n; ++i) {
                LayerMem* M = mem_of(B->layers[i]);
                const bool rb = !M->members_valid;
                OBB_CK(ctx, cudaGraphLaunch(rb ? B->g_rpre_rebuild[i] : B->g_rpre[i], B->par[i % P]));
                note_launch(ctx, rb ? B->k_rpre_rebuild[i] : B->k_rpre[i]);
                M->members_valid = true;
                reqs.push_back(B->rreq[i]);
            }
            OBB_CK(ctx, join());
        } else {
            DeferGuard guard(ctx, &reqs);
            for (obb_layer* L : B->layers) OBB_TRY(refit_covariance(ctx, L, kPre));
        }
        OBB_TRY(count_flush(ctx, reqs, B->tables, B->scratch));
        if (use_graphs) {
            OBB_CK(ctx, launch_all(5));
        } else {
            for (obb_layer* L : B->layers) OBB_TRY(refit_covariance(ctx, L, kPost));
        }
    }
    if (refit_mode & 2)
        for (obb_layer* L : B->layers) OBB_TRY(layer_box_update(ctx, L, 2, dsteps));
    if (stats) {
        // every layer's counters and total in one launch and one copy
        const size_t fo = (sizeof(uint64_t*) * n + sizeof(int32_t) * n + 255) / 256 * 256;
        int64_t* d_fin = reinterpret_cast<int64_t*>(B->fin.as<char>() + fo);
        k_batch_totals<<<n, 256, 0, s>>>(d_ptrs, B->fin.as<const uint64_t*>(),
                                          reinterpret_cast<const int32_t*>(B->fin.as<char>() + sizeof(uint64_t*) * n),
                                          d_fin);
        note_launch(ctx);
        OBB_CK(ctx, cudaMemcpyAsync(B->h_fin, d_fin, sizeof(int64_t) * (kStCount + 1) * n, cudaMemcpyDeviceToHost,
                                    s));
        OBB_TRY(check_device_error(ctx));
        for (int32_t i = 0; i < n; ++i) {
            const int64_t* h = B->h_fin + (int64_t)i * (kStCount + 1);
            obb_step_stats& st = stats[i];
            st.rounds_run = ran[i];
            st.refits_accepted = (int32_t)h[kStRefits];
            st.proposals = h[kStProposals];
            st.moves = h[kStAccepted];
            st.gain = h[kStGain];
            st.box_evals = h[kStEvals];
            st.points_counted = (uint64_t)h[kStPoints];
            st.total_obv = (uint64_t)h[kStCount];
        }
    }
    return check_device_error(ctx);
}

// Copies the layer's device counters and total outer volume into *st (if
// non-null) after a step that ran `ran` partition rounds; synchronises.
obb_status layer_finish_stats(obb_ctx* ctx, obb_layer* L, int ran, obb_step_stats* st)
{
    cudaStream_t s = ctx->stream;
    const int K = L->K;
    int64_t* h = host_stats(ctx);
    if (st) {
        OBB_CK(ctx, ctx->tmp_d.reserve(sizeof(int64_t), s));
        k_total<<<1, 1024, 0, s>>>(L->d_obv, K, ctx->tmp_d.as<int64_t>());
        note_launch(ctx);
        OBB_CK(ctx, cudaMemcpyAsync(h, L->d_stats, sizeof(int64_t) * kStCount, cudaMemcpyDeviceToHost, s));
        OBB_CK(ctx, cudaMemcpyAsync(h + kStCount, ctx->tmp_d.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        OBB_TRY(check_device_error(ctx));
        st->rounds_run = ran;
        st->refits_accepted = (int32_t)h[kStRefits];
        st->proposals = h[kStProposals];
        st->moves = h[kStAccepted];
        st->gain = h[kStGain];
        st->box_evals = h[kStEvals];
        st->points_counted = (uint64_t)h[kStPoints];
        st->total_obv = (uint64_t)h[kStCount];
    }
    return OBB_OK;
}


uint8_t* layer_dirty(obb_layer* L) { return mem_of(L)->dirty; }
const int32_t* layer_dev_K(obb_layer* L) { return mem_of(L)->dK; }
int32_t* layer_level(obb_layer* L) { return mem_of(L)->level; }

obb_status layer_members(obb_ctx* ctx, obb_layer* L)
{
    return mem_of(L)->members_valid ? OBB_OK : rebuild_members(ctx, L);
}

void layer_members_changed(obb_layer* L)
{
    mem_of(L)->members_valid = false;
    mem_of(L)->incr_ok = false;   // moved by something that keeps no move records
}

void launch_sum_points(obb_ctx* ctx, const uint64_t* d_pts, const int32_t* d_n, int64_t* d_stats)
{
    k_sum_points<<<32, 256, 0, ctx->stream>>>(d_pts, d_n, d_stats);
    note_launch(ctx);
}

obb_status layer_set_surrogate(obb_ctx* ctx, obb_layer* L, const obb_mlp* mlp, int32_t topk)
{
    cudaStream_t s = ctx->stream;
    LayerMem* M = mem_of(L);
    if (topk < 0 || topk > kMaxTopk) return fail(ctx, OBB_ERR_ARG, "topk must be in [0, 16]");
    if (mlp && !M->feats) {
        const size_t cap2 = (size_t)std::max<int64_t>(M->eval_cap, (int64_t)kProbes * L->K);
        cudaError_t e = dalloc(&M->feats, cap2 * kSurrogateInputs, s);
        if (e == cudaSuccess) e = dalloc(&M->pred, cap2, s);
        if (e == cudaSuccess) e = dalloc(&M->skey, M->cand_cap, s);
        if (e == cudaSuccess) e = dalloc(&M->slot, (size_t)kMaxTopk * L->K, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "surrogate screening scratch");
    }
    L->mlp = mlp;
    L->topk = topk;
    return OBB_OK;
}

obb_status layer_moments(obb_ctx* ctx, obb_layer* L, int32_t compensated, double* out)
{
    cudaStream_t s = ctx->stream;
    OBB_TRY(layer_members(ctx, L));
    const obb_lattice* lat = L->lat;
    double* d = nullptr;
    OBB_CK(ctx, pool_alloc((void**)&d, sizeof(double) * 10 * L->K, s));
    if (compensated)
        k_moments<kNT, true><<<L->K, kNT, 0, s>>>(lat->mesh->d_verts, lat->mesh->d_tris, L->d_members, L->d_start,
                                                  lat->d_frame, d, nullptr);
    else
        k_moments<kNT, false><<<L->K, kNT, 0, s>>>(lat->mesh->d_verts, lat->mesh->d_tris, L->d_members, L->d_start,
                                                   lat->d_frame, d, nullptr);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    OBB_CK(ctx, cudaMemcpyAsync(out, d, sizeof(double) * 10 * L->K, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(d, s);
    return check_device_error(ctx);
}

obb_status layer_last_candidates(obb_ctx* ctx, const obb_layer* L, obb_qbox* out, uint64_t* counts, int64_t cap,
                                 int64_t* n)
{
    LayerMem* M = mem_of(L);
    int32_t ne = 0;
    OBB_CK(ctx, cudaMemcpyAsync(&ne, M->ctr + kCtrEval, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    OBB_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t m = ne < cap ? ne : cap;
    if (m > 0) {
        OBB_CK(ctx, cudaMemcpyAsync(out, M->evals, sizeof(obb_qbox) * m, cudaMemcpyDeviceToHost, ctx->stream));
        if (counts)
            OBB_CK(ctx, cudaMemcpyAsync(counts, M->ecount, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost, ctx->stream));
    }
    *n = ne;
    return check_device_error(ctx);
}

}  // namespace obbv
