// Patch division by flooding (Sec. 4.2.1 step 1), on the GPU.
//
// The boxes of a layer keep their frames and centres; the triangles are
// re-partitioned.  A triangle may only join a box of its group (the parent
// of its current cluster), so groups are independent and run side by side.
//   priority   per triangle: distance from its centroid (FP64, the mean of its
//              three float vertices) to the nearest centre of its group's
//              boxes, rounded to float, packed with the triangle index;
//   seeds      per group, its boxes in index order each take the nearest
//              untaken triangle of the group;
//   waves      a triangle is available once an edge neighbour of its group is
//              assigned (a group with none available falls back to its
//              unassigned triangle of smallest priority, with every box of the
//              group as candidate).  Exact mode takes the available triangle of
//              smallest priority per group per wave -- the paper's sequential
//              priority-queue order, since groups never interact -- and the
//              wavefront mode takes every available triangle at once.  A taken
//              triangle joins the candidate box (boxes holding one of its
//              neighbours) whose exact outer volume grows least (Eq. 12-13,
//              ties -> smaller box); in the wavefront mode several triangles
//              may join one box in a wave, each evaluated against the box as the
//              wave found it, and the box is recounted afterwards.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace obbv {
namespace {

constexpr int kMaxFloodCand = 8;   // boxes one triangle may choose between
constexpr int kFT = 128;

struct FloodRec {
    int32_t t, nk;
    int32_t k[kMaxFloodCand];
    int32_t e[kMaxFloodCand];   // eval slot of the grown box, -1 if unchanged
};

__device__ __forceinline__ unsigned long long tri_key(const float* __restrict__ V, const int32_t* __restrict__ F,
                                                      int32_t t, const double* c)
{
    double d2 = 0.0;
    for (int b = 0; b < 3; ++b) {
        double m = __dadd_rn((double)V[3 * (int64_t)F[3 * t] + b], (double)V[3 * (int64_t)F[3 * t + 1] + b]);
        m = __dadd_rn(m, (double)V[3 * (int64_t)F[3 * t + 2] + b]);
        m = __ddiv_rn(m, 3.0);
        const double d = __dsub_rn(m, c[b]);
        d2 = __dadd_rn(d2, __dmul_rn(d, d));
    }
    const float f = __double2float_rn(__dsqrt_rn(d2));
    return ((unsigned long long)__float_as_uint(f) << 32) | (unsigned long long)(uint32_t)t;
}

__device__ __forceinline__ void tri_proj(const int32_t* __restrict__ U, const int32_t* __restrict__ F, int32_t t,
                                         const int32_t* n, int64_t* e)
{
    for (int a = 0; a < 3; ++a) {
        e[2 * a] = INT64_MAX;
        e[2 * a + 1] = INT64_MIN;
    }
    for (int v = 0; v < 3; ++v) {
        const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
        for (int a = 0; a < 3; ++a) {
            const int64_t d = (int64_t)n[3 * a] * P[0] + (int64_t)n[3 * a + 1] * P[1] + (int64_t)n[3 * a + 2] * P[2];
            e[2 * a] = min(e[2 * a], d);
            e[2 * a + 1] = max(e[2 * a + 1], d);
        }
    }
}

__global__ void k_fl_group(const int32_t* __restrict__ assign, const int32_t* __restrict__ parent, int64_t T,
                           int32_t* __restrict__ group, int32_t* __restrict__ nassign)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    group[t] = parent[assign[t]];
    nassign[t] = -1;
}

__global__ void k_fl_box_count(const int32_t* __restrict__ parent, int32_t K, int32_t* __restrict__ gcount,
                               int32_t* err)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int32_t g = parent[k];
    if (g < 0 || g >= K) {
        atomicOr(err, kErrArg);
        return;
    }
    atomicAdd(&gcount[g], 1);
}

__global__ void k_fl_box_fill(const int32_t* __restrict__ parent, int32_t K, const int32_t* __restrict__ gstart,
                              int32_t* __restrict__ gfill, int32_t* __restrict__ gbox)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int32_t g = parent[k];
    gbox[gstart[g] + atomicAdd(&gfill[g], 1)] = k;
}

// ascending box order inside each group
__global__ void k_fl_box_sort(const int32_t* __restrict__ gstart, int32_t K, int32_t* __restrict__ gbox)
{
    int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= K) return;
    for (int32_t i = gstart[g] + 1; i < gstart[g + 1]; ++i)
        for (int32_t j = i; j > gstart[g] && gbox[j - 1] > gbox[j]; --j) {
            const int32_t x = gbox[j];
            gbox[j] = gbox[j - 1];
            gbox[j - 1] = x;
        }
}

__global__ void k_fl_keys(const float* __restrict__ V, const int32_t* __restrict__ F, int64_t T,
                          const int32_t* __restrict__ group, const int32_t* __restrict__ gstart,
                          const int32_t* __restrict__ gbox, const double* __restrict__ centre,
                          unsigned long long* __restrict__ key)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int32_t g = group[t];
    unsigned long long best = ~0ull;
    for (int32_t i = gstart[g]; i < gstart[g + 1]; ++i) {
        const unsigned long long k = tri_key(V, F, (int32_t)t, centre + 3 * (int64_t)gbox[i]);
        best = k < best ? k : best;
    }
    key[t] = best;
}

// Seeds: one block per group; its boxes in index order take the nearest
// triangle of the group not taken by an earlier box.  The group's triangles
// are the members of the clusters whose parent is the group.
__global__ void __launch_bounds__(kFT) k_fl_seed(const float* __restrict__ V, const int32_t* __restrict__ F,
                                                 const int32_t* __restrict__ gstart, const int32_t* __restrict__ gbox,
                                                 const int32_t* __restrict__ members,
                                                 const int32_t* __restrict__ mstart,
                                                 const double* __restrict__ centre, int32_t* __restrict__ nassign,
                                                 int32_t* __restrict__ seed, int32_t* err)
{
    __shared__ unsigned long long red[kFT / 32];
    __shared__ int32_t taken[kMaxFloodCand];
    const int32_t g = blockIdx.x;
    const int32_t b0 = gstart[g], b1 = gstart[g + 1];
    if (b1 - b0 > kMaxFloodCand) {
        if (threadIdx.x == 0) atomicOr(err, kErrOverflow);
        return;
    }
    for (int32_t i = b0; i < b1; ++i) {
        const int32_t k = gbox[i];
        const double* c = centre + 3 * (int64_t)k;
        unsigned long long best = ~0ull;
        for (int32_t j = b0; j < b1; ++j) {
            const int32_t cl = gbox[j];   // the group's triangles: members of its old clusters
            for (int32_t m = mstart[cl] + threadIdx.x; m < mstart[cl + 1]; m += kFT) {
                const int32_t t = members[m];
                bool used = false;
                for (int32_t q = 0; q < i - b0; ++q) used |= taken[q] == t;
                if (used) continue;
                const unsigned long long kk = tri_key(V, F, t, c);
                best = kk < best ? kk : best;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
            best = w < best ? w : best;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = red[0];
            for (int w = 1; w < kFT / 32; ++w) b = red[w] < b ? red[w] : b;
            if (b == ~0ull) {
                atomicOr(err, kErrEmpty);
                taken[i - b0] = -1;
                seed[k] = -1;
            } else {
                const int32_t t = (int32_t)(b & 0xffffffffu);
                taken[i - b0] = t;
                seed[k] = t;
                nassign[t] = k;
            }
        }
        __syncthreads();
    }
}

// every box's slab from its seed triangle
__global__ void k_fl_seed_bounds(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                                 const int32_t* __restrict__ seed, int32_t K, obb_qbox* __restrict__ q)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int32_t t = seed[k];
    if (t < 0) return;
    int64_t e[6];
    tri_proj(U, F, t, q[k].n, e);
    for (int i = 0; i < 6; ++i) q[k].b[i] = e[i];
}

__global__ void k_fl_reset(unsigned long long* __restrict__ gbest, unsigned long long* __restrict__ gfall,
                           int32_t K)
{
    int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= K) return;
    gbest[g] = ~0ull;
    gfall[g] = ~0ull;
}

__device__ __forceinline__ bool available(const int32_t* __restrict__ adj, const int32_t* __restrict__ group,
                                          const int32_t* __restrict__ nassign, int32_t t)
{
    bool a = false;
    for (int e = 0; e < 3; ++e) {
        const int32_t u = adj[3 * t + e];
        a |= nassign[u] >= 0 && group[u] == group[t];
    }
    return a;
}

// per group: smallest priority among available triangles (gbest) and among
// all unassigned ones (gfall)
__global__ void k_fl_minkeys(const int32_t* __restrict__ adj, const int32_t* __restrict__ group,
                             const int32_t* __restrict__ nassign, const unsigned long long* __restrict__ key,
                             int64_t T, unsigned long long* __restrict__ gbest, unsigned long long* __restrict__ gfall)
{
    int64_t tt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tt >= T) return;
    const int32_t t = (int32_t)tt;
    if (nassign[t] >= 0) return;
    const int32_t g = group[t];
    atomicMin(&gfall[g], key[t]);
    if (available(adj, group, nassign, t)) atomicMin(&gbest[g], key[t]);
}

__global__ void k_fl_select(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                            const int32_t* __restrict__ adj, const int32_t* __restrict__ group,
                            const int32_t* __restrict__ nassign, const unsigned long long* __restrict__ key,
                            int64_t T, const unsigned long long* __restrict__ gbest,
                            const unsigned long long* __restrict__ gfall, const int32_t* __restrict__ gstart,
                            const int32_t* __restrict__ gbox, const obb_qbox* __restrict__ q, int32_t wavefront,
                            FloodRec* __restrict__ rec, obb_qbox* __restrict__ evals, int32_t* __restrict__ ctr,
                            int32_t rec_cap, int32_t eval_cap, int32_t* err)
{
    int64_t tt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tt >= T) return;
    const int32_t t = (int32_t)tt;
    if (nassign[t] >= 0) return;
    const int32_t g = group[t];
    const bool avail = available(adj, group, nassign, t);
    bool take;
    if (gbest[g] != ~0ull) take = wavefront ? avail : key[t] == gbest[g];
    else take = key[t] == gfall[g];
    if (!take) return;
    FloodRec r;
    r.t = t;
    r.nk = 0;
    if (avail) {
        for (int e = 0; e < 3; ++e) {
            const int32_t u = adj[3 * t + e];
            const int32_t k = nassign[u];
            if (k < 0 || group[u] != g) continue;
            bool dup = false;
            for (int i = 0; i < r.nk; ++i) dup |= r.k[i] == k;
            if (!dup) r.k[r.nk++] = k;
        }
    } else {
        const int32_t nb = gstart[g + 1] - gstart[g];
        if (nb > kMaxFloodCand) {
            atomicOr(err, kErrOverflow);
            return;
        }
        for (int i = 0; i < nb; ++i) r.k[r.nk++] = gbox[gstart[g] + i];
    }
    for (int i = 0; i < r.nk; ++i) {
        const obb_qbox& qk = q[r.k[i]];
        int64_t pr[6];
        tri_proj(U, F, t, qk.n, pr);
        obb_qbox gq = qk;
        bool grew = false;
        for (int a = 0; a < 3; ++a) {
            if (pr[2 * a] < gq.b[2 * a]) {
                gq.b[2 * a] = pr[2 * a];
                grew = true;
            }
            if (pr[2 * a + 1] > gq.b[2 * a + 1]) {
                gq.b[2 * a + 1] = pr[2 * a + 1];
                grew = true;
            }
        }
        r.e[i] = -1;
        if (grew) {
            const int32_t ei = atomicAdd(&ctr[1], 1);
            if (ei >= eval_cap) {
                atomicOr(err, kErrOverflow);
                return;
            }
            evals[ei] = gq;
            r.e[i] = ei;
        }
    }
    const int32_t ri = atomicAdd(&ctr[0], 1);
    if (ri >= rec_cap) {
        atomicOr(err, kErrOverflow);
        return;
    }
    rec[ri] = r;
}

// best box per taken triangle (smallest growth, ties -> smaller box) and, in
// exact mode, the box update (one taken triangle per group, so the boxes
// touched are distinct)
__global__ void k_fl_apply(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                           const FloodRec* __restrict__ rec, const int32_t* __restrict__ ctr,
                           const obb_qbox* __restrict__ evals, const uint64_t* __restrict__ ecount,
                           int32_t wavefront, int32_t* __restrict__ nassign, obb_qbox* __restrict__ q,
                           uint64_t* __restrict__ obv, uint8_t* __restrict__ changed, int32_t* __restrict__ left)
{
    int32_t ri = blockIdx.x * blockDim.x + threadIdx.x;
    if (ri >= ctr[0]) return;
    const FloodRec& r = rec[ri];
    int bi = -1;
    int64_t bc = 0;
    int32_t bk = INT32_MAX;
    for (int i = 0; i < r.nk; ++i) {
        const int32_t k = r.k[i];
        const int64_t c = r.e[i] >= 0 ? (int64_t)ecount[r.e[i]] - (int64_t)obv[k] : 0;
        if (bi < 0 || c < bc || (c == bc && k < bk)) {
            bi = i;
            bc = c;
            bk = k;
        }
    }
    nassign[r.t] = bk;
    atomicSub(left, 1);
    if (!wavefront) {
        if (r.e[bi] >= 0) {
            for (int i = 0; i < 6; ++i) q[bk].b[i] = evals[r.e[bi]].b[i];
            obv[bk] = ecount[r.e[bi]];
        }
    } else {
        int64_t pr[6];
        tri_proj(U, F, r.t, q[bk].n, pr);
        for (int a = 0; a < 3; ++a) {
            atomicMin(reinterpret_cast<long long*>(&q[bk].b[2 * a]), (long long)pr[2 * a]);
            atomicMax(reinterpret_cast<long long*>(&q[bk].b[2 * a + 1]), (long long)pr[2 * a + 1]);
        }
        changed[bk] = 1;
    }
}

__global__ void k_fl_compact(const uint8_t* __restrict__ changed, int32_t K, const obb_qbox* __restrict__ q,
                             obb_qbox* __restrict__ evals, int32_t* __restrict__ map, int32_t* __restrict__ n)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K || !changed[k]) return;
    const int32_t i = atomicAdd(n, 1);
    evals[i] = q[k];
    map[i] = k;
}

__global__ void k_fl_recount(const int32_t* __restrict__ map, const int32_t* __restrict__ n,
                             const uint64_t* __restrict__ cnt, uint64_t* __restrict__ obv,
                             uint8_t* __restrict__ changed)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n) return;
    obv[map[i]] = cnt[i];
    changed[map[i]] = 0;
}

// world-space centres of the layer's boxes (the slab midpoints through the frame)
__global__ void k_fl_centres(const LatticeFrame* __restrict__ f, const double* __restrict__ frames,
                             const obb_qbox* __restrict__ q, int32_t K, double* __restrict__ out)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double* R = frames + 9 * (int64_t)k;
    const double s = 4294967296.0 / f->hmax;
    double c[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        double base = 0.0;
        for (int b = 0; b < 3; ++b) base = __dadd_rn(base, __dmul_rn(R[3 * a + b], __dadd_rn(f->lo[b], 0.5 * f->h[b])));
        const double mid = __dadd_rn(__ddiv_rn(0.5 * ((double)q[k].b[2 * a] + (double)q[k].b[2 * a + 1]), s), base);
        for (int b = 0; b < 3; ++b) c[b] = __dadd_rn(c[b], __dmul_rn(R[3 * a + b], mid));
    }
    for (int b = 0; b < 3; ++b) out[3 * (int64_t)k + b] = c[b];
}

struct FloodMem {
    obb_ctx* ctx = nullptr;
    std::vector<void*> ptrs;
    cudaError_t e = cudaSuccess;
    template <class T>
    T* get(size_t n)
    {
        void* p = nullptr;
        if (e == cudaSuccess) e = pool_alloc(&p, sizeof(T) * (n > 0 ? n : 1), ctx->stream);
        if (e == cudaSuccess) ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~FloodMem()
    {
        for (void* p : ptrs) cudaFreeAsync(p, ctx->stream);
    }
};

}  // namespace

obb_status flood_partition(obb_ctx* ctx, obb_layer* L, const double* d_centres, int32_t mode, obb_flood_stats* out)
{
    cudaStream_t s = ctx->stream;
    const obb_lattice* lat = L->lat;
    const obb_mesh* mesh = lat->mesh;
    const int32_t K = L->K;
    const int64_t T = L->T;
    if (mode != 0 && mode != 1) return fail(ctx, OBB_ERR_ARG, "flood mode must be 0 (exact) or 1 (wavefront)");
    OBB_TRY(layer_members(ctx, L));
    FloodMem mem;
    mem.ctx = ctx;
    // exact mode takes at most one triangle per group and wave; the wavefront
    // up to every triangle, with three candidates unless it is a group's
    // fallback (up to kMaxFloodCand, at most one per group)
    const int32_t rec_cap = mode == 0 ? K : (int32_t)T;
    const int32_t eval_cap = (mode == 0 ? 0 : 3 * (int32_t)T) + kMaxFloodCand * K;
    int32_t* group = mem.get<int32_t>(T);
    int32_t* nassign = mem.get<int32_t>(T);
    unsigned long long* key = mem.get<unsigned long long>(T);
    int32_t* gcount = mem.get<int32_t>(K);
    int32_t* gstart = mem.get<int32_t>((size_t)K + 1);
    int32_t* gfill = mem.get<int32_t>(K);
    int32_t* gbox = mem.get<int32_t>(K);
    int32_t* seed = mem.get<int32_t>(K);
    unsigned long long* gbest = mem.get<unsigned long long>(K);
    unsigned long long* gfall = mem.get<unsigned long long>(K);
    double* centre = mem.get<double>(3 * (size_t)K);
    FloodRec* rec = mem.get<FloodRec>(rec_cap);
    obb_qbox* evals = mem.get<obb_qbox>(eval_cap);
    uint64_t* ecount = mem.get<uint64_t>(eval_cap);
    uint8_t* changed = mem.get<uint8_t>(K);
    int32_t* map = mem.get<int32_t>(K);
    int32_t* ctr = mem.get<int32_t>(4);   // records, evals, unassigned, recount size
    if (mem.e != cudaSuccess) return cuda_fail(ctx, mem.e, "flood scratch");
    const unsigned gT = (unsigned)((T + 255) / 256), gK = (unsigned)((K + 127) / 128);
    if (d_centres) OBB_CK(ctx, cudaMemcpyAsync(centre, d_centres, sizeof(double) * 3 * K, cudaMemcpyDefault, s));
    else {
        k_fl_centres<<<gK, 128, 0, s>>>(lat->d_frame, L->d_frames, L->d_q, K, centre);
        note_launch(ctx);
    }
    k_fl_group<<<gT, 256, 0, s>>>(L->d_assign, L->d_parent, T, group, nassign);
    OBB_CK(ctx, cudaMemsetAsync(gcount, 0, sizeof(int32_t) * K, s));
    OBB_CK(ctx, cudaMemsetAsync(gfill, 0, sizeof(int32_t) * K, s));
    OBB_CK(ctx, cudaMemsetAsync(changed, 0, K, s));
    k_fl_box_count<<<gK, 128, 0, s>>>(L->d_parent, K, gcount, ctx->d_err);
    note_launch(ctx, 2);
    OBB_TRY(set_device_int(ctx, ctr + 3, K));
    launch_scan_i32(ctx, gcount, gstart, ctr + 3);
    k_fl_box_fill<<<gK, 128, 0, s>>>(L->d_parent, K, gstart, gfill, gbox);
    k_fl_box_sort<<<gK, 128, 0, s>>>(gstart, K, gbox);
    k_fl_keys<<<gT, 256, 0, s>>>(mesh->d_verts, mesh->d_tris, T, group, gstart, gbox, centre, key);
    note_launch(ctx, 4);
    OBB_TRY(check_device_error(ctx));
    // seeds: the groups are the parents; L->d_start / d_members list the old clusters
    k_fl_seed<<<K, kFT, 0, s>>>(mesh->d_verts, mesh->d_tris, gstart, gbox, L->d_members, L->d_start, centre, nassign,
                                 seed, ctx->d_err);
    k_fl_seed_bounds<<<gK, 128, 0, s>>>(lat->d_fixed, mesh->d_tris, seed, K, L->d_q);
    note_launch(ctx, 2);
    OBB_TRY(check_device_error(ctx));
    OBB_TRY(count_boxes(ctx, lat, L->d_q, layer_dev_K(L), K, L->d_obv, nullptr));
    int64_t* h = host_stats(ctx);
    int32_t* hi = reinterpret_cast<int32_t*>(h);
    OBB_TRY(set_device_int(ctx, ctr + 2, (int32_t)(T - K)));
    obb_flood_stats st{};
    int64_t evals_total = 0;
    for (;;) {
        OBB_CK(ctx, cudaMemcpyAsync(hi, ctr + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        OBB_TRY(check_device_error(ctx));
        if (hi[0] <= 0) break;
        k_fl_reset<<<gK, 128, 0, s>>>(gbest, gfall, K);
        k_fl_minkeys<<<gT, 256, 0, s>>>(mesh->d_adj, group, nassign, key, T, gbest, gfall);
        OBB_CK(ctx, cudaMemsetAsync(ctr, 0, sizeof(int32_t) * 2, s));
        k_fl_select<<<gT, 256, 0, s>>>(lat->d_fixed, mesh->d_tris, mesh->d_adj, group, nassign, key, T, gbest, gfall,
                                       gstart, gbox, L->d_q, mode, rec, evals, ctr, rec_cap, eval_cap, ctx->d_err);
        note_launch(ctx, 3);
        OBB_TRY(count_boxes(ctx, lat, evals, ctr + 1, eval_cap, ecount, nullptr));
        k_fl_apply<<<(unsigned)((rec_cap + 127) / 128), 128, 0, s>>>(lat->d_fixed, mesh->d_tris, rec, ctr, evals,
                                                                     ecount, mode, nassign, L->d_q, L->d_obv,
                                                                     changed, ctr + 2);
        note_launch(ctx);
        if (mode == 1) {
            OBB_CK(ctx, cudaMemsetAsync(ctr + 3, 0, sizeof(int32_t), s));
            k_fl_compact<<<gK, 128, 0, s>>>(changed, K, L->d_q, evals, map, ctr + 3);
            note_launch(ctx);
            OBB_TRY(count_boxes(ctx, lat, evals, ctr + 3, K, ecount, nullptr));
            k_fl_recount<<<gK, 128, 0, s>>>(map, ctr + 3, ecount, L->d_obv, changed);
            note_launch(ctx);
        }
        OBB_CK(ctx, cudaMemcpyAsync(hi + 1, ctr + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        OBB_CK(ctx, cudaGetLastError());
        ++st.waves;
        OBB_CK(ctx, cudaStreamSynchronize(s));
        evals_total += hi[1];
    }
    OBB_CK(ctx, cudaMemcpyAsync(L->d_assign, nassign, sizeof(int32_t) * T, cudaMemcpyDeviceToDevice, s));
    layer_members_changed(L);
    OBB_CK(ctx, cudaMemsetAsync(layer_dirty(L), 1, K, s));
    OBB_CK(ctx, cudaMemsetAsync(layer_level(L), 0, sizeof(int32_t) * K, s));
    OBB_TRY(layer_members(ctx, L));
    OBB_TRY(check_device_error(ctx));
    st.box_evals = evals_total;
    if (out) *out = st;
    return OBB_OK;
}

}  // namespace obbv
