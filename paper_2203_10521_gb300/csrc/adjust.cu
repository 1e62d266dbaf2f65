// Adjustment of boxes out of a local minimum (Sec. 4.2.1 step 3), on the GPU.
//
// The least important box k (fewest triangles, ties -> smaller index; only
// boxes with a sibling) hands its triangles to the sibling m sharing most
// triangle edges with it (ties -> smaller index), whose slab is recomputed.
// The sibling j with the largest outer volume (ties -> smaller index) is then
// split at the median of its triangles along its major axis, key
// n_0 . (U_p + U_q + U_r) with ties by triangle index: the first ceil(n / 2)
// stay in j, the rest form box k with j's frame.  Lloyd iterations follow,
// and the layer is restored unless its total outer volume dropped.  The
// choices are made on the device (block reductions over packed keys); the
// host only reads the few indices that size the next launches.
#include <cub/cub.cuh>

#include <vector>

#include "internal.h"

namespace obbv {
namespace {

__global__ void k_adj_gcount(const int32_t* __restrict__ parent, int32_t K, int32_t* __restrict__ gcnt, int32_t* err)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int32_t g = parent[k];
    if (g < 0 || g >= K) {
        atomicOr(err, kErrArg);
        return;
    }
    atomicAdd(&gcnt[g], 1);
}

// block-wide minimum of one 64-bit key per thread; thread 0 gets the result
__device__ unsigned long long block_min_u64(unsigned long long v)
{
    __shared__ unsigned long long sh[32];
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) v = sh[i] < v ? sh[i] : v;
    __syncthreads();
    return v;
}

// out[0] = k: the box of least (size, index) among boxes with a sibling, -1 if none
__global__ void k_adj_pick_k(const int32_t* __restrict__ size, const int32_t* __restrict__ parent,
                             const int32_t* __restrict__ gcnt, int32_t K, int32_t* __restrict__ out)
{
    unsigned long long best = ~0ull;
    for (int32_t k = threadIdx.x; k < K; k += blockDim.x)
        if (gcnt[parent[k]] >= 2) {
            const unsigned long long key = ((unsigned long long)(uint32_t)size[k] << 32) | (uint32_t)k;
            best = key < best ? key : best;
        }
    best = block_min_u64(best);
    if (threadIdx.x == 0) out[0] = best == ~0ull ? -1 : (int32_t)(best & 0xffffffffu);
}

__global__ void k_adj_edges(const int32_t* __restrict__ adj, const int32_t* __restrict__ assign,
                            const int32_t* __restrict__ parent, int64_t T, const int32_t* __restrict__ sel,
                            int32_t* __restrict__ edges)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int32_t k = sel[0];
    if (assign[t] != k) return;
    for (int e = 0; e < 3; ++e) {
        const int32_t c = assign[adj[3 * t + e]];
        if (c != k && parent[c] == parent[k]) atomicAdd(&edges[c], 1);
    }
}

// out[1] = m: the sibling of k with most shared edges, ties -> smaller index
__global__ void k_adj_pick_m(const int32_t* __restrict__ edges, const int32_t* __restrict__ parent, int32_t K,
                             int32_t* __restrict__ sel)
{
    const int32_t k = sel[0];
    unsigned long long best = ~0ull;
    for (int32_t c = threadIdx.x; c < K; c += blockDim.x)
        if (c != k && parent[c] == parent[k]) {
            // largest edges first, then smallest index: minimise the complement
            const unsigned long long key = ((unsigned long long)(0x7fffffffu - (uint32_t)edges[c]) << 32) | (uint32_t)c;
            best = key < best ? key : best;
        }
    best = block_min_u64(best);
    if (threadIdx.x == 0) sel[1] = (int32_t)(best & 0xffffffffu);
}

// out[2] = j: the sibling of k with the largest outer volume, ties -> smaller index
__global__ void k_adj_pick_j(const uint64_t* __restrict__ obv, const int32_t* __restrict__ parent, int32_t K,
                             int32_t* __restrict__ sel)
{
    const int32_t k = sel[0];
    unsigned long long best = ~0ull;
    for (int32_t c = threadIdx.x; c < K; c += blockDim.x)
        if (c != k && parent[c] == parent[k]) {
            const unsigned long long key = ((0xffffffffffull - obv[c]) << 24) | (uint32_t)c;
            best = key < best ? key : best;
        }
    best = block_min_u64(best);
    if (threadIdx.x == 0) sel[2] = (int32_t)(best & 0xffffffu);
}

__global__ void k_adj_relabel(int32_t* __restrict__ assign, int64_t T, const int32_t* __restrict__ sel, int from,
                              int to)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < T && assign[t] == sel[from]) assign[t] = sel[to];
}

// slabs of the listed boxes (sel[which[i]]) from scratch: reset, then
// atomic min / max over their triangles
__global__ void k_adj_reset(obb_qbox* __restrict__ q, const int32_t* __restrict__ sel, int32_t a, int32_t b)
{
    const int i = threadIdx.x;
    if (i >= 2) return;
    const int32_t c = sel[i == 0 ? a : b];
    for (int s = 0; s < 6; ++s) q[c].b[s] = (s & 1) ? INT64_MIN : INT64_MAX;
}

__global__ void k_adj_bounds(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                             const int32_t* __restrict__ assign, int64_t T, const int32_t* __restrict__ sel, int32_t a,
                             int32_t b, obb_qbox* __restrict__ q)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int32_t c = assign[t];
    if (c != sel[a] && c != sel[b]) return;
    const int32_t* n = q[c].n;
    for (int v = 0; v < 3; ++v) {
        const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
        for (int x = 0; x < 3; ++x) {
            const long long d = (long long)n[3 * x] * P[0] + (long long)n[3 * x + 1] * P[1] + (long long)n[3 * x + 2] * P[2];
            atomicMin(reinterpret_cast<long long*>(&q[c].b[2 * x]), d);
            atomicMax(reinterpret_cast<long long*>(&q[c].b[2 * x + 1]), d);
        }
    }
}

__global__ void k_adj_gather(const obb_qbox* __restrict__ q, const int32_t* __restrict__ sel, int32_t a, int32_t b,
                             obb_qbox* __restrict__ out)
{
    const int i = threadIdx.x;
    if (i < 2) out[i] = q[sel[i == 0 ? a : b]];
}

__global__ void k_adj_scatter(const uint64_t* __restrict__ cnt, const int32_t* __restrict__ sel, int32_t a, int32_t b,
                              uint64_t* __restrict__ obv)
{
    const int i = threadIdx.x;
    if (i < 2) obv[sel[i == 0 ? a : b]] = cnt[i];
}

__global__ void k_adj_keys(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                           const int32_t* __restrict__ assign, int64_t T, const int32_t* __restrict__ sel,
                           const obb_qbox* __restrict__ q, int32_t* __restrict__ tri, int64_t* __restrict__ key,
                           int32_t* __restrict__ n)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int32_t j = sel[2];
    if (assign[t] != j) return;
    const int32_t* nj = q[j].n;
    int64_t s[3] = {0, 0, 0};
    for (int v = 0; v < 3; ++v)
        for (int x = 0; x < 3; ++x) s[x] += U[3 * (int64_t)F[3 * t + v] + x];
    const int32_t i = atomicAdd(n, 1);
    tri[i] = (int32_t)t;
    key[i] = (int64_t)nj[0] * s[0] + (int64_t)nj[1] * s[1] + (int64_t)nj[2] * s[2];
}

__global__ void k_adj_split(const int32_t* __restrict__ order, int32_t n, const int32_t* __restrict__ sel,
                            int32_t* __restrict__ assign)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && i >= (n + 1) / 2) assign[order[i]] = sel[0];
}

__global__ void k_adj_seat(const int32_t* __restrict__ sel, double* __restrict__ frames, obb_qbox* __restrict__ q,
                           uint8_t* __restrict__ dirty, int32_t* __restrict__ level)
{
    if (threadIdx.x != 0) return;
    const int32_t k = sel[0], m = sel[1], j = sel[2];
    for (int i = 0; i < 9; ++i) {
        frames[9 * (int64_t)k + i] = frames[9 * (int64_t)j + i];
        q[k].n[i] = q[j].n[i];
    }
    dirty[k] = dirty[m] = dirty[j] = 1;
    level[k] = level[m] = level[j] = 0;
}

struct AdjMem {
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
    ~AdjMem()
    {
        for (void* p : ptrs) cudaFreeAsync(p, ctx->stream);
    }
};

}  // namespace

obb_status layer_adjust(obb_ctx* ctx, obb_layer* L, const obb_step_opts* opts, int32_t iters, obb_adjust_stats* out)
{
    cudaStream_t s = ctx->stream;
    const obb_lattice* lat = L->lat;
    const obb_mesh* mesh = lat->mesh;
    const int32_t K = L->K;
    const int64_t T = L->T;
    if (iters < 0) return fail(ctx, OBB_ERR_ARG, "iters must be >= 0");
    obb_adjust_stats st{};
    st.k = st.m = st.j = -1;
    OBB_TRY(layer_members(ctx, L));   // sizes up to date
    obb_step_stats s0{};
    OBB_TRY(layer_finish_stats(ctx, L, 0, &s0));
    st.total_before = s0.total_obv;
    st.total_after = s0.total_obv;
    AdjMem mem;
    mem.ctx = ctx;
    int32_t* gcnt = mem.get<int32_t>(K);
    int32_t* edges = mem.get<int32_t>(K);
    int32_t* sel = mem.get<int32_t>(4);
    int32_t* sv_assign = mem.get<int32_t>(T);
    double* sv_frames = mem.get<double>(9 * (size_t)K);
    obb_qbox* sv_q = mem.get<obb_qbox>(K);
    uint64_t* sv_obv = mem.get<uint64_t>(K);
    uint8_t* sv_dirty = mem.get<uint8_t>(K);
    int32_t* sv_level = mem.get<int32_t>(K);
    obb_qbox* two = mem.get<obb_qbox>(2);
    uint64_t* cnt2 = mem.get<uint64_t>(2);
    int32_t* tri = mem.get<int32_t>(T);
    int32_t* tri2 = mem.get<int32_t>(T);
    int64_t* key = mem.get<int64_t>(T);
    int64_t* key2 = mem.get<int64_t>(T);
    if (mem.e != cudaSuccess) return cuda_fail(ctx, mem.e, "adjustment scratch");
    auto save = [&](bool back) -> obb_status {
        const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
        int32_t* a0 = back ? L->d_assign : sv_assign;
        const int32_t* a1 = back ? sv_assign : L->d_assign;
        OBB_CK(ctx, cudaMemcpyAsync(a0, a1, sizeof(int32_t) * T, dd, s));
        OBB_CK(ctx, cudaMemcpyAsync(back ? L->d_frames : sv_frames, back ? sv_frames : L->d_frames,
                                    sizeof(double) * 9 * K, dd, s));
        OBB_CK(ctx, cudaMemcpyAsync(back ? L->d_q : sv_q, back ? sv_q : L->d_q, sizeof(obb_qbox) * K, dd, s));
        OBB_CK(ctx, cudaMemcpyAsync(back ? L->d_obv : sv_obv, back ? sv_obv : L->d_obv, sizeof(uint64_t) * K, dd, s));
        OBB_CK(ctx, cudaMemcpyAsync(back ? layer_dirty(L) : sv_dirty, back ? sv_dirty : layer_dirty(L), K, dd, s));
        OBB_CK(ctx, cudaMemcpyAsync(back ? layer_level(L) : sv_level, back ? sv_level : layer_level(L),
                                    sizeof(int32_t) * K, dd, s));
        if (back) layer_members_changed(L);
        return OBB_OK;
    };
    const unsigned gT = (unsigned)((T + 255) / 256), gK = (unsigned)((K + 127) / 128);
    int32_t* h = reinterpret_cast<int32_t*>(host_stats(ctx));
    // the box to re-seat and the sibling that takes its triangles
    OBB_CK(ctx, cudaMemsetAsync(gcnt, 0, sizeof(int32_t) * K, s));
    OBB_CK(ctx, cudaMemsetAsync(edges, 0, sizeof(int32_t) * K, s));
    k_adj_gcount<<<gK, 128, 0, s>>>(L->d_parent, K, gcnt, ctx->d_err);
    k_adj_pick_k<<<1, 1024, 0, s>>>(L->d_size, L->d_parent, gcnt, K, sel);
    note_launch(ctx, 2);
    OBB_CK(ctx, cudaMemcpyAsync(h, sel, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    OBB_TRY(check_device_error(ctx));
    if (h[0] < 0) {
        if (out) *out = st;
        return OBB_OK;   // no box has a sibling
    }
    OBB_TRY(save(false));
    k_adj_edges<<<gT, 256, 0, s>>>(mesh->d_adj, L->d_assign, L->d_parent, T, sel, edges);
    k_adj_pick_m<<<1, 1024, 0, s>>>(edges, L->d_parent, K, sel);
    k_adj_relabel<<<gT, 256, 0, s>>>(L->d_assign, T, sel, 0, 1);
    // m's slab over its grown member set (k's slab is not used again)
    k_adj_reset<<<1, 32, 0, s>>>(L->d_q, sel, 1, 1);
    k_adj_bounds<<<gT, 256, 0, s>>>(lat->d_fixed, mesh->d_tris, L->d_assign, T, sel, 1, 1, L->d_q);
    k_adj_gather<<<1, 32, 0, s>>>(L->d_q, sel, 1, 1, two);
    note_launch(ctx, 6);
    OBB_CK(ctx, ctx->kdev.reserve(sizeof(int32_t), s));
    int32_t* dtwo = ctx->kdev.as<int32_t>();
    OBB_TRY(set_device_int(ctx, dtwo, 2));
    OBB_TRY(count_boxes(ctx, lat, two, dtwo, 2, cnt2, nullptr));
    k_adj_scatter<<<1, 32, 0, s>>>(cnt2, sel, 1, 1, L->d_obv);
    // the box to split and its triangles in (key, index) order
    k_adj_pick_j<<<1, 1024, 0, s>>>(L->d_obv, L->d_parent, K, sel);
    OBB_CK(ctx, cudaMemsetAsync(sel + 3, 0, sizeof(int32_t), s));
    k_adj_keys<<<gT, 256, 0, s>>>(lat->d_fixed, mesh->d_tris, L->d_assign, T, sel, L->d_q, tri, key, sel + 3);
    note_launch(ctx, 3);
    OBB_CK(ctx, cudaMemcpyAsync(h, sel, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, s));
    OBB_TRY(check_device_error(ctx));
    st.k = h[0];
    st.m = h[1];
    st.j = h[2];
    const int32_t n = h[3];
    if (n < 2) {
        OBB_TRY(save(true));
        OBB_TRY(layer_members(ctx, L));
        if (out) *out = st;
        return check_device_error(ctx);
    }
    size_t b1 = 0, b2 = 0;
    OBB_CK(ctx, cub::DeviceRadixSort::SortPairs(nullptr, b1, tri, tri2, key, key2, n, 0, 32, s));
    OBB_CK(ctx, cub::DeviceRadixSort::SortPairs(nullptr, b2, key2, key, tri2, tri, n, 0, 64, s));
    OBB_CK(ctx, ctx->cub_tmp.reserve(std::max(b1, b2), s));
    b1 = ctx->cub_tmp.bytes;
    OBB_CK(ctx, cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, b1, tri, tri2, key, key2, n, 0, 32, s));   // by index
    b2 = ctx->cub_tmp.bytes;
    OBB_CK(ctx, cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, b2, key2, key, tri2, tri, n, 0, 64, s));   // then key, stable
    note_launch(ctx, 2 * 4);
    k_adj_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tri, n, sel, L->d_assign);
    k_adj_seat<<<1, 32, 0, s>>>(sel, L->d_frames, L->d_q, layer_dirty(L), layer_level(L));
    k_adj_reset<<<1, 32, 0, s>>>(L->d_q, sel, 2, 0);
    k_adj_bounds<<<gT, 256, 0, s>>>(lat->d_fixed, mesh->d_tris, L->d_assign, T, sel, 2, 0, L->d_q);
    k_adj_gather<<<1, 32, 0, s>>>(L->d_q, sel, 2, 0, two);
    note_launch(ctx, 5);
    OBB_TRY(count_boxes(ctx, lat, two, dtwo, 2, cnt2, nullptr));
    k_adj_scatter<<<1, 32, 0, s>>>(cnt2, sel, 2, 0, L->d_obv);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    layer_members_changed(L);
    obb_step_stats ls{};
    OBB_TRY(layer_finish_stats(ctx, L, 0, &ls));
    for (int it = 0; it < iters; ++it) OBB_TRY(lloyd_step(ctx, L, opts, &ls));
    if (ls.total_obv < st.total_before) {
        st.kept = 1;
        st.total_after = ls.total_obv;
    } else {
        OBB_TRY(save(true));
        OBB_TRY(layer_members(ctx, L));
    }
    if (out) *out = st;
    return check_device_error(ctx);
}

}  // namespace obbv
