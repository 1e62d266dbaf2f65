// Top-down construction of the binary OBB tree (Sec. 4.2.2) and its Eq. 7 score.
//
// Each level splits every node at the median of its triangles along the
// node's major axis and then runs Lloyd iterations restricted to siblings.
// The split is exact: key(t) = n_0 . (U_p + U_q + U_r) in int64 (three times
// the fixed-point centroid projected on the quantised major axis), ordered by
// (cluster, key, triangle) with two stable radix sorts; the first
// ceil(size / 2) triangles of a cluster go to child 2c, the rest to 2c + 1.
#include <cub/cub.cuh>

#include "internal.h"

namespace obbv {
namespace {

__global__ void k_split_keys(const int32_t* __restrict__ U, const int32_t* __restrict__ F, int64_t T,
                             const int32_t* __restrict__ assign, const obb_qbox* __restrict__ q,
                             int64_t* __restrict__ keys, int32_t* __restrict__ iota)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int32_t* n = q[assign[t]].n;
    int64_t s[3] = {0, 0, 0};
    for (int v = 0; v < 3; ++v) {
        const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
        for (int b = 0; b < 3; ++b) s[b] += P[b];
    }
    keys[t] = (int64_t)n[0] * s[0] + (int64_t)n[1] * s[1] + (int64_t)n[2] * s[2];
    iota[t] = (int32_t)t;
}

__global__ void k_gather(const int32_t* __restrict__ src, const int32_t* __restrict__ idx, int64_t n,
                         int32_t* __restrict__ dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_split_assign(const int32_t* __restrict__ order, const int32_t* __restrict__ cl,
                               const int32_t* __restrict__ start, int64_t T, int32_t* __restrict__ child,
                               int32_t* err)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    const int32_t c = cl[i];
    const int32_t size = start[c + 1] - start[c];
    if (size < 2) atomicOr(err, kErrEmpty);
    const int32_t rank = (int32_t)i - start[c];
    child[order[i]] = 2 * c + (rank < (size + 1) / 2 ? 0 : 1);
}

__global__ void k_children(int32_t K2, const double* __restrict__ frames, int32_t* __restrict__ parent,
                           double* __restrict__ fallback)
{
    int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K2) return;
    parent[c] = c >> 1;
    for (int i = 0; i < 9; ++i) fallback[9 * (int64_t)c + i] = frames[9 * (int64_t)(c >> 1) + i];
}

}  // namespace

// Median split of every cluster of `up` into children 2c and 2c + 1; writes
// d_child[T].  Uses ctx->tmp_a for the sort buffers.
obb_status split_layer(obb_ctx* ctx, const obb_layer* up, int32_t* d_child)
{
    cudaStream_t s = ctx->stream;
    const obb_lattice* lat = up->lat;
    const int64_t T = up->T;
    const int32_t K = up->K;
    OBB_CK(ctx, ctx->tmp_a.reserve(sizeof(int32_t) * T * 3 + sizeof(int64_t) * T * 2, s));
    int32_t* iota = ctx->tmp_a.as<int32_t>();
    int32_t* order1 = iota + T;
    int32_t* order2 = order1 + T;
    int64_t* keys = reinterpret_cast<int64_t*>(order2 + T);
    int64_t* keys_sorted = keys + T;
    int32_t* cl = reinterpret_cast<int32_t*>(keys_sorted);    // reused after the first sort
    int32_t* cl_sorted = cl + T;
    int end_bit = 1;
    while ((1 << end_bit) < K) ++end_bit;
    const unsigned gb = (unsigned)((T + 255) / 256);
    k_split_keys<<<gb, 256, 0, s>>>(lat->d_fixed, lat->mesh->d_tris, T, up->d_assign, up->d_q, keys, iota);
    note_launch(ctx);
    size_t b1 = 0, b2 = 0;
    OBB_CK(ctx, cub::DeviceRadixSort::SortPairs(nullptr, b1, keys, keys_sorted, iota, order1, (int)T, 0, 64, s));
    OBB_CK(ctx, cub::DeviceRadixSort::SortPairs(nullptr, b2, cl, cl_sorted, order1, order2, (int)T, 0, end_bit, s));
    OBB_CK(ctx, ctx->cub_tmp.reserve(b1 > b2 ? b1 : b2, s));
    auto sort1 = [&](cudaStream_t cs) {
        size_t bb = ctx->cub_tmp.bytes;
        return cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, bb, keys, keys_sorted, iota, order1, (int)T, 0, 64, cs);
    };
    OBB_CK(ctx, sort1(s));
    note_launch(ctx, captured_launches(ctx, T, 1000 + 64, sort1));
    k_gather<<<gb, 256, 0, s>>>(up->d_assign, order1, T, cl);
    note_launch(ctx);
    auto sort2 = [&](cudaStream_t cs) {
        size_t bb = ctx->cub_tmp.bytes;
        return cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, bb, cl, cl_sorted, order1, order2, (int)T, 0, end_bit,
                                               cs);
    };
    OBB_CK(ctx, sort2(s));
    note_launch(ctx, captured_launches(ctx, T, end_bit, sort2));
    k_split_assign<<<gb, 256, 0, s>>>(order2, cl_sorted, up->d_start, T, d_child, ctx->d_err);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return check_device_error(ctx);
}

obb_status build_tree(obb_ctx* ctx, const obb_lattice* lat, const obb_tree_opts* opts, obb_tree* tree)
{
    cudaStream_t s = ctx->stream;
    const int64_t T = lat->mesh->nt;
    const int depth = opts->depth;
    if (depth < 0 || depth > 20) return fail(ctx, OBB_ERR_ARG, "depth must be in [0, 20]");
    if ((int64_t(1) << depth) > T) return fail(ctx, OBB_ERR_EMPTY_CLUSTER, "fewer triangles than leaves");
    tree->ctx = ctx;
    tree->lat = lat;
    const int64_t Kmax = int64_t(1) << depth;
    OBB_CK(ctx, ctx->tmp_c.reserve(sizeof(int32_t) * T, s));
    OBB_CK(ctx, ctx->tmp_b.reserve(sizeof(int32_t) * Kmax + 64 + 9 * sizeof(double) * Kmax, s));
    int32_t* child = ctx->tmp_c.as<int32_t>();
    int32_t* parent = ctx->tmp_b.as<int32_t>();
    double* fallback = reinterpret_cast<double*>(ctx->tmp_b.as<char>() + ((sizeof(int32_t) * Kmax + 63) / 64) * 64);

    // root: every triangle in cluster 0, frame from the covariance
    OBB_CK(ctx, cudaMemsetAsync(child, 0, sizeof(int32_t) * T, s));
    OBB_CK(ctx, cudaMemsetAsync(parent, 0, sizeof(int32_t), s));
    obb_layer* root = nullptr;
    OBB_TRY(layer_create(ctx, lat, child, parent, 1, nullptr, nullptr, &root));
    tree->layers.push_back(root);
    obb_step_opts so{opts->rounds, opts->refit, 0, 0};
    for (int lev = 1; lev <= depth; ++lev) {
        obb_layer* up = tree->layers.back();
        OBB_TRY(split_layer(ctx, up, child));
        const int32_t K2 = 2 * up->K;
        k_children<<<(K2 + 127) / 128, 128, 0, s>>>(K2, up->d_frames, parent, fallback);
        note_launch(ctx);
        OBB_CK(ctx, cudaGetLastError());
        obb_layer* L = nullptr;
        OBB_TRY(layer_create(ctx, lat, child, parent, K2, nullptr, fallback, &L));
        tree->layers.push_back(L);
        for (int it = 0; it < opts->iters; ++it) {
            obb_step_stats st{};
            OBB_TRY(lloyd_step(ctx, L, &so, &st));
            if (st.moves == 0 && st.refits_accepted == 0) break;
        }
    }
    return OBB_OK;
}

}  // namespace obbv
