// Mesh upload and validation on the device (the closed mesh X of Sec. 3,
// Definition 1): every coordinate finite, every index in range, no triangle
// with a repeated vertex, and every undirected edge shared by exactly two
// triangles.  The edge check sorts the 3T edge keys (min << B | max, B the
// bits of a vertex index, so the sort reads 2B key bits) with their slots and
// pairs equal neighbours; the pairing is also the triangle adjacency
// (triangle across edge (v_e, v_e+1)).
#include <cub/cub.cuh>

#include <string>

#include "internal.h"

namespace obbv {
namespace {

enum { kMeshNonFinite = 1, kMeshRange = 2, kMeshRepeated = 4, kMeshEdge = 8 };

__global__ void k_mesh_verts(const float* __restrict__ V, int64_t n, int32_t* __restrict__ flags)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !isfinite(V[i])) atomicOr(flags, kMeshNonFinite);
}

__global__ void k_mesh_edges(const int32_t* __restrict__ F, int64_t nt, int64_t nv, int B,
                             unsigned long long* __restrict__ key, int32_t* __restrict__ slot,
                             int32_t* __restrict__ flags)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * nt) return;
    const int64_t t = i / 3;
    const int e = (int)(i - 3 * t);
    const int64_t a = F[3 * t + e], b = F[3 * t + (e + 1) % 3];
    slot[i] = (int32_t)i;
    if (a < 0 || a >= nv || b < 0 || b >= nv) {
        atomicOr(flags, kMeshRange);
        key[i] = ~0ull;
        return;
    }
    if (a == b) atomicOr(flags, kMeshRepeated);
    const unsigned long long lo = (unsigned long long)min(a, b), hi = (unsigned long long)max(a, b);
    key[i] = (lo << B) | hi;
}

// sorted keys: a run must be exactly two long; its two slots are adjacent
__global__ void k_mesh_pair(const unsigned long long* __restrict__ key, const int32_t* __restrict__ slot, int64_t n,
                            int32_t* __restrict__ adj, unsigned long long* __restrict__ bad,
                            int32_t* __restrict__ flags)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = key[i];
    if (i > 0 && key[i - 1] == k) return;   // not the first of its run
    const bool two = i + 1 < n && key[i + 1] == k && (i + 2 >= n || key[i + 2] != k);
    if (!two) {
        atomicOr(flags, kMeshEdge);
        atomicMin(bad, k);
        return;
    }
    const int64_t x = slot[i], y = slot[i + 1];
    adj[x] = (int32_t)(y / 3);
    adj[y] = (int32_t)(x / 3);
}

__global__ void k_mesh_count_key(const unsigned long long* __restrict__ key, int64_t n,
                                 const unsigned long long* __restrict__ bad, int32_t* __restrict__ count)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && key[i] == *bad) atomicAdd(count, 1);
}

}  // namespace

obb_status mesh_upload(obb_ctx* ctx, const float* verts, int64_t nv, const int32_t* tris, int64_t nt, obb_mesh* m)
{
    cudaStream_t s = ctx->stream;
    const int64_t ne = 3 * nt;
    OBB_CK(ctx, pool_alloc((void**)&m->d_verts, sizeof(float) * 3 * nv, s));
    OBB_CK(ctx, pool_alloc((void**)&m->d_tris, sizeof(int32_t) * ne, s));
    OBB_CK(ctx, pool_alloc((void**)&m->d_adj, sizeof(int32_t) * ne, s));
    OBB_CK(ctx, cudaMemcpyAsync(m->d_verts, verts, sizeof(float) * 3 * nv, cudaMemcpyHostToDevice, s));
    OBB_CK(ctx, cudaMemcpyAsync(m->d_tris, tris, sizeof(int32_t) * ne, cudaMemcpyHostToDevice, s));
    // scratch: keys and slots twice (sort in / out), flags, the smallest bad key, its count
    const size_t kb = (sizeof(unsigned long long) * ne + 255) / 256 * 256;
    const size_t sb = (sizeof(int32_t) * ne + 255) / 256 * 256;
    int B = 1;   // bits of a vertex index
    while (B < 31 && (int64_t(1) << B) < nv) ++B;
    OBB_CK(ctx, ctx->tmp_a.reserve(2 * kb + 2 * sb + 256, s));
    char* base = ctx->tmp_a.as<char>();
    unsigned long long* key = reinterpret_cast<unsigned long long*>(base);
    unsigned long long* key2 = reinterpret_cast<unsigned long long*>(base + kb);
    int32_t* slot = reinterpret_cast<int32_t*>(base + 2 * kb);
    int32_t* slot2 = reinterpret_cast<int32_t*>(base + 2 * kb + sb);
    int32_t* flags = reinterpret_cast<int32_t*>(base + 2 * kb + 2 * sb);
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(base + 2 * kb + 2 * sb + 64);
    int32_t* bad_count = reinterpret_cast<int32_t*>(base + 2 * kb + 2 * sb + 128);
    OBB_CK(ctx, cudaMemsetAsync(flags, 0, sizeof(int32_t), s));
    OBB_CK(ctx, cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), s));
    OBB_CK(ctx, cudaMemsetAsync(bad_count, 0, sizeof(int32_t), s));
    k_mesh_verts<<<(unsigned)((3 * nv + 255) / 256), 256, 0, s>>>(m->d_verts, 3 * nv, flags);
    k_mesh_edges<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(m->d_tris, nt, nv, B, key, slot, flags);
    note_launch(ctx, 2);
    auto sort = [&](cudaStream_t cs) {
        size_t bytes = ctx->cub_tmp.bytes;
        return cub::DeviceRadixSort::SortPairs(ctx->cub_tmp.p, bytes, key, key2, slot, slot2, (int)ne, 0, 2 * B, cs);
    };
    size_t bytes = 0;
    OBB_CK(ctx, cub::DeviceRadixSort::SortPairs(nullptr, bytes, key, key2, slot, slot2, (int)ne, 0, 2 * B, s));
    OBB_CK(ctx, ctx->cub_tmp.reserve(bytes, s));
    OBB_CK(ctx, sort(s));
    note_launch(ctx, captured_launches(ctx, ne, 2 * B, sort));
    k_mesh_pair<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(key2, slot2, ne, m->d_adj, bad, flags);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    int32_t* h = reinterpret_cast<int32_t*>(host_stats(ctx));
    OBB_CK(ctx, cudaMemcpyAsync(h, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    OBB_CK(ctx, cudaStreamSynchronize(s));
    const int32_t f = h[0];
    if (f & kMeshNonFinite) return fail(ctx, OBB_ERR_ARG, "non-finite vertex coordinate");
    if (f & kMeshRange) return fail(ctx, OBB_ERR_ARG, "triangle index out of range");
    if (f & kMeshRepeated) return fail(ctx, OBB_ERR_NOT_WATERTIGHT, "triangle with a repeated vertex");
    if (f & kMeshEdge) {
        k_mesh_count_key<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(key2, ne, bad, bad_count);
        note_launch(ctx);
        unsigned long long hb = 0;
        OBB_CK(ctx, cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
        OBB_CK(ctx, cudaMemcpyAsync(h + 1, bad_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        OBB_CK(ctx, cudaStreamSynchronize(s));
        return fail(ctx, OBB_ERR_NOT_WATERTIGHT,
                    "edge (" + std::to_string(hb >> B) + ", " + std::to_string(hb & ((1ull << B) - 1)) + ") is shared by " +
                        std::to_string(h[1]) + " triangles (need exactly 2)");
    }
    return OBB_OK;
}

}  // namespace obbv
