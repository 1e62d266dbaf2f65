// Optimisation between levels of the tree (Sec. 4.2.2): the bottom-up merge
// step, whose division units are the boxes of the level below, and the
// reciprocating sweeps over the levels.
//
// Unit step on an upper layer `up` (K clusters) whose units are the clusters
// of the lower layer `low` (Ku units; low's parent map is the unit -> cluster
// map and is updated in place).  One partition round, all exact integers:
//   scan       block per unit: the sibling clusters of its cluster s that hold
//              a triangle edge-adjacent to one of its triangles (at most
//              kMaxUnitCand), the unit's extents along s's normals and along
//              each candidate's normals;
//   top-2      per cluster and slab side: the extreme over its units, how many
//              units attain it, and the extreme over the others;
//   evals      per unit whose cluster keeps another unit: the box of s without
//              the unit (the side it alone attains falls back to the others'
//              extreme) and, per candidate k, the box of k grown by the unit;
//              boxes that differ from the current one are counted exactly;
//   gains      gain = [OBV(s) - OBV(s - u)] - [OBV(k + u) - OBV(k)], best k per
//              unit (ties -> smaller k); key (gain << 24 | (2^24 - 1 - u)) posted
//              with atomicMax at both clusters;
//   accept     a proposal holding the maximum key at both clusters is applied.
// After the rounds the upper layer's triangle map is rebuilt from the units and
// its boxes get the same update as in the Lloyd step (covariance refit of the
// changed clusters, rotation descent).
#include <vector>

#include "internal.h"

namespace obbv {
namespace {

constexpr int kMaxUnitCand = 8;   // sibling clusters one unit may border
constexpr int kUT = 128;          // threads of the per-unit scan

enum { kUCtrCand = 0, kUCtrEval, kUCtrCount };

struct UnitCand {
    int32_t u, s, nk, e_shr;
    int32_t k[kMaxUnitCand];
    int32_t e_gro[kMaxUnitCand];
    int32_t best, pad;
    int64_t gain;
    unsigned long long key;
};

struct UnitScan {
    int64_t ext[6];                        // along the own cluster's normals
    int64_t grow[kMaxUnitCand][6];         // along each candidate's normals
    int32_t k[kMaxUnitCand];
    int32_t nk;
    int32_t pad;
};

__global__ void k_check_nesting(const int32_t* __restrict__ up_assign, const int32_t* __restrict__ low_assign,
                                const int32_t* __restrict__ low_parent, int64_t T, int32_t K, int32_t* err)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int32_t c = low_parent[low_assign[t]];
    if (c < 0 || c >= K || c != up_assign[t]) atomicOr(err, kErrArg);
}

__global__ void k_unit_init(int32_t K, int64_t* __restrict__ m1, int64_t* __restrict__ m2,
                            int32_t* __restrict__ cnt1, int32_t* __restrict__ usize)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    for (int side = 0; side < 6; ++side) {
        const int64_t sent = (side & 1) ? INT64_MIN : INT64_MAX;
        m1[6 * (int64_t)k + side] = sent;
        m2[6 * (int64_t)k + side] = sent;
        cnt1[6 * (int64_t)k + side] = 0;
    }
    usize[k] = 0;
}

__device__ __forceinline__ void proj_minmax(const int32_t* __restrict__ U, const int32_t* __restrict__ F, int32_t t,
                                            const int32_t* n, int64_t* e)
{
    for (int v = 0; v < 3; ++v) {
        const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
        const int64_t x = P[0], y = P[1], z = P[2];
        for (int a = 0; a < 3; ++a) {
            const int64_t d = (int64_t)n[3 * a] * x + (int64_t)n[3 * a + 1] * y + (int64_t)n[3 * a + 2] * z;
            e[2 * a] = min(e[2 * a], d);
            e[2 * a + 1] = max(e[2 * a + 1], d);
        }
    }
}

// block-wide min (even entries) / max (odd entries) of six int64; result in out
__device__ void block_minmax6(int64_t* e, int64_t* sh /* [kUT / 32][6] */, int64_t* out)
{
    for (int i = 0; i < 6; ++i)
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t w = __shfl_xor_sync(0xffffffffu, e[i], o);
            e[i] = (i & 1) ? max(e[i], w) : min(e[i], w);
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int i = 0; i < 6; ++i) sh[6 * warp + i] = e[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 6; ++i) {
            int64_t v = sh[i];
            for (int w = 1; w < kUT / 32; ++w) v = (i & 1) ? max(v, sh[6 * w + i]) : min(v, sh[6 * w + i]);
            out[i] = v;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kUT) k_unit_scan(const int32_t* __restrict__ U, const int32_t* __restrict__ F,
                                                   const int32_t* __restrict__ adj,
                                                   const int32_t* __restrict__ low_assign,
                                                   const int32_t* __restrict__ members,
                                                   const int32_t* __restrict__ start,
                                                   const int32_t* __restrict__ cl,
                                                   const int32_t* __restrict__ up_parent,
                                                   const obb_qbox* __restrict__ q, int32_t* __restrict__ usize,
                                                   UnitScan* __restrict__ scan, int32_t* err)
{
    __shared__ int32_t cset[kMaxUnitCand];
    __shared__ int32_t overflow;
    __shared__ int64_t sh[kUT / 32 * 6];
    __shared__ int64_t res[6];
    const int32_t u = blockIdx.x;
    const int32_t s = cl[u];
    const int32_t b0 = start[u], b1 = start[u + 1];
    if (threadIdx.x < kMaxUnitCand) cset[threadIdx.x] = -1;
    if (threadIdx.x == 0) {
        overflow = 0;
        atomicAdd(&usize[s], 1);
    }
    __syncthreads();
    const int32_t ps = up_parent[s];
    for (int32_t i = b0 + threadIdx.x; i < b1; i += kUT) {
        const int32_t t = members[i];
        for (int e = 0; e < 3; ++e) {
            const int32_t k = cl[low_assign[adj[3 * t + e]]];
            if (k == s || up_parent[k] != ps) continue;
            bool placed = false;
            for (int j = 0; j < kMaxUnitCand && !placed; ++j) {
                const int32_t old = atomicCAS(&cset[j], -1, k);
                placed = old == -1 || old == k;
            }
            if (!placed) overflow = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (overflow) atomicOr(err, kErrOverflow);
        // ascending candidate order
        int nk = 0;
        while (nk < kMaxUnitCand && cset[nk] >= 0) ++nk;
        for (int i = 1; i < nk; ++i)
            for (int j = i; j > 0 && cset[j - 1] > cset[j]; --j) {
                const int32_t tmp = cset[j];
                cset[j] = cset[j - 1];
                cset[j - 1] = tmp;
            }
        scan[u].nk = nk;
        scan[u].pad = 0;
        for (int j = 0; j < kMaxUnitCand; ++j) scan[u].k[j] = j < nk ? cset[j] : -1;
    }
    __syncthreads();
    for (int c = -1; c < kMaxUnitCand; ++c) {
        const int32_t k = c < 0 ? s : cset[c];
        if (k < 0) break;
        int64_t e[6] = {INT64_MAX, INT64_MIN, INT64_MAX, INT64_MIN, INT64_MAX, INT64_MIN};
        const int32_t* n = q[k].n;
        for (int32_t i = b0 + threadIdx.x; i < b1; i += kUT) proj_minmax(U, F, members[i], n, e);
        block_minmax6(e, sh, res);
        if (threadIdx.x == 0)
            for (int i = 0; i < 6; ++i) {
                if (c < 0) scan[u].ext[i] = res[i];
                else scan[u].grow[c][i] = res[i];
            }
    }
}

__global__ void k_unit_m1(const UnitScan* __restrict__ scan, const int32_t* __restrict__ cl, int32_t Ku,
                          int64_t* __restrict__ m1)
{
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= Ku) return;
    const int64_t* e = scan[u].ext;
    int64_t* m = m1 + 6 * (int64_t)cl[u];
    for (int side = 0; side < 6; ++side) {
        if (side & 1) atomicMax(reinterpret_cast<long long*>(m + side), (long long)e[side]);
        else atomicMin(reinterpret_cast<long long*>(m + side), (long long)e[side]);
    }
}

__global__ void k_unit_m2(const UnitScan* __restrict__ scan, const int32_t* __restrict__ cl, int32_t Ku,
                          const int64_t* __restrict__ m1, int64_t* __restrict__ m2, int32_t* __restrict__ cnt1)
{
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= Ku) return;
    const int64_t* e = scan[u].ext;
    const int64_t s6 = 6 * (int64_t)cl[u];
    for (int side = 0; side < 6; ++side) {
        if (e[side] == m1[s6 + side]) atomicAdd(&cnt1[s6 + side], 1);
        else if (side & 1) atomicMax(reinterpret_cast<long long*>(m2 + s6 + side), (long long)e[side]);
        else atomicMin(reinterpret_cast<long long*>(m2 + s6 + side), (long long)e[side]);
    }
}

__global__ void k_unit_evals(const UnitScan* __restrict__ scan, const int32_t* __restrict__ cl, int32_t Ku,
                             const int32_t* __restrict__ usize, const int64_t* __restrict__ m1,
                             const int64_t* __restrict__ m2, const int32_t* __restrict__ cnt1,
                             const obb_qbox* __restrict__ q, UnitCand* __restrict__ cand, obb_qbox* __restrict__ evals,
                             int32_t* __restrict__ ctr, int32_t cand_cap, int32_t eval_cap, int32_t* err)
{
    int32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= Ku) return;
    const int32_t s = cl[u];
    const UnitScan& sc = scan[u];
    if (usize[s] < 2 || sc.nk == 0) return;
    const int64_t s6 = 6 * (int64_t)s;
    obb_qbox shr = q[s];
    bool changed = false;
    for (int side = 0; side < 6; ++side) {
        if (m1[s6 + side] != q[s].b[side]) atomicOr(err, kErrArg);   // boxes must be tight
        if (sc.ext[side] == m1[s6 + side] && cnt1[s6 + side] == 1) {
            shr.b[side] = m2[s6 + side];
            changed = true;
        }
    }
    if (!changed) return;
    const int32_t r = atomicAdd(&ctr[kUCtrCand], 1);
    if (r >= cand_cap) {
        atomicOr(err, kErrOverflow);
        return;
    }
    UnitCand c;
    c.u = u;
    c.s = s;
    c.nk = sc.nk;
    c.best = -1;
    c.pad = 0;
    c.gain = 0;
    c.key = 0;
    c.e_shr = atomicAdd(&ctr[kUCtrEval], 1);
    if (c.e_shr >= eval_cap) {
        atomicOr(err, kErrOverflow);
        return;
    }
    evals[c.e_shr] = shr;
    for (int j = 0; j < kMaxUnitCand; ++j) {
        c.k[j] = sc.k[j];
        c.e_gro[j] = -1;
        if (j >= sc.nk) continue;
        const obb_qbox& qk = q[sc.k[j]];
        obb_qbox g = qk;
        bool grew = false;
        for (int a = 0; a < 3; ++a) {
            if (sc.grow[j][2 * a] < g.b[2 * a]) {
                g.b[2 * a] = sc.grow[j][2 * a];
                grew = true;
            }
            if (sc.grow[j][2 * a + 1] > g.b[2 * a + 1]) {
                g.b[2 * a + 1] = sc.grow[j][2 * a + 1];
                grew = true;
            }
        }
        if (grew) {
            const int32_t ei = atomicAdd(&ctr[kUCtrEval], 1);
            if (ei >= eval_cap) {
                atomicOr(err, kErrOverflow);
                return;
            }
            evals[ei] = g;
            c.e_gro[j] = ei;
        }
    }
    cand[r] = c;
}

__global__ void k_unit_gains(UnitCand* __restrict__ cand, const int32_t* __restrict__ ctr,
                             const uint64_t* __restrict__ obv, const uint64_t* __restrict__ ecount,
                             unsigned long long* __restrict__ best, int64_t* __restrict__ stats)
{
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ctr[kUCtrCand]) return;
    const UnitCand c = cand[r];
    const int64_t rem = (int64_t)obv[c.s] - (int64_t)ecount[c.e_shr];
    int bi = -1;
    int64_t bg = 0;
    for (int i = 0; i < c.nk; ++i) {   // candidates ascend, so the first of equal gains is the smallest k
        const int64_t add = c.e_gro[i] >= 0 ? (int64_t)ecount[c.e_gro[i]] - (int64_t)obv[c.k[i]] : 0;
        const int64_t g = rem - add;
        if (g > 0 && (bi < 0 || g > bg)) {
            bi = i;
            bg = g;
        }
    }
    cand[r].best = bi;
    if (bi < 0) return;
    const unsigned long long key = ((unsigned long long)bg << 24) | (unsigned long long)(0xffffff - c.u);
    cand[r].gain = bg;
    cand[r].key = key;
    atomicMax(&best[c.s], key);
    atomicMax(&best[c.k[bi]], key);
    atomicAdd((unsigned long long*)&stats[kStProposals], 1ull);
}

__global__ void k_unit_accept(const UnitCand* __restrict__ cand, const int32_t* __restrict__ ctr,
                              const unsigned long long* __restrict__ best, const obb_qbox* __restrict__ evals,
                              const uint64_t* __restrict__ ecount, int32_t* __restrict__ cl,
                              obb_qbox* __restrict__ q, uint64_t* __restrict__ obv, int64_t* __restrict__ stats,
                              uint8_t* __restrict__ dirty, int32_t* __restrict__ level)
{
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ctr[kUCtrCand]) return;
    const UnitCand c = cand[r];
    if (c.best < 0) return;
    const int32_t k = c.k[c.best];
    if (best[c.s] != c.key || best[k] != c.key) return;
    cl[c.u] = k;
    for (int i = 0; i < 6; ++i) q[c.s].b[i] = evals[c.e_shr].b[i];
    obv[c.s] = ecount[c.e_shr];
    const int32_t eg = c.e_gro[c.best];
    if (eg >= 0) {
        for (int i = 0; i < 6; ++i) q[k].b[i] = evals[eg].b[i];
        obv[k] = ecount[eg];
    }
    dirty[c.s] = 1;
    dirty[k] = 1;
    level[c.s] = 0;   // a new member set restarts the box-parameter search
    level[k] = 0;
    atomicAdd((unsigned long long*)&stats[kStAccepted], 1ull);
    atomicAdd((unsigned long long*)&stats[kStGain], (unsigned long long)c.gain);
}

__global__ void k_unit_assign(const int32_t* __restrict__ low_assign, const int32_t* __restrict__ cl, int64_t T,
                              int32_t* __restrict__ up_assign)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < T) up_assign[t] = cl[low_assign[t]];
}

// Scratch of one unit step, released when it returns.
struct UnitMem {
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
    ~UnitMem()
    {
        for (void* p : ptrs) cudaFreeAsync(p, ctx->stream);
    }
};

}  // namespace

obb_status unit_step(obb_ctx* ctx, obb_layer* up, obb_layer* low, const obb_step_opts* opts, obb_step_stats* st)
{
    cudaStream_t s = ctx->stream;
    if (!up || !low) return fail(ctx, OBB_ERR_ARG, "null layer");
    if (up->lat != low->lat) return fail(ctx, OBB_ERR_ARG, "layers of different lattices");
    const obb_lattice* lat = up->lat;
    const obb_mesh* mesh = lat->mesh;
    const int32_t K = up->K, Ku = low->K;
    const int64_t T = up->T;
    const int rounds = (opts && opts->rounds > 0) ? opts->rounds : 16;
    const int refit_mode = opts ? opts->refit : 1;
    const int dsteps = (opts && opts->descent_steps > 0) ? opts->descent_steps : 2;
    const unsigned gT = (unsigned)((T + 255) / 256), gU = (unsigned)((Ku + 127) / 128);
    k_check_nesting<<<gT, 256, 0, s>>>(up->d_assign, low->d_assign, low->d_parent, T, K, ctx->d_err);
    note_launch(ctx);
    OBB_TRY(check_device_error(ctx));
    OBB_TRY(layer_members(ctx, low));
    UnitMem mem;
    mem.ctx = ctx;
    const int32_t cand_cap = Ku + 32, eval_cap = (1 + kMaxUnitCand) * cand_cap;
    UnitScan* scan = mem.get<UnitScan>(Ku);
    int64_t* m1 = mem.get<int64_t>(6 * (size_t)K);
    int64_t* m2 = mem.get<int64_t>(6 * (size_t)K);
    int32_t* cnt1 = mem.get<int32_t>(6 * (size_t)K);
    int32_t* usize = mem.get<int32_t>(K);
    UnitCand* cand = mem.get<UnitCand>(cand_cap);
    obb_qbox* evals = mem.get<obb_qbox>(eval_cap);
    uint64_t* ecount = mem.get<uint64_t>(eval_cap);
    uint64_t* epoints = mem.get<uint64_t>(eval_cap);
    int32_t* ctr = mem.get<int32_t>(kUCtrCount);
    if (mem.e != cudaSuccess) return cuda_fail(ctx, mem.e, "unit step scratch");
    OBB_CK(ctx, cudaMemsetAsync(up->d_stats, 0, sizeof(int64_t) * kStCount, s));
    int64_t* h = host_stats(ctx);
    int ran = 0;
    int64_t before = 0;
    for (int r = 0; r < rounds; ++r) {
        k_unit_init<<<(K + 127) / 128, 128, 0, s>>>(K, m1, m2, cnt1, usize);
        k_unit_scan<<<Ku, kUT, 0, s>>>(lat->d_fixed, mesh->d_tris, mesh->d_adj, low->d_assign, low->d_members,
                                       low->d_start, low->d_parent, up->d_parent, up->d_q, usize, scan, ctx->d_err);
        k_unit_m1<<<gU, 128, 0, s>>>(scan, low->d_parent, Ku, m1);
        k_unit_m2<<<gU, 128, 0, s>>>(scan, low->d_parent, Ku, m1, m2, cnt1);
        note_launch(ctx, 4);
        OBB_CK(ctx, cudaMemsetAsync(ctr, 0, sizeof(int32_t) * kUCtrCount, s));
        OBB_CK(ctx, cudaMemsetAsync(up->d_best, 0, sizeof(unsigned long long) * K, s));
        k_unit_evals<<<gU, 128, 0, s>>>(scan, low->d_parent, Ku, usize, m1, m2, cnt1, up->d_q, cand, evals, ctr,
                                        cand_cap, eval_cap, ctx->d_err);
        note_launch(ctx);
        OBB_TRY(count_boxes(ctx, lat, evals, ctr + kUCtrEval, eval_cap, ecount, epoints));
        launch_sum_points(ctx, epoints, ctr + kUCtrEval, up->d_stats);
        const unsigned cb = (unsigned)((cand_cap + 127) / 128);
        k_unit_gains<<<cb, 128, 0, s>>>(cand, ctr, up->d_obv, ecount, up->d_best, up->d_stats);
        k_unit_accept<<<cb, 128, 0, s>>>(cand, ctr, up->d_best, evals, ecount, low->d_parent, up->d_q, up->d_obv,
                                         up->d_stats, layer_dirty(up), layer_level(up));
        note_launch(ctx, 2);
        OBB_CK(ctx, cudaGetLastError());
        OBB_CK(ctx, cudaMemcpyAsync(h, up->d_stats, sizeof(int64_t) * kStCount, cudaMemcpyDeviceToHost, s));
        OBB_TRY(check_device_error(ctx));
        ++ran;
        const int64_t moved = h[kStAccepted] - before;
        before = h[kStAccepted];
        if (moved == 0) break;
        // the lower layer's sibling structure changed with its parent map
        k_unit_assign<<<gT, 256, 0, s>>>(low->d_assign, low->d_parent, T, up->d_assign);
        note_launch(ctx);
        layer_members_changed(up);
    }
    OBB_TRY(layer_box_update(ctx, up, refit_mode, dsteps));
    return layer_finish_stats(ctx, up, ran, st);
}

// Eq. 7 of the tree from its layers' outer volumes (lattice points).
static obb_status tree_eq7(obb_ctx* ctx, const obb_tree* tree, double* out)
{
    return obb_tree_score(ctx, tree, out, nullptr);
}

obb_status tree_sweep(obb_ctx* ctx, obb_tree* tree, const obb_sweep_opts* opts, obb_sweep_stats* out)
{
    const int D = (int)tree->layers.size() - 1;
    const int sweeps = opts ? opts->sweeps : 1;
    const int iters = opts ? opts->iters : 2;
    obb_step_opts so{opts ? opts->rounds : 16, opts ? opts->refit : 1, 0, 0};
    if (sweeps < 0 || iters < 0) return fail(ctx, OBB_ERR_ARG, "sweeps and iters must be >= 0");
    obb_sweep_stats acc{};
    OBB_TRY(tree_eq7(ctx, tree, &acc.eq7_before));
    auto level = [&](int lev) -> obb_status {
        for (int it = 0; it < iters; ++it) {
            obb_step_stats st{};
            if (lev < D) {
                OBB_TRY(unit_step(ctx, tree->layers[lev], tree->layers[lev + 1], &so, &st));
                acc.unit_moves += st.moves;
            } else {
                OBB_TRY(lloyd_step(ctx, tree->layers[lev], &so, &st));
                acc.triangle_moves += st.moves;
            }
            acc.level_iters += 1;
            if (st.moves == 0 && st.refits_accepted == 0) break;
        }
        return OBB_OK;
    };
    for (int sw = 0; sw < sweeps && D >= 1; ++sw) {
        // bottom-up merging: stop at the first level whose Eq. 7 does not drop
        for (int lev = D - 1; lev >= 1; --lev) {
            double e0 = 0.0, e1 = 0.0;
            OBB_TRY(tree_eq7(ctx, tree, &e0));
            OBB_TRY(level(lev));
            OBB_TRY(tree_eq7(ctx, tree, &e1));
            if (!(e1 < e0)) break;
        }
        // top-down decomposition: units at the inner levels, triangles at the leaves
        for (int lev = 1; lev <= D; ++lev) OBB_TRY(level(lev));
    }
    OBB_TRY(tree_eq7(ctx, tree, &acc.eq7_after));
    if (out) *out = acc;
    return OBB_OK;
}

}  // namespace obbv
