// Host runtime and the C ABI of include/obbvar.h: contexts, mesh validation
// and adjacency, handle lifetimes, host<->device marshalling, error mapping.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <unordered_set>

#include "internal.h"

namespace obbv {

namespace {
std::mutex g_pool_mu;
std::vector<cudaMemPool_t> g_pools;   // per device, created once, kept for the process
}  // namespace

cudaError_t pool_init(int device)
{
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if ((int)g_pools.size() <= device) g_pools.resize(device + 1, nullptr);
    if (g_pools[device]) return cudaSuccess;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;   // never hand freed memory back on synchronisation
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
    }
    g_pools[device] = pool;
    return cudaSuccess;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (dev < (int)g_pools.size()) pool = g_pools[dev];
    }
    if (!pool) return cudaMallocAsync(p, bytes, s);   // a device no context was created on
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t DevBuf::reserve(size_t n, cudaStream_t s)
{
    if (n <= bytes && p) return cudaSuccess;
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
    size_t want = n < 256 ? 256 : n + n / 4;
    cudaError_t e = pool_alloc(&p, want, s);
    if (e == cudaSuccess) bytes = want;
    return e;
}

void DevBuf::release(cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
}

obb_status fail(obb_ctx* ctx, obb_status code, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

obb_status cuda_fail(obb_ctx* ctx, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, OBB_ERR_OOM, m);
    return fail(ctx, OBB_ERR_CUDA, m);
}

obb_status check_device_error(obb_ctx* ctx)
{
    OBB_CK(ctx, cudaMemcpyAsync(ctx->h_small, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    OBB_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const int32_t w = ctx->h_small[0];
    if (w == 0) return OBB_OK;
    OBB_CK(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), ctx->stream));
    if (w & kErrArg) return fail(ctx, OBB_ERR_ARG, "invalid box or assignment (non-finite, negative extent, singular or out of range)");
    if (w & kErrEmpty) return fail(ctx, OBB_ERR_EMPTY_CLUSTER, "a cluster is empty or too small to split");
    if (w & kErrTimeout) return fail(ctx, OBB_ERR_TIMEOUT, "a tensor-core wait timed out inside a kernel");
    if (w & kErrDegenerate) return fail(ctx, OBB_ERR_RANGE, "degenerate lattice: the vertex AABB has zero extent on an axis");
    if (w & kErrRange) return fail(ctx, OBB_ERR_RANGE, "a box's lattice bounding box exceeds the supported range");
    return fail(ctx, OBB_ERR_STATE, "internal capacity exceeded");
}

obb_status lattice_frame_host(const obb_lattice* lat)
{
    if (!lat->frame_stale) return OBB_OK;
    obb_ctx* ctx = lat->ctx;
    OBB_CK(ctx, cudaMemcpyAsync(&lat->frame, lat->d_frame, sizeof(LatticeFrame), cudaMemcpyDeviceToHost, ctx->stream));
    OBB_CK(ctx, cudaStreamSynchronize(ctx->stream));
    lat->frame_stale = false;
    return OBB_OK;
}

int captured_launches(obb_ctx* ctx, int64_t key0, int key1, const std::function<cudaError_t(cudaStream_t)>& fn)
{
    auto key = std::make_pair(key0, key1);
    auto it = ctx->sort_launch_cache.find(key);
    if (it != ctx->sort_launch_cache.end()) return it->second;
    int n = 0;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return 0;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cudaError_t e = fn(cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess && e2 == cudaSuccess && g) {
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(g, nodes.data(), &nn);
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++n;
            }
        }
        if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    cudaStreamDestroy(cs);
    ctx->sort_launch_cache[key] = n;
    return n;
}

const obb_ctx* mlp_owner(const obb_mlp* m);   // surrogate.cu, where the network type is complete

}  // namespace obbv

using namespace obbv;

namespace {

struct HostTmp {
    obb_ctx* ctx;
    void* p = nullptr;
    explicit HostTmp(obb_ctx* c) : ctx(c) {}
    ~HostTmp()
    {
        if (p) cudaFreeAsync(p, ctx->stream);
    }
};

// Device copy of a caller array (or the caller's device pointer itself).
template <class T>
obb_status to_device(obb_ctx* ctx, const T* src, size_t n, int on_device, HostTmp& hold, const T** out)
{
    if (on_device || n == 0) {
        *out = src;
        return OBB_OK;
    }
    OBB_CK(ctx, pool_alloc(&hold.p, sizeof(T) * n, ctx->stream));
    OBB_CK(ctx, cudaMemcpyAsync(hold.p, src, sizeof(T) * n, cudaMemcpyHostToDevice, ctx->stream));
    *out = static_cast<const T*>(hold.p);
    return OBB_OK;
}

// Output buffer: the caller's device array, or a temporary copied back after.
template <class T>
obb_status out_device(obb_ctx* ctx, T* dst, size_t n, int on_device, HostTmp& hold, T** out)
{
    if (!dst) {
        *out = nullptr;
        return OBB_OK;
    }
    if (on_device) {
        *out = dst;
        return OBB_OK;
    }
    OBB_CK(ctx, pool_alloc(&hold.p, sizeof(T) * (n > 0 ? n : 1), ctx->stream));
    *out = static_cast<T*>(hold.p);
    return OBB_OK;
}

template <class T>
obb_status copy_back(obb_ctx* ctx, T* host, const T* dev, size_t n, int on_device)
{
    if (!host || on_device || n == 0) return OBB_OK;
    OBB_CK(ctx, cudaMemcpyAsync(host, dev, sizeof(T) * n, cudaMemcpyDeviceToHost, ctx->stream));
    return OBB_OK;
}

}  // namespace

extern "C" {

obb_status obb_create(obb_ctx** out, int32_t device, void* stream)
{
    if (!out) return OBB_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return OBB_ERR_CUDA;
    if (device < 0 || device >= n) return OBB_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return OBB_ERR_CUDA;
    if (pool_init(device) != cudaSuccess) return OBB_ERR_CUDA;
    obb_ctx* c = new (std::nothrow) obb_ctx();
    if (!c) return OBB_ERR_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->d_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&c->d_ticket, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc((void**)&c->d_prof, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&c->d_order_hist, kOrderBuckets * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(c->d_order_hist, 0, kOrderBuckets * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(c->d_prof, 0, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&c->h_small, 64 * sizeof(int64_t)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(c->d_ticket, 0, sizeof(unsigned int)) != cudaSuccess) {
        obb_destroy(c);
        return OBB_ERR_CUDA;
    }
    *out = c;
    return OBB_OK;
}

obb_status obb_set_stream(obb_ctx* ctx, void* stream)
{
    if (!ctx) return OBB_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return OBB_OK;
}

obb_status obb_synchronize(obb_ctx* ctx)
{
    if (!ctx) return OBB_ERR_ARG;
    return check_device_error(ctx);
}

void obb_destroy(obb_ctx* ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    DevBuf* bufs[] = {&ctx->prep, &ctx->chunk_off, &ctx->qscratch, &ctx->cscratch, &ctx->pscratch, &ctx->kdev,
                      &ctx->tmp_a, &ctx->tmp_b, &ctx->tmp_c, &ctx->tmp_d, &ctx->cub_tmp, &ctx->order};
    for (DevBuf* b : bufs) b->release(ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (auto& ev : ctx->prof_ev) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    if (ctx->d_prof) cudaFree(ctx->d_prof);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_ticket) cudaFree(ctx->d_ticket);
    if (ctx->d_order_hist) cudaFree(ctx->d_order_hist);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    delete ctx;
}

const char* obb_last_error(const obb_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

obb_status obb_mesh_create(obb_ctx* ctx, const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
                           obb_mesh** out)
{
    if (!ctx || !out || !verts || !tris) return fail(ctx, OBB_ERR_ARG, "null argument");
    *out = nullptr;
    if (n_verts < 3 || n_tris < 4) return fail(ctx, OBB_ERR_ARG, "a closed mesh needs >= 3 vertices and >= 4 triangles");
    if (n_tris >= (int64_t(1) << 29) || n_verts >= (int64_t(1) << 31))
        return fail(ctx, OBB_ERR_RANGE, "mesh too large");
    obb_mesh* m = new (std::nothrow) obb_mesh();
    if (!m) return fail(ctx, OBB_ERR_OOM, "host allocation");
    m->ctx = ctx;
    m->nv = n_verts;
    m->nt = n_tris;
    // upload, then validate and build the adjacency on the device
    const obb_status st = mesh_upload(ctx, verts, n_verts, tris, n_tris, m);
    if (st != OBB_OK) {
        obb_mesh_free(m);
        return st;
    }
    *out = m;
    return OBB_OK;
}

void obb_mesh_free(obb_mesh* m)
{
    if (!m) return;
    cudaStream_t s = m->ctx ? m->ctx->stream : nullptr;
    if (m->d_verts) cudaFreeAsync(m->d_verts, s);
    if (m->d_tris) cudaFreeAsync(m->d_tris, s);
    if (m->d_adj) cudaFreeAsync(m->d_adj, s);
    delete m;
}

obb_status obb_build_occupancy(obb_ctx* ctx, const obb_mesh* mesh, int32_t N, obb_lattice** out)
{
    if (!ctx || !mesh || !out) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (mesh->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "mesh belongs to another context");
    *out = nullptr;
    obb_lattice* lat = new (std::nothrow) obb_lattice();
    if (!lat) return fail(ctx, OBB_ERR_OOM, "host allocation");
    obb_status st = build_occupancy(ctx, mesh, N, lat);
    if (st != OBB_OK) {
        obb_lattice_free(lat);
        return st;
    }
    *out = lat;
    return OBB_OK;
}

obb_status obb_occupancy_rebuild(obb_ctx* ctx, obb_lattice* lat)
{
    if (!ctx || !lat) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    return rebuild_occupancy(ctx, lat);
}

obb_status obb_profile_enable(obb_ctx* ctx, int32_t on)
{
    if (!ctx) return OBB_ERR_ARG;
    OBB_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& ev : ctx->prof_ev) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    ctx->prof_ev.clear();
    if (on < 0 || on > 2) return fail(ctx, OBB_ERR_ARG, "profiling mode must be 0, 1 or 2");
    OBB_CK(ctx, cudaMemset(ctx->d_prof, 0, 8 * sizeof(unsigned long long)));
    ctx->prof = on;
    return OBB_OK;
}

obb_status obb_profile_read(obb_ctx* ctx, obb_profile_stats* out)
{
    if (!ctx || !out) return OBB_ERR_ARG;
    OBB_CK(ctx, cudaStreamSynchronize(ctx->stream));
    out->launches = ctx->launches;
    out->count_launches = (int64_t)ctx->prof_ev.size();
    double ms = 0.0;
    for (auto& ev : ctx->prof_ev) {
        float t = 0.f;
        OBB_CK(ctx, cudaEventElapsedTime(&t, ev.first, ev.second));
        ms += t;
    }
    out->count_ms = ms;
    unsigned long long acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (ctx->d_prof) OBB_CK(ctx, cudaMemcpy(acc, ctx->d_prof, sizeof(acc), cudaMemcpyDeviceToHost));
    out->count_bytes = (double)acc[0];
    out->count_rows = (double)acc[1];
    out->count_points_in_domain = (double)acc[2];
    out->count_rows_rank = (double)acc[3];
    return OBB_OK;
}

obb_status obb_lattice_desc(const obb_lattice* lat, double lo[3], double h[3], int32_t* N, int64_t* row_words,
                            const uint64_t** d_words, const int32_t** d_fixed)
{
    if (!lat) return OBB_ERR_ARG;
    if (lo || h) OBB_TRY(obbv::lattice_frame_host(lat));
    for (int b = 0; b < 3; ++b) {
        if (lo) lo[b] = lat->frame.lo[b];
        if (h) h[b] = lat->frame.h[b];
    }
    if (N) *N = lat->frame.N;
    if (row_words) *row_words = lat->frame.W;
    if (d_words) *d_words = lat->d_words;
    if (d_fixed) *d_fixed = lat->d_fixed;
    return OBB_OK;
}

void obb_lattice_free(obb_lattice* lat)
{
    if (!lat) return;
    cudaStream_t s = lat->ctx ? lat->ctx->stream : nullptr;
    if (lat->d_frame) cudaFreeAsync(lat->d_frame, s);
    if (lat->d_fixed) cudaFreeAsync(lat->d_fixed, s);
    if (lat->d_words) cudaFreeAsync(lat->d_words, s);
    if (lat->d_cwords) cudaFreeAsync(lat->d_cwords, s);
    if (lat->d_words_y) cudaFreeAsync(lat->d_words_y, s);
    if (lat->d_words_z) cudaFreeAsync(lat->d_words_z, s);
    if (lat->d_rank) cudaFreeAsync(lat->d_rank, s);
    if (lat->d_rank_y) cudaFreeAsync(lat->d_rank_y, s);
    if (lat->d_rank_z) cudaFreeAsync(lat->d_rank_z, s);
    if (lat->d_ref) cudaFreeAsync(lat->d_ref, s);
    delete lat;
}

obb_status obb_quantize_boxes(obb_ctx* ctx, const obb_lattice* lat, const obb_box* boxes, int64_t K, obb_qbox* out,
                              int32_t on_device)
{
    if (!ctx || !lat || (K > 0 && (!boxes || !out))) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    if (K < 0) return fail(ctx, OBB_ERR_ARG, "negative K");
    if (K == 0) return OBB_OK;
    HostTmp hb(ctx), hq(ctx);
    const obb_box* db;
    obb_qbox* dq;
    OBB_TRY(to_device(ctx, boxes, (size_t)K, on_device, hb, &db));
    OBB_TRY(out_device(ctx, out, (size_t)K, on_device, hq, &dq));
    OBB_TRY(quantize_boxes(ctx, lat, db, K, dq));
    OBB_TRY(copy_back(ctx, out, dq, (size_t)K, on_device));
    if (!on_device) return check_device_error(ctx);
    return OBB_OK;
}

static obb_status outer_volume_impl(obb_ctx* ctx, const obb_lattice* lat, const obb_box* boxes,
                                    const obb_qbox* qboxes, int64_t K, uint64_t* counts, uint64_t* points,
                                    int32_t on_device)
{
    if (!ctx || !lat || (K > 0 && (!counts || !(boxes || qboxes)))) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    if (K < 0 || K > (int64_t(1) << 30)) return fail(ctx, OBB_ERR_ARG, "K out of range");
    if (K == 0) return OBB_OK;
    HostTmp hb(ctx), hc(ctx), hp(ctx);
    const obb_qbox* dq = nullptr;
    if (boxes) {
        const obb_box* db;
        OBB_TRY(to_device(ctx, boxes, (size_t)K, on_device, hb, &db));
        OBB_CK(ctx, ctx->qscratch.reserve(sizeof(obb_qbox) * K, ctx->stream));
        OBB_TRY(quantize_boxes(ctx, lat, db, K, ctx->qscratch.as<obb_qbox>()));
        dq = ctx->qscratch.as<obb_qbox>();
    } else {
        OBB_TRY(to_device(ctx, qboxes, (size_t)K, on_device, hb, &dq));
    }
    uint64_t *dc, *dp;
    OBB_TRY(out_device(ctx, counts, (size_t)K, on_device, hc, &dc));
    OBB_TRY(out_device(ctx, points, (size_t)K, on_device, hp, &dp));
    OBB_CK(ctx, ctx->kdev.reserve(sizeof(int32_t), ctx->stream));
    OBB_TRY(set_device_int(ctx, ctx->kdev.as<int32_t>(), (int32_t)K));
    OBB_TRY(count_boxes(ctx, lat, dq, ctx->kdev.as<int32_t>(), K, dc, dp));
    OBB_TRY(copy_back(ctx, counts, dc, (size_t)K, on_device));
    OBB_TRY(copy_back(ctx, points, dp, (size_t)K, on_device));
    if (!on_device) return check_device_error(ctx);
    return OBB_OK;
}

obb_status obb_outer_volume_q(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* boxes, int64_t K,
                              uint64_t* counts, uint64_t* points, int32_t on_device)
{
    return outer_volume_impl(ctx, lat, nullptr, boxes, K, counts, points, on_device);
}

obb_status obb_test_inject(obb_ctx* ctx, int32_t flags)
{
    if (!ctx) return OBB_ERR_ARG;
    if (flags & ~OBB_INJECT_TC_STALL) return fail(ctx, OBB_ERR_ARG, "unknown injection flag");
    ctx->inject = flags;
    return OBB_OK;
}

obb_status obb_set_counting_axis(obb_ctx* ctx, int32_t axis)
{
    if (!ctx) return OBB_ERR_ARG;
    if (axis < -1 || axis > 2) return fail(ctx, OBB_ERR_ARG, "axis must be -1 (per box), 0, 1 or 2");
    if (axis != ctx->count_axis) ++ctx->tile_gen;
    ctx->count_axis = axis;
    return OBB_OK;
}

obb_status obb_set_counting_order(obb_ctx* ctx, int32_t on)
{
    if (!ctx) return OBB_ERR_ARG;
    if (on != 0 && on != 1) return fail(ctx, OBB_ERR_ARG, "order mode must be 0 or 1");
    ctx->count_order = on;
    return OBB_OK;
}

obb_status obb_set_counting_rank(obb_ctx* ctx, int32_t on)
{
    if (!ctx) return OBB_ERR_ARG;
    if (on != 0 && on != 1) return fail(ctx, OBB_ERR_ARG, "rank mode must be 0 or 1");
    if (on != ctx->count_rank) ++ctx->tile_gen;
    ctx->count_rank = on;
    return OBB_OK;
}

obb_status obb_set_counting_tile(obb_ctx* ctx, int32_t tile_k)
{
    if (!ctx) return OBB_ERR_ARG;
    if (tile_k < 1 || tile_k > 128) return fail(ctx, OBB_ERR_ARG, "tile_k must be in [1, 128]");
    if (tile_k != ctx->tile_k) ++ctx->tile_gen;
    ctx->tile_k = tile_k;
    return OBB_OK;
}

obb_status obb_tune_counting(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* qboxes, int64_t K,
                             int32_t on_device, int32_t* tile_k, float* ms)
{
    if (!ctx || !lat || !qboxes || K <= 0) return fail(ctx, OBB_ERR_ARG, "null argument or empty batch");
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    if (K > (int64_t(1) << 30)) return fail(ctx, OBB_ERR_ARG, "K out of range");
    cudaStream_t s = ctx->stream;
    HostTmp hb(ctx);
    const obb_qbox* db;
    OBB_TRY(to_device(ctx, qboxes, (size_t)K, on_device, hb, &db));
    OBB_CK(ctx, ctx->cscratch.reserve(sizeof(uint64_t) * K, s));
    OBB_CK(ctx, ctx->kdev.reserve(sizeof(int32_t), s));
    int32_t* dK = ctx->kdev.as<int32_t>();
    OBB_TRY(set_device_int(ctx, dK, (int32_t)K));
    const int32_t cand[4] = {8, 16, 32, 64};
    float t[4] = {0, 0, 0, 0};
    cudaEvent_t e0, e1;
    OBB_CK(ctx, cudaEventCreate(&e0));
    OBB_CK(ctx, cudaEventCreate(&e1));
    const int32_t prof = ctx->prof;
    ctx->prof = 0;
    obb_status rc = OBB_OK;
    for (int i = 0; i < 4 && rc == OBB_OK; ++i) {
        ctx->tile_k = cand[i];
        rc = count_boxes(ctx, lat, db, dK, K, ctx->cscratch.as<uint64_t>(), nullptr);   // warm-up
        if (rc != OBB_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && rc == OBB_OK; ++r)
            rc = count_boxes(ctx, lat, db, dK, K, ctx->cscratch.as<uint64_t>(), nullptr);
        cudaEventRecord(e1, s);
        const cudaError_t ee = cudaEventSynchronize(e1);
        if (ee != cudaSuccess) rc = cuda_fail(ctx, ee, "autotune timing");
        else cudaEventElapsedTime(&t[i], e0, e1);
        t[i] /= 3.0f;
    }
    ctx->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != OBB_OK) return rc;
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (t[i] < t[best]) best = i;
    ctx->tile_k = cand[best];
    ++ctx->tile_gen;
    if (tile_k) *tile_k = cand[best];
    if (ms)
        for (int i = 0; i < 4; ++i) ms[i] = t[i];
    return check_device_error(ctx);
}

obb_status obb_directional_outer_volume(obb_ctx* ctx, const obb_mesh* mesh, const obb_box* boxes, int64_t K,
                                        int32_t m, double* out, int32_t on_device)
{
    if (!ctx || !mesh || (K > 0 && (!boxes || !out))) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (mesh->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "mesh belongs to another context");
    if (m < 1 || m > 256) return fail(ctx, OBB_ERR_ARG, "m must be in [1, 256]");
    if (K < 0 || K > (int64_t(1) << 24)) return fail(ctx, OBB_ERR_ARG, "K out of range");
    if (K == 0) return OBB_OK;
    HostTmp hb(ctx), ho(ctx);
    const obb_box* db;
    double* dout;
    OBB_TRY(to_device(ctx, boxes, (size_t)K, on_device, hb, &db));
    OBB_TRY(out_device(ctx, out, (size_t)K, on_device, ho, &dout));
    OBB_TRY(directional_outer_volume(ctx, mesh, db, K, m, dout));
    OBB_TRY(copy_back(ctx, out, dout, (size_t)K, on_device));
    return on_device ? OBB_OK : check_device_error(ctx);
}

obb_status obb_outer_volume_multi(obb_ctx* ctx, const obb_lattice* const* lats, int32_t n_lats, const obb_qbox* boxes,
                                  const int32_t* lattice_of_box, int64_t K, uint64_t* counts, uint64_t* points,
                                  int32_t on_device)
{
    if (!ctx || !lats || n_lats < 1 || (K > 0 && (!boxes || !lattice_of_box || !counts)))
        return fail(ctx, OBB_ERR_ARG, "null argument");
    if (K < 0 || K > (int64_t(1) << 30)) return fail(ctx, OBB_ERR_ARG, "K out of range");
    if (K == 0) return OBB_OK;
    std::vector<LatRef> table(n_lats);
    int64_t lattice_bytes = 0;
    for (int32_t i = 0; i < n_lats; ++i) {
        if (!lats[i]) return fail(ctx, OBB_ERR_ARG, "null lattice in the table");
        if (lats[i]->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
        table[i] = lats[i]->ref;
        lattice_bytes += (int64_t)lats[i]->n_words * 8;
    }
    HostTmp ht(ctx), hb(ctx), hl(ctx), hc(ctx), hp(ctx);
    const LatRef* dt;
    const obb_qbox* db;
    const int32_t* dl;
    OBB_TRY(to_device(ctx, table.data(), table.size(), 0, ht, &dt));
    OBB_TRY(to_device(ctx, boxes, (size_t)K, on_device, hb, &db));
    OBB_TRY(to_device(ctx, lattice_of_box, (size_t)K, on_device, hl, &dl));
    uint64_t *dc, *dp;
    OBB_TRY(out_device(ctx, counts, (size_t)K, on_device, hc, &dc));
    OBB_TRY(out_device(ctx, points, (size_t)K, on_device, hp, &dp));
    OBB_CK(ctx, ctx->kdev.reserve(sizeof(int32_t), ctx->stream));
    OBB_TRY(set_device_int(ctx, ctx->kdev.as<int32_t>(), (int32_t)K));
    OBB_TRY(count_boxes_multi(ctx, dt, n_lats, dl, db, ctx->kdev.as<int32_t>(), K, dc, dp, lattice_bytes));
    OBB_TRY(copy_back(ctx, counts, dc, (size_t)K, on_device));
    OBB_TRY(copy_back(ctx, points, dp, (size_t)K, on_device));
    // the lattice table lives in a temporary: wait before it is released
    return check_device_error(ctx);
}

obb_status obb_outer_volume(obb_ctx* ctx, const obb_lattice* lat, const obb_box* boxes, int64_t K, uint64_t* counts,
                            uint64_t* points, int32_t on_device)
{
    if (!boxes && K > 0) return fail(ctx, OBB_ERR_ARG, "null boxes");
    return outer_volume_impl(ctx, lat, boxes, nullptr, K, counts, points, on_device);
}

obb_status obb_layer_init(obb_ctx* ctx, const obb_lattice* lat, const int32_t* assign, const int32_t* parent,
                          int32_t K, const double* frames, int32_t on_device, obb_layer** out)
{
    if (!ctx || !lat || !assign || !parent || !out) return fail(ctx, OBB_ERR_ARG, "null argument");
    *out = nullptr;
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    if (K < 1) return fail(ctx, OBB_ERR_ARG, "K must be >= 1");
    const int64_t T = lat->mesh->nt;
    HostTmp ha(ctx), hp(ctx), hf(ctx);
    const int32_t *da, *dp;
    const double* df = nullptr;
    OBB_TRY(to_device(ctx, assign, (size_t)T, on_device, ha, &da));
    OBB_TRY(to_device(ctx, parent, (size_t)K, on_device, hp, &dp));
    if (frames) OBB_TRY(to_device(ctx, frames, (size_t)9 * K, on_device, hf, &df));
    if (!on_device) {
        // parents must name clusters of the layer above; only their equality matters here
        for (int32_t k = 0; k < K; ++k)
            if (parent[k] < 0) return fail(ctx, OBB_ERR_ARG, "negative parent id");
    }
    return layer_create(ctx, lat, da, dp, K, df, nullptr, out);
}

obb_status obb_lloyd_step(obb_ctx* ctx, obb_layer* layer, const obb_step_opts* opts, obb_step_stats* stats)
{
    if (!ctx || !layer) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (layer->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    return lloyd_step(ctx, layer, opts, stats);
}

obb_status obb_layer_parents(obb_ctx* ctx, const obb_layer* L, int32_t* parent)
{
    if (!ctx || !L || !parent) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (L->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    OBB_CK(ctx, cudaMemcpyAsync(parent, L->d_parent, sizeof(int32_t) * L->K, cudaMemcpyDeviceToHost, ctx->stream));
    return check_device_error(ctx);
}

obb_status obb_flood_partition(obb_ctx* ctx, obb_layer* layer, const double* centres, int32_t mode,
                               obb_flood_stats* stats)
{
    if (!ctx || !layer) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (layer->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    return flood_partition(ctx, layer, centres, mode, stats);
}

obb_status obb_layer_adjust(obb_ctx* ctx, obb_layer* layer, const obb_step_opts* opts, int32_t iters,
                            obb_adjust_stats* stats)
{
    if (!ctx || !layer) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (layer->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    return layer_adjust(ctx, layer, opts, iters, stats);
}

obb_status obb_unit_step(obb_ctx* ctx, obb_layer* upper, obb_layer* lower, const obb_step_opts* opts,
                         obb_step_stats* stats)
{
    if (!ctx || !upper || !lower) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (upper->ctx != ctx || lower->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    if (upper == lower) return fail(ctx, OBB_ERR_ARG, "upper and lower are the same layer");
    return unit_step(ctx, upper, lower, opts, stats);
}

obb_status obb_layer_read(obb_ctx* ctx, const obb_layer* L, int32_t* assign, double* frames, obb_qbox* qboxes,
                          obb_box* boxes, uint64_t* obv, int32_t on_device)
{
    if (!ctx || !L) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (L->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    cudaStream_t s = ctx->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (assign) OBB_CK(ctx, cudaMemcpyAsync(assign, L->d_assign, sizeof(int32_t) * L->T, kind, s));
    if (frames) OBB_CK(ctx, cudaMemcpyAsync(frames, L->d_frames, sizeof(double) * 9 * L->K, kind, s));
    if (qboxes) OBB_CK(ctx, cudaMemcpyAsync(qboxes, L->d_q, sizeof(obb_qbox) * L->K, kind, s));
    if (obv) OBB_CK(ctx, cudaMemcpyAsync(obv, L->d_obv, sizeof(uint64_t) * L->K, kind, s));
    if (boxes) {
        HostTmp hb(ctx);
        obb_box* db;
        OBB_TRY(out_device(ctx, boxes, (size_t)L->K, on_device, hb, &db));
        launch_box_report(ctx, L->lat, L->d_frames, L->d_q, L->K, db);
        OBB_CK(ctx, cudaGetLastError());
        OBB_TRY(copy_back(ctx, boxes, db, (size_t)L->K, on_device));
        if (!on_device) return check_device_error(ctx);
    }
    if (!on_device) return check_device_error(ctx);
    return OBB_OK;
}

int32_t obb_layer_clusters(const obb_layer* L) { return L ? L->K : 0; }

obb_status obb_layer_set_surrogate(obb_ctx* ctx, obb_layer* L, const obb_mlp* mlp, int32_t topk)
{
    if (!ctx || !L) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (L->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    if (mlp && obbv::mlp_owner(mlp) != ctx) return fail(ctx, OBB_ERR_STATE, "network belongs to another context");
    if (topk < 0 || topk > 6) return fail(ctx, OBB_ERR_ARG, "topk must be in [0, 6]");
    return layer_set_surrogate(ctx, L, mlp, topk);
}

obb_status obb_layer_last_candidates(obb_ctx* ctx, const obb_layer* L, obb_qbox* boxes, uint64_t* counts, int64_t cap,
                                     int64_t* n)
{
    if (!ctx || !L || !n || (cap > 0 && !boxes)) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (L->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    return layer_last_candidates(ctx, L, boxes, counts, cap, n);
}

obb_status obb_layer_moments(obb_ctx* ctx, obb_layer* L, int32_t compensated, double* out)
{
    if (!ctx || !L || !out) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (L->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    return layer_moments(ctx, L, compensated, out);
}

obb_status obb_layer_members(obb_ctx* ctx, obb_layer* L, int32_t* members, int32_t* start)
{
    if (!ctx || !L) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (L->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    OBB_TRY(layer_members(ctx, L));
    if (members)
        OBB_CK(ctx, cudaMemcpyAsync(members, L->d_members, sizeof(int32_t) * L->T, cudaMemcpyDeviceToHost,
                                    ctx->stream));
    if (start)
        OBB_CK(ctx, cudaMemcpyAsync(start, L->d_start, sizeof(int32_t) * (L->K + 1), cudaMemcpyDeviceToHost,
                                    ctx->stream));
    OBB_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

void obb_layer_free(obb_layer* L) { layer_destroy(L); }

obb_status obb_batch_create(obb_ctx* ctx, obb_layer* const* layers, int32_t n, obb_batch** out)
{
    if (!ctx || !layers || !out) return fail(ctx, OBB_ERR_ARG, "null argument");
    *out = nullptr;
    if (n < 1 || n > (1 << 20)) return fail(ctx, OBB_ERR_ARG, "a batch holds 1 to 2^20 layers");
    std::unordered_set<const obb_layer*> seen;
    for (int32_t i = 0; i < n; ++i) {
        if (!layers[i]) return fail(ctx, OBB_ERR_ARG, "null layer in the batch");
        if (layers[i]->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
        if (!seen.insert(layers[i]).second) return fail(ctx, OBB_ERR_ARG, "a layer appears twice in the batch");
    }
    obb_batch* B = new (std::nothrow) obb_batch();
    if (!B) return fail(ctx, OBB_ERR_OOM, "batch");
    obb_status st = batch_create(ctx, layers, n, B);
    if (st != OBB_OK) {
        batch_destroy(B);
        return st;
    }
    *out = B;
    return OBB_OK;
}

obb_status obb_batch_lloyd_step(obb_ctx* ctx, obb_batch* B, const obb_step_opts* opts, obb_step_stats* stats)
{
    if (!ctx || !B) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (B->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "batch belongs to another context");
    return batch_lloyd_step(ctx, B, opts, stats);
}

void obb_batch_free(obb_batch* B) { batch_destroy(B); }

obb_status obb_layer_split(obb_ctx* ctx, const obb_layer* L, int32_t* child, int32_t on_device)
{
    if (!ctx || !L || !child) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (L->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "layer belongs to another context");
    HostTmp hc(ctx);
    int32_t* dc;
    OBB_TRY(out_device(ctx, child, (size_t)L->T, on_device, hc, &dc));
    OBB_TRY(split_layer(ctx, L, dc));
    OBB_TRY(copy_back(ctx, child, dc, (size_t)L->T, on_device));
    return check_device_error(ctx);
}

obb_status obb_build_tree(obb_ctx* ctx, const obb_lattice* lat, const obb_tree_opts* opts, obb_tree** out)
{
    if (!ctx || !lat || !opts || !out) return fail(ctx, OBB_ERR_ARG, "null argument");
    *out = nullptr;
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    obb_tree* t = new (std::nothrow) obb_tree();
    if (!t) return fail(ctx, OBB_ERR_OOM, "host allocation");
    obb_status st = build_tree(ctx, lat, opts, t);
    if (st == OBB_OK) st = check_device_error(ctx);
    if (st != OBB_OK) {
        obb_tree_free(t);
        return st;
    }
    *out = t;
    return OBB_OK;
}

obb_status obb_tree_read(obb_ctx* ctx, const obb_tree* tree, int32_t level, int32_t* assign, double* frames,
                         obb_qbox* qboxes, obb_box* boxes, uint64_t* obv)
{
    if (!ctx || !tree) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (tree->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "tree belongs to another context");
    if (level < 0 || level >= (int32_t)tree->layers.size()) return fail(ctx, OBB_ERR_ARG, "level out of range");
    return obb_layer_read(ctx, tree->layers[level], assign, frames, qboxes, boxes, obv, 0);
}

obb_status obb_tree_parents(obb_ctx* ctx, const obb_tree* tree, int32_t level, int32_t* parent)
{
    if (!ctx || !tree || !parent) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (tree->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "tree belongs to another context");
    if (level < 0 || level >= (int32_t)tree->layers.size()) return fail(ctx, OBB_ERR_ARG, "level out of range");
    return obb_layer_parents(ctx, tree->layers[level], parent);
}

int32_t obb_tree_depth(const obb_tree* tree) { return tree ? (int32_t)tree->layers.size() - 1 : -1; }

obb_status obb_tree_sweep(obb_ctx* ctx, obb_tree* tree, const obb_sweep_opts* opts, obb_sweep_stats* stats)
{
    if (!ctx || !tree) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (tree->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "tree belongs to another context");
    return tree_sweep(ctx, tree, opts, stats);
}

obb_status obb_tree_score(obb_ctx* ctx, const obb_tree* tree, double* points, double* volume)
{
    if (!ctx || !tree) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (tree->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "tree belongs to another context");
    const int depth = (int)tree->layers.size() - 1;
    double acc = 0.0;
    for (int L = 0; L <= depth; ++L) {
        const obb_layer* ly = tree->layers[L];
        std::vector<uint64_t> o(ly->K);
        OBB_CK(ctx, cudaMemcpyAsync(o.data(), ly->d_obv, sizeof(uint64_t) * ly->K, cudaMemcpyDeviceToHost, ctx->stream));
        OBB_TRY(check_device_error(ctx));
        double sum = 0.0;
        for (uint64_t v : o) sum += (double)v;
        acc += (double)(depth - L + 1) * sum;
    }
    if (points) *points = acc;
    if (volume) {
        OBB_TRY(obbv::lattice_frame_host(tree->lat));
        const LatticeFrame& f = tree->lat->frame;
        *volume = acc * f.h[0] * f.h[1] * f.h[2];
    }
    return OBB_OK;
}

void obb_tree_free(obb_tree* tree)
{
    if (!tree) return;
    for (auto it = tree->layers.rbegin(); it != tree->layers.rend(); ++it) layer_destroy(*it);
    delete tree;
}

}  // extern "C"
