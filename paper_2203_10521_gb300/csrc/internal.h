// Internal declarations shared by the translation units of libobbvar.
// Nothing here crosses the C ABI (include/obbvar.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/obbvar.h"

namespace obbv {

constexpr int kS = 8;            // fixed-point fraction bits of snapped vertices
constexpr int kQ = 24;           // fraction bits of quantised normals
constexpr int kMaxN = 2048;      // lattice points per axis
constexpr int kSurrogateInputs = 524;   // 12 box parameters + 8^3 occupancy patch
constexpr int64_t kBoxRange = int64_t(1) << 20;  // |index-space AABB| limit of a counted box
#ifndef OBB_TILE_K
#define OBB_TILE_K 32
#endif
constexpr int kTileK = OBB_TILE_K;               // rows along z one lane steps through per tile
constexpr int kOrderBuckets = 4096;              // spatial-order buckets of a counting launch (16^3 Morton cells)
constexpr int kScanBlock = 2048;                 // positions per block of the counting path's two-pass offset scan

#ifdef __CUDACC__
// Integer -> FP32 through 32-bit conversions (relative error below 3 * 2^-24,
// 4 * 2^-24 from 128 bits):
// 64-bit conversions issue on the FP64 pipe.
__device__ __forceinline__ float u64_to_float(uint64_t x)
{
    return fmaf((float)(uint32_t)(x >> 32), 4294967296.0f, (float)(uint32_t)x);
}

__device__ __forceinline__ float i64_to_float(int64_t x)
{
    const float f = u64_to_float(x < 0 ? 0ull - (uint64_t)x : (uint64_t)x);
    return x < 0 ? -f : f;
}

__device__ __forceinline__ float i128_to_float(__int128 x)   // |x| < 2^126
{
    const unsigned __int128 a = x < 0 ? (unsigned __int128)(-x) : (unsigned __int128)x;
    const float f = fmaf(u64_to_float((uint64_t)(a >> 64)), 18446744073709551616.0f, u64_to_float((uint64_t)a));
    return x < 0 ? -f : f;
}
#endif

// device error word bits
enum : int32_t {
    kErrRange = 1,
    kErrArg = 2,
    kErrEmpty = 4,
    kErrDegenerate = 8,
    kErrOverflow = 16,
    kErrTimeout = 32,   // a bounded wait in a kernel gave up
};

// Lattice frame; identical copies on the host and the device.
struct LatticeFrame {
    double lo[3];
    double h[3];
    double hmax;
    double center[3];   // lo + N h / 2
    double s256[3];     // 256 rn(1 / h) (the snap's fast path)
    int32_t N;
    int32_t W;          // uint64 words per row (even)
};

// Per-box data the counting kernel needs, prepared once per box.
// Rows (j, k) of the box's index-space AABB are cut into tiles of wj rows
// along y by wk * tk rows along z (wj * wk = 32 lanes); each lane owns one j
// and visits tk rows spaced wk apart along z.  Slab a bounds i through
// quotients by dd_a = |n_a0|; from one visited row to the next the quotient
// moves by qstep_a with remainder carry rstep_a, or by fstep_a in 32.32 fixed
// point (an integer DDA either way).
struct alignas(128) BoxPrep {
    // read by every tile of the box (first two 128-byte lines) ...
    const uint64_t* words;   // the box's lattice with rows along `axis`
    int32_t latN, latW;      // its N and words per row
    int32_t ntj;             // tiles along y: ceil(nj / wj)
    int32_t lwj;             // log2 of wj, the lanes of a tile along y (wk = 32 / wj along z)
    int32_t tk;              // rows one lane visits per tile (tiles are wj x wk * tk rows)
    int32_t mode;            // 2 bits per slab: 0 n_a0 = 0, 1 32-bit DDA, 2 per-row clip
    int32_t j0, k0;          // first row
    int32_t nj, nk;          // rows along y and z (0 = empty box)
    int32_t i0, span;        // index-space AABB along x: [i0, i0 + span]
    int32_t axis;            // rows run along index axis 0 (x), 1 (y) or 2 (z); n's columns permuted to match
    int32_t lat;             // index of the box's lattice in the launch's lattice table
    int32_t rank;            // row counting: 0 every word, 1 end words + rank table, 2 end words (rows <= 64 points)
    const uint16_t* ranks;   // the rank table of `words` (ones before each word of a row)
    // Separating axes of the box's shadow on the (j, k) plane: the normals of
    // its three projected edge directions, and the shadow's extent along each,
    // widened by two rows.  A tile whose rectangle lies outside one of these
    // bands holds no row of the box.
    float sat_nu[3][2];
    float sat_lo[3], sat_hi[3];
    // The same bands solved for k: rows k - k0 of column j lie within
    // [kc_lo[a] + kc_s[a] (j - j0), kc_hi[a] + kc_s[a] (j - j0)] for every a
    // (widened by a rounding margin; an unconstraining band has kc_s = 0 and
    // infinite bounds).
    float kc_s[3], kc_lo[3], kc_hi[3];
    int32_t n[9];
    int32_t dd[3];           // |n_a0|
    // ... by the exact seeds of a tile's first row
    int64_t Lq[3], Hq[3];    // ceil(lo / 256), floor(hi / 256)
    uint64_t fmul[3];        // floor((2^64 - 1) / dd): remainder -> 32-bit fraction
    int64_t fstep[3];        // floor(step * 2^32), step = qstep + rstep / dd (32.32 fixed point)
    // ... and by the general row loop only
    int32_t rstep[3];        // remainder of that step, in [0, dd)
    int32_t qstep[3];        // quotient of the step between a lane's rows (|.| < 2^25 for DDA slabs)
};

// One lattice as the counting kernel sees it (a table of these lets one launch
// count boxes of many meshes).
// The counting copies interleave the rows of a slice by column: word w of
// row (slice s, column c) at (s W + w) N + c, so that the lanes of a warp,
// which count neighbouring columns, read neighbouring words.
struct LatRef {
    const uint64_t* words;     // rows along x: row (k, j), bit i (slice k, column j)
    const uint64_t* words_y;   // rows along y: row (k, i), bit j (slice k, column i)
    const uint64_t* words_z;   // rows along z: row (j, i), bit k (slice j, column i)
    // rank tables of the three: entry (row, w) = occupied bits in words 0..w-1
    // of that row (uint16, the same interleaved layout)
    const uint16_t* rank;
    const uint16_t* rank_y;
    const uint16_t* rank_z;
    int32_t N;
    int32_t W;
};

// Stream-ordered device allocation that only grows.
// Scratch of the counting path at fixed addresses (used while a step is
// captured into a CUDA graph): prep [cap], tiles + offsets [2 cap + 2] and
// the offset scan's block totals.
struct CountScratch {
    BoxPrep* prep = nullptr;
    int64_t* tiles = nullptr;
    int64_t* bsum = nullptr;          // [cap / kScanBlock + 1] block totals of the offset scan
    int64_t cap = 0;
};

// A counting request recorded instead of launched while a batched step
// collects the requests of many layers (obb_batch_lloyd_step): K = *d_K boxes
// (at most K_cap) of one lattice into counts / points (points may be null).
struct CountReq {
    const ::obb_lattice* lat;
    const obb_qbox* boxes;
    const int32_t* d_K;
    int64_t K_cap;
    uint64_t* counts;
    uint64_t* points;
};

// The same request as the flush kernels read it (device copy).
struct BatchReq {
    const obb_qbox* boxes;
    const int32_t* d_K;
    uint64_t* counts;
    uint64_t* points;
    int64_t cap;
    int32_t lat;      // index into the flush's lattice table
    int32_t pad;
};

// Stream-ordered device allocation from the library's own memory pool of the
// current device (created by obb_create; freed memory stays reserved in the
// pool for the next allocation instead of going back to the driver at every
// synchronisation).  Same contract as cudaMallocAsync; cudaFreeAsync frees.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t pool_alloc(T** p, size_t bytes, cudaStream_t s)
{
    return pool_alloc(reinterpret_cast<void**>(p), bytes, s);
}
// creates (once per device) the pool pool_alloc draws on
cudaError_t pool_init(int device);

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t n, cudaStream_t s);
    void release(cudaStream_t s);
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

}  // namespace obbv

struct obb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    int32_t* d_err = nullptr;        // device error word
    unsigned int* d_ticket = nullptr; // finish counter of the box-preparation blocks (zero between launches)
    const obbv::CountScratch* count_scratch = nullptr;   // set while a step is being captured
    std::vector<obbv::CountReq>* count_defer = nullptr;  // set while a batched step collects counting requests
    int32_t tile_k = obbv::kTileK;   // rows per lane per counting tile
    int32_t count_axis = 0;          // row axis of counted boxes (0: x; -1: per box, the smallest shadow)
    int32_t count_rank = 1;          // long rows counted from their end words and the rank table (0: every word)
    int32_t count_order = 1;         // large batches counted in spatial order (0: in the caller's order)
    int32_t inject = 0;              // test hooks armed by obb_test_inject (OBB_INJECT_*)
    int32_t tile_gen = 0;            // bumped when tile_k changes (captured steps recapture)
    int32_t* h_small = nullptr;      // pinned host staging (512 bytes; the first 64 hold the error word)
    // scratch reused across calls
    obbv::DevBuf prep, chunk_off, qscratch, cscratch, pscratch, kdev, tmp_a, tmp_b, tmp_c, tmp_d,
        cub_tmp, order;
    unsigned int* d_order_hist = nullptr;   // spatial-order buckets of the counting path
    // instrumentation: kernels launched by this context, and the optional
    // profile of the outer-volume counting kernel (CUDA events + byte totals)
    int64_t launches = 0;
    int32_t prof = 0;                // 0 off, 1 events and counters, 2 events only
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
    // [0] algorithmic bytes, [1] rows, [3] rows counted with the rank table (profiled
    // launches); [2] in-domain points (every launch)
    unsigned long long* d_prof = nullptr;
    std::map<std::pair<int64_t, int>, int> sort_launch_cache;
};

struct obb_mesh {
    obb_ctx* ctx = nullptr;
    int64_t nv = 0, nt = 0;
    float* d_verts = nullptr;        // [nv][3]
    int32_t* d_tris = nullptr;       // [nt][3]
    int32_t* d_adj = nullptr;        // [nt][3] neighbour across edge (v_e, v_e+1)
};

struct obb_lattice {
    obb_ctx* ctx = nullptr;
    const obb_mesh* mesh = nullptr;
    mutable obbv::LatticeFrame frame{};   // host copy (lo, h refreshed on demand after a rebuild)
    mutable bool frame_stale = false;      // a rebuild may have moved lo / h since the last copy
    obbv::LatticeFrame* d_frame = nullptr;
    int32_t* d_fixed = nullptr;      // [nv][3] snapped vertices
    uint64_t* d_words = nullptr;     // occupancy, rows along x: row (k, j) at (k N + j) W, bit i
    uint64_t* d_cwords = nullptr;    // its counting copy, rows interleaved by column (LatRef)
    uint64_t* d_words_y = nullptr;   // counting copies with rows along y, then z (counting boxes
    uint64_t* d_words_z = nullptr;   // along their shortest-shadow axis)
    uint16_t* d_rank = nullptr;      // rank tables of the counting copies along x, y, z
    uint16_t* d_rank_y = nullptr;
    uint16_t* d_rank_z = nullptr;
    size_t n_words = 0;
    obbv::LatRef ref{};              // host copy of the table entry below
    obbv::LatRef* d_ref = nullptr;   // this lattice as a one-entry table
};

// per-cluster top-2 extents along the six slab sides (2a = low side, 2a+1 = high side)
struct ClusterExt {
    int64_t v1[6];   // extreme value (min for low sides, max for high sides)
    int64_t v2[6];   // extreme over the members other than arg[side]
    int32_t arg[6];  // smallest triangle index attaining v1
    int32_t pad[2];
};

struct obb_layer {
    obb_ctx* ctx = nullptr;
    const obb_lattice* lat = nullptr;
    int32_t K = 0;
    int64_t T = 0;
    int32_t* d_assign = nullptr;
    int32_t* d_parent = nullptr;
    double* d_frames = nullptr;      // [K][9]
    obb_qbox* d_q = nullptr;         // [K]
    uint64_t* d_obv = nullptr;       // [K]
    int32_t* d_size = nullptr;       // [K]
    int32_t* d_start = nullptr;      // [K + 1]
    int32_t* d_members = nullptr;    // [T] triangles sorted by cluster (stable)
    ClusterExt* d_ext = nullptr;     // [K]
    unsigned long long* d_best = nullptr;  // [K] best proposal key per cluster
    int64_t* d_stats = nullptr;      // device counters (see lloyd.cu)
    void* aux = nullptr;             // per-layer scratch owned by lloyd.cu
    const obb_mlp* mlp = nullptr;    // optional surrogate screening candidate moves
    int32_t topk = 0;                // candidates kept per source cluster when screening
};

#ifndef OBB_BATCH_STREAMS
#define OBB_BATCH_STREAMS 16   // streams a batched step spreads its layers' graphs over
#endif
struct obb_batch {
    obb_ctx* ctx = nullptr;
    std::vector<obb_layer*> layers;
    obbv::DevBuf tables, scratch;    // counting requests of a batched phase, and their gathered boxes
    obbv::DevBuf stat_ptrs;          // the layers' device counters, then their accepted-move totals
    int64_t* h_acc = nullptr;        // pinned host copy of the accepted-move totals
    // Each layer's partition round as CUDA graphs, captured on first use: the
    // phase before the counting launch (with and without the member-list
    // rebuild) and the phase after it, with their kernel counts and the
    // layer's counting request; replayed over kBatchStreams streams.
    static constexpr int kBatchStreams = OBB_BATCH_STREAMS;
    bool graphs = false;
    // the same for the covariance refit after the rounds (g_rpre*, g_rpost)
    std::vector<cudaGraphExec_t> g_pre, g_pre_rebuild, g_post, g_rpre, g_rpre_rebuild, g_rpost;
    std::vector<int32_t> k_pre, k_pre_rebuild, k_post, k_rpre, k_rpre_rebuild, k_rpost;
    std::vector<obbv::CountReq> req, rreq;
    obbv::DevBuf fin;                // the layers' outer-volume pointers and K, then their counters + totals
    int64_t* h_fin = nullptr;        // pinned host copy of the counters + totals
    cudaStream_t par[kBatchStreams] = {};
    cudaEvent_t ev[kBatchStreams + 1] = {};
};

struct obb_tree {
    obb_ctx* ctx = nullptr;
    const obb_lattice* lat = nullptr;
    std::vector<obb_layer*> layers;
};

namespace obbv {

inline void note_launch(obb_ctx* ctx, int n = 1) { ctx->launches += n; }
// pinned staging for step counters, clear of the error word check_device_error reads
inline int64_t* host_stats(obb_ctx* ctx) { return reinterpret_cast<int64_t*>(ctx->h_small) + 8; }
// Number of kernels one library call enqueues, found once per shape by
// capturing the call into a CUDA graph on a side stream (nothing runs).
int captured_launches(obb_ctx* ctx, int64_t key0, int key1, const std::function<cudaError_t(cudaStream_t)>& fn);

obb_status fail(obb_ctx* ctx, obb_status code, const std::string& msg);
obb_status cuda_fail(obb_ctx* ctx, cudaError_t e, const char* what);
obb_status check_device_error(obb_ctx* ctx);   // synchronises, reads and clears the error word
obb_status lattice_frame_host(const obb_lattice* lat);   // refreshes lat->frame if stale (synchronises)

#define OBB_CK(ctx, call)                                              \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::obbv::cuda_fail((ctx), e_, #call); \
    } while (0)

#define OBB_TRY(expr)                         \
    do {                                      \
        obb_status s_ = (expr);               \
        if (s_ != OBB_OK) return s_;          \
    } while (0)

// occupancy.cu
obb_status build_occupancy(obb_ctx* ctx, const obb_mesh* mesh, int32_t N, obb_lattice* lat);
obb_status rebuild_occupancy(obb_ctx* ctx, obb_lattice* lat);

// outer_volume.cu
obb_status quantize_boxes(obb_ctx* ctx, const obb_lattice* lat, const obb_box* d_boxes, int64_t K,
                          obb_qbox* d_out);
// counts / points (points may be null) for K boxes whose count is held on the device at
// d_K (int32); K_cap bounds it for scratch sizing.  counts/points are zeroed here.
obb_status count_boxes(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* d_boxes,
                       const int32_t* d_K, int64_t K_cap, uint64_t* d_counts, uint64_t* d_points);
// the same over boxes of several lattices: box k uses d_lats[d_lat_of_box[k]];
// lattice_bytes (the lattices' occupancy words together) decides the spatial order
obb_status count_boxes_multi(obb_ctx* ctx, const LatRef* d_lats, int32_t n_lats, const int32_t* d_lat_of_box,
                             const obb_qbox* d_boxes, const int32_t* d_K, int64_t K_cap, uint64_t* d_counts,
                             uint64_t* d_points, int64_t lattice_bytes);
obb_status set_device_int(obb_ctx* ctx, int32_t* d_dst, int32_t value);
// Count the recorded requests in one multi-lattice launch: their boxes are
// gathered into one list (device-side offsets from each request's box count),
// counted, and the counts scattered back.  `tables` (device, held by the
// caller) must hold at least reqs.size() BatchReq; `scratch` (device, held by
// the caller) grows as needed.
obb_status count_flush(obb_ctx* ctx, const std::vector<CountReq>& reqs, DevBuf& tables, DevBuf& scratch);
// exclusive scan of n int32 values into out[n + 1] (out[n] = total), single block
void launch_scan_i32(obb_ctx* ctx, const int32_t* in, int32_t* out, const int32_t* d_n);
void launch_box_report(obb_ctx* ctx, const obb_lattice* lat, const double* d_frames, const obb_qbox* d_q,
                       int32_t K, obb_box* d_out);

// lloyd.cu
obb_status layer_create(obb_ctx* ctx, const obb_lattice* lat, const int32_t* d_assign,
                        const int32_t* d_parent, int32_t K, const double* d_frames,
                        const double* d_fallback, obb_layer** out);
obb_status lloyd_step(obb_ctx* ctx, obb_layer* L, const obb_step_opts* opts, obb_step_stats* st);
void layer_destroy(obb_layer* L);
obb_status rebuild_members(obb_ctx* ctx, obb_layer* L);
obb_status layer_set_surrogate(obb_ctx* ctx, obb_layer* L, const obb_mlp* mlp, int32_t topk);
obb_status layer_last_candidates(obb_ctx* ctx, const obb_layer* L, obb_qbox* out, uint64_t* counts, int64_t cap,
                                 int64_t* n);
// cluster moments [K][10] (host) summed as the refit sums them (compensated) or in plain FP32
obb_status layer_moments(obb_ctx* ctx, obb_layer* L, int32_t compensated, double* out);
// batched layers (obb_batch_*)
obb_status batch_create(obb_ctx* ctx, obb_layer* const* layers, int32_t n, obb_batch* B);
void batch_destroy(obb_batch* B);
obb_status batch_lloyd_step(obb_ctx* ctx, obb_batch* B, const obb_step_opts* opts, obb_step_stats* stats);
// pieces of the Lloyd step that the step between levels (sweep.cu) reuses
enum { kStProposals = 0, kStAccepted, kStGain, kStEvals, kStRefits, kStPoints, kStCount };
obb_status layer_box_update(obb_ctx* ctx, obb_layer* L, int refit_mode, int dsteps);
obb_status layer_finish_stats(obb_ctx* ctx, obb_layer* L, int ran, obb_step_stats* st);
uint8_t* layer_dirty(obb_layer* L);      // [K] membership changed since the last covariance refit
int32_t* layer_level(obb_layer* L);      // [K] rotation-descent level
const int32_t* layer_dev_K(obb_layer* L);   // device copy of K
obb_status layer_members(obb_ctx* ctx, obb_layer* L);   // member lists valid on return
void layer_members_changed(obb_layer* L);
void launch_sum_points(obb_ctx* ctx, const uint64_t* d_pts, const int32_t* d_n, int64_t* d_stats);

// surrogate.cu: features of boxes [0, *d_K) and predicted outer volumes (FP16 weights)
obb_status surrogate_predict(obb_ctx* ctx, const obb_mlp* mlp, const obb_lattice* lat, const obb_qbox* d_boxes,
                             const int32_t* d_K, int64_t cap, float* d_feats, float* d_pred);

// directional.cu: Eq. 9-10 estimator
obb_status directional_outer_volume(obb_ctx* ctx, const obb_mesh* mesh, const obb_box* d_boxes, int64_t K, int32_t m,
                                    double* d_out);

// sweep.cu: steps between levels (Sec. 4.2.2)
obb_status unit_step(obb_ctx* ctx, obb_layer* up, obb_layer* low, const obb_step_opts* opts, obb_step_stats* st);
obb_status tree_sweep(obb_ctx* ctx, obb_tree* tree, const obb_sweep_opts* opts, obb_sweep_stats* out);

// flood.cu: patch division by flooding (Sec. 4.2.1 step 1)
obb_status flood_partition(obb_ctx* ctx, obb_layer* L, const double* d_centres, int32_t mode, obb_flood_stats* out);

// adjust.cu: box adjustment out of local minima (Sec. 4.2.1 step 3)
obb_status layer_adjust(obb_ctx* ctx, obb_layer* L, const obb_step_opts* opts, int32_t iters, obb_adjust_stats* out);

// mesh.cu: upload and device-side validation + adjacency of a closed mesh
obb_status mesh_upload(obb_ctx* ctx, const float* verts, int64_t nv, const int32_t* tris, int64_t nt, obb_mesh* m);

// tree.cu
obb_status build_tree(obb_ctx* ctx, const obb_lattice* lat, const obb_tree_opts* opts, obb_tree* tree);
obb_status split_layer(obb_ctx* ctx, const obb_layer* up, int32_t* d_child);

}  // namespace obbv
