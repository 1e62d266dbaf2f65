/*
 * obbvar — exact outer volume of oriented bounding boxes and the variational
 * OBB-tree construction of "Variational Hierarchical Directed Bounding Box
 * Construction for Solid Mesh Models" (arXiv 2203.10521), on one GPU.
 *
 * C ABI.  Plain pointers and sizes; no C++ or framework types cross it.
 *
 * Conventions
 *  - Every function returning obb_status returns OBB_OK (0) or a negative
 *    code; obb_last_error(ctx) gives a one-line explanation of the last
 *    failure on that context.  No exception crosses the ABI.
 *  - Opaque handles (obb_ctx, obb_mesh, obb_lattice, obb_layer, obb_tree,
 *    obb_batch, obb_mlp) are owned by the library and released with their
 *    *_free / obb_destroy call.  A lattice borrows its mesh, a layer its
 *    lattice, a tree its lattice: free in the reverse order of creation.
 *    Every handle belongs to the context that created it; a call given a
 *    handle of another context returns OBB_ERR_STATE before any work.
 *  - Input arrays are borrowed for the duration of the call.  Output arrays
 *    are owned by the caller.  Arguments named on_device say whether the
 *    caller's arrays live in device memory (1) or host memory (0).
 *  - Work is enqueued on the context's CUDA stream.  Calls whose outputs are
 *    host arrays synchronise that stream before returning; calls with device
 *    outputs return as soon as the work is enqueued.  Errors detected on the
 *    device (range overflow of a box) are reported by the next call that
 *    synchronises.
 *  - One GPU, no CPU fallback: a context fails to create without a device.
 *
 * Geometry (readings of the paper shared by every call)
 *  - Lattice: N points per axis, cell centred over the vertex AABB:
 *    x_b(i) = lo_b + (i + 1/2) h_b with h_b = (hi_b - lo_b) / N.  The solid
 *    Omega(X) of Sec. 3 is sampled at these points; the lattice continues
 *    over all of Z^3 with every point outside [0, N)^3 outside the solid.
 *  - Fixed point: vertex coordinates snap to U_b = rint(((x_b - lo_b) / h_b
 *    - 1/2) * 2^8) (FP64, round half to even); lattice point i sits at
 *    U = 256 i.  All inside/outside decisions are exact integer predicates
 *    on U.
 *  - Box: frame R (rows = unit axes), quantised normals
 *    n_ab = rint(2^24 R_ab h_b / h_max) and integer slab bounds:
 *    a lattice point p is in the box iff lo_a <= n_a . (256 p) <= hi_a for
 *    a = 0, 1, 2 (closed box).
 *  - Outer volume (Eq. 4, Sec. 3): the number of lattice points inside the
 *    box and outside the solid.  Multiply by h_0 h_1 h_2 for a volume.
 */
#ifndef OBBVAR_H
#define OBBVAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t obb_status;

enum {
    OBB_OK = 0,
    OBB_ERR_ARG = -1,             /* null pointer, bad size, non-finite or negative box extent */
    OBB_ERR_NOT_WATERTIGHT = -2,  /* an undirected edge is not shared by exactly two triangles */
    OBB_ERR_RANGE = -3,           /* lattice size, fixed-point or box range out of bounds */
    OBB_ERR_EMPTY_CLUSTER = -4,   /* a cluster with no triangle, or one too small to split */
    OBB_ERR_CUDA = -5,            /* a CUDA runtime call failed */
    OBB_ERR_TIMEOUT = -6,         /* a bounded device wait gave up */
    OBB_ERR_OOM = -7,             /* device allocation failed */
    OBB_ERR_STATE = -8            /* handle used with the wrong context or in the wrong order */
};

typedef struct obb_ctx obb_ctx;
typedef struct obb_mesh obb_mesh;
typedef struct obb_lattice obb_lattice;
typedef struct obb_layer obb_layer;
typedef struct obb_tree obb_tree;
typedef struct obb_mlp obb_mlp;
typedef struct obb_batch obb_batch;

/* A world-space oriented box: centre, first two unit axes (axis2 = axis0 x
 * axis1), half extents along the three axes.  48 bytes. */
typedef struct {
    float c[3];
    float axis0[3];
    float axis1[3];
    float half[3];
} obb_box;

/* A quantised box (the exact form every count uses): normals n[a*3+b]
 * (int32, row a = normal of slab a) and bounds b[2a] = lo_a, b[2a+1] = hi_a
 * in fixed-point units.  88 bytes, 8-byte aligned. */
typedef struct {
    int32_t n[9];
    int32_t reserved;
    int64_t b[6];
} obb_qbox;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, enqueuing on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream may be
 * one owned by another framework; it must outlive the context.  The first
 * context on a device creates the library's device memory pool, from which
 * every library allocation on that device comes; memory the library frees
 * stays reserved in the pool for its next allocations (until the process
 * ends).  The device's default memory pool is not touched. */
obb_status obb_create(obb_ctx** out, int32_t device, void* stream);
/* Point the context at another stream (same device). */
obb_status obb_set_stream(obb_ctx* ctx, void* stream);
/* Wait for all work enqueued by the context; reports pending device errors. */
obb_status obb_synchronize(obb_ctx* ctx);
void obb_destroy(obb_ctx* ctx);
const char* obb_last_error(const obb_ctx* ctx);

/* Instrumentation.  `launches` counts every kernel this context has enqueued
 * (library kernels and the radix-sort kernels compiled into the library).
 * With profiling enabled, each launch of the outer-volume counting kernel is
 * bracketed by CUDA events on the context stream (launches inside a Lloyd
 * iteration run as a CUDA graph are not) and the kernel adds up its
 * algorithmic traffic (16 bytes per 128-bit occupancy chunk that a box row's
 * x-interval touches inside the lattice; a row counted through the rank
 * table touches its first and last word's chunks and two 2-byte rank
 * entries), the rows with a non-empty interval and, of these, the rows
 * counted through the rank table.  Every counting launch of the context, profiled or not (those of
 * a captured Lloyd iteration included), also adds up the lattice points of
 * its boxes that lie inside the lattice domain [0, N)^3: the points whose
 * occupancy bit it reads (points outside the domain are empty by definition
 * and cost no memory).  obb_profile_enable resets the totals: on = 1 times
 * every counting launch and adds up its bytes and rows, on = 2 only times it
 * (the kernel then runs without the byte and row counters, as it does with
 * profiling off), on = 0 stops; obb_profile_read synchronises and reports
 * the totals. */
typedef struct {
    int64_t launches;        /* kernels enqueued by the context since creation */
    int64_t count_launches;  /* counting-kernel launches since profiling was enabled */
    double count_ms;         /* their summed duration (CUDA events) */
    double count_bytes;      /* their summed algorithmic bytes */
    double count_rows;       /* (j, k) rows with a non-empty interval inside the lattice or not */
    double count_points_in_domain;   /* in-domain lattice points of all counted boxes (every launch) */
    double count_rows_rank;          /* of count_rows, those counted from their end words and the rank table */
} obb_profile_stats;
obb_status obb_profile_enable(obb_ctx* ctx, int32_t on);
obb_status obb_profile_read(obb_ctx* ctx, obb_profile_stats* out);

/* ------------------------------------------------------------------- mesh */

/* The closed triangle mesh X of Sec. 3 (Definition 1 needs a solid):
 * verts float32 [n_verts][3], tris int32 [n_tris][3], host memory.
 * Validates that every undirected edge is shared by exactly two triangles
 * (OBB_ERR_NOT_WATERTIGHT otherwise) and that every index is in range, builds
 * the edge adjacency used by the Lloyd step (Sec. 4.2.1 "adjacent faces")
 * and copies everything to the device. */
obb_status obb_mesh_create(obb_ctx* ctx, const float* verts, int64_t n_verts, const int32_t* tris,
                           int64_t n_tris, obb_mesh** out);
void obb_mesh_free(obb_mesh* mesh);

/* ---------------------------------------------------------- occupancy (a) */

/* Solid occupancy Omega(X) (Sec. 3) on the N^3 lattice, 1 <= N <= 2048,
 * by per-column crossing parity: snap the vertices (fixed point above); for
 * every column (j, k) covered by a triangle's (y, z) projection, decide
 * containment of the column point with Simulation of Simplicity (query point
 * perturbed by (+eps, +eps^2)), compute the first index i* = ceil(x* / 256)
 * whose point is at or beyond the crossing, and flip bit i*; a prefix XOR
 * along each row then gives inside = odd number of crossings at or before
 * the point.  Bit-exact.
 * Layout (device, owned by the lattice): uint64 words, row (j, k) starts at
 * word (k*N + j) * W with W = 2 * ceil(N / 128) (rows padded to 16 bytes);
 * point i is bit (i & 63) of word (i >> 6); padding bits are 0.
 * Synchronises once (reads back the lattice frame and the error word). */
obb_status obb_build_occupancy(obb_ctx* ctx, const obb_mesh* mesh, int32_t N, obb_lattice** out);

/* Recompute the occupancy of an existing lattice from its mesh in place
 * (same N, same buffers, no allocation): the work of obb_build_occupancy
 * without the handle creation.  Asynchronous on the context stream: errors
 * found on the device surface at the next synchronising call, and the host
 * copy of the frame read by obb_lattice_desc is refreshed when it is next
 * read. */
obb_status obb_occupancy_rebuild(obb_ctx* ctx, obb_lattice* lat);

/* Borrowed view of a lattice: frame (lo, h), N, words per row, device
 * pointers to the occupancy words and to the snapped vertices (int32 [n][3]).
 * Any pointer argument may be NULL. */
obb_status obb_lattice_desc(const obb_lattice* lat, double lo[3], double h[3], int32_t* N,
                            int64_t* row_words, const uint64_t** d_words, const int32_t** d_fixed);
void obb_lattice_free(obb_lattice* lat);

/* -------------------------------------------------------- outer volume (b) */

/* Quantise K world-space boxes to the exact integer form (Sec. 4.2.1: a box
 * is its position and axes plus the extents; here normals and slab bounds):
 * axis2 = axis0 x axis1 (FP64), n_ab = rint(2^24 R_ab h_b / h_max),
 * m_a = sum_b R_ab ((c_b - lo_b) - h_b / 2), s = 2^32 / h_max,
 * lo_a = floor((m_a - half_a) s), hi_a = ceil((m_a + half_a) s), every step a
 * correctly rounded FP64 operation in this order.  A box with a non-finite
 * value or a negative half extent flags OBB_ERR_ARG. */
obb_status obb_quantize_boxes(obb_ctx* ctx, const obb_lattice* lat, const obb_box* boxes, int64_t K,
                              obb_qbox* out, int32_t on_device);

/* Outer volume OBV(X, O) of Eq. 4 for K quantised boxes: counts[k] = number
 * of lattice points of Z^3 in box k that are outside the solid (exact);
 * points[k] (optional, may be NULL) = number of lattice points in box k.
 * Each box's index-space bounding box must lie within +-2^20 of the lattice
 * (OBB_ERR_RANGE otherwise).  counts/points are uint64 [K]. */
obb_status obb_outer_volume_q(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* boxes, int64_t K,
                              uint64_t* counts, uint64_t* points, int32_t on_device);

/* Outer volume of K quantised boxes without allocating any device memory.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory once they are running, such as a real-time collision or
 * physics loop working inside a fixed memory budget, or a host framework that
 * owns the whole device memory pool and forbids allocations outside it.
 * Results equal obb_outer_volume_q's.  boxes, counts and points (optional)
 * are device arrays the caller provides; K <= OBB_NOALLOC_MAX_BOXES, larger K
 * is rejected with OBB_ERR_RANGE.  The per-box scratch lives in one fixed
 * device array inside the library (about 1.6 MB), held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up that array's device address; make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents, so calls that overlap on the GPU (different streams or threads
 * without ordering) race: order them on one stream.  Asynchronous on the
 * context stream; device-detected errors surface at the next synchronising
 * call. */
#define OBB_NOALLOC_MAX_BOXES 4096
obb_status obb_outer_volume_q_noalloc(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* boxes, int64_t K,
                                      uint64_t* counts, uint64_t* points);

/* obb_outer_volume_q over boxes of several lattices (many meshes) in one
 * counting launch: box k is counted on lats[lattice_of_box[k]] (int32 [K]).
 * lats is a host array of n_lats lattice handles of this context.  An index
 * out of range flags OBB_ERR_ARG.  Synchronises. */
obb_status obb_outer_volume_multi(obb_ctx* ctx, const obb_lattice* const* lats, int32_t n_lats, const obb_qbox* boxes,
                                  const int32_t* lattice_of_box, int64_t K, uint64_t* counts, uint64_t* points,
                                  int32_t on_device);

/* Rows one lane visits per counting tile (1..128; default 32).  The count is
 * exact for every value; only its speed changes.  Steps already captured as
 * CUDA graphs are recaptured on their next call. */
obb_status obb_set_counting_tile(obb_ctx* ctx, int32_t tile_k);

/* Rank tables (default on = 1): every lattice keeps, per row, the number of
 * occupied bits before each 64-bit word (2 bytes per word, rebuilt with the
 * occupancy), and a box whose rows are long is counted from each row's two
 * end words and two rank entries instead of every word of the interval
 * (constant work per row).  on = 0 reads every word.  The count is exact
 * either way; only its speed changes.  Steps already captured as CUDA graphs
 * are recaptured on their next call.  OBB_ERR_ARG unless 0 or 1. */
obb_status obb_set_counting_rank(obb_ctx* ctx, int32_t on);

/* Spatial order (default on = 1): a batch of at least 1,024 boxes on lattices
 * of at least 64 MiB of occupancy words (larger than about half the L2),
 * counted outside a CUDA-graph capture, is scheduled by the 16^3 Morton cell
 * of each box's centre, so that boxes of every size over one region of the
 * lattice are counted together and reuse its words from L2.  on = 0 counts the boxes
 * in the caller's order.  Counts do not depend on it.  OBB_ERR_ARG unless 0
 * or 1. */
obb_status obb_set_counting_order(obb_ctx* ctx, int32_t on);

/* Row axis of the counting kernel.  By default (axis = 0) every box is counted
 * in rows along x.  With axis = -1 each box is counted along the index axis
 * whose perpendicular plane receives its smallest shadow (the fewest rows);
 * 1 or 2 force rows along y or z.  For these the lattice keeps two more copies
 * of its occupancy with rows along y and z (bit transposes, 2x the lattice's
 * memory, refreshed by every rebuild); lattices get them at their next build
 * or rebuild after the axis is set, and a lattice without them is counted
 * along x.  Worth it when a lattice is counted many times between rebuilds.
 * The count is exact for every choice; only its speed changes.  Steps already
 * captured as CUDA graphs are recaptured on their next call.  OBB_ERR_ARG
 * outside -1..2. */
obb_status obb_set_counting_axis(obb_ctx* ctx, int32_t axis);

/* Test hook for the device-side timeouts.  OBB_INJECT_TC_STALL arms the next
 * launch of the tensor-core network (surrogate inference) to skip its first
 * group of MMAs and their commit, so its bounded mbarrier wait (250 ms) gives
 * up: the kernel sets a device error flag, frees its tensor memory and
 * returns, and the call reports OBB_ERR_TIMEOUT at its next synchronisation.
 * Nothing is left in flight and the context stays usable.  One launch only;
 * OBB_ERR_ARG for unknown bits. */
#define OBB_INJECT_TC_STALL 1
obb_status obb_test_inject(obb_ctx* ctx, int32_t flags);

/* Autotuner of the counting kernel: times the outer-volume count of the given
 * quantised boxes with 8, 16, 32 and 64 rows per tile (one warm-up and three
 * timed runs each, CUDA events on the context stream), keeps the fastest for
 * the context and returns it in *tile_k; ms (may be NULL) receives the four
 * average times in milliseconds.  qboxes: [K], host or device (on_device).
 * Synchronises. */
obb_status obb_tune_counting(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* qboxes, int64_t K,
                             int32_t on_device, int32_t* tile_k, float* ms);

/* The paper's own estimator of the outer volume (Sec. 4.1, Eq. 9-10), as ray
 * casting in place of cube-map rasterisation: from each box centre o one ray
 * per texel of a 6 x m x m cube map (through the texel centre, weighted by
 * the texel's exact solid angle dOmega).  Mesh crossings at r_i below the box
 * exit r_e carry s_i = +1 leaving the solid, -1 entering (Fig. 1a); with
 * chi(o) = 1 inside the solid and chi_e = chi(o) - sum s_i, a texel adds
 * dOmega / 3 (r_e^3 - sum s_i r_i^3 - chi_e r_e^3) (cone volumes; Eq. 10 read
 * as a volume integral).  out[k] float64 is the estimate in world units^3 for
 * box k; the mesh must be closed with outward-oriented triangles.  FP32 ray
 * tests against every triangle: a cross-check, not the exact count.
 * 1 <= m <= 256. */
obb_status obb_directional_outer_volume(obb_ctx* ctx, const obb_mesh* mesh, const obb_box* boxes, int64_t K,
                                        int32_t m, double* out, int32_t on_device);

/* obb_quantize_boxes followed by obb_outer_volume_q. */
obb_status obb_outer_volume(obb_ctx* ctx, const obb_lattice* lat, const obb_box* boxes, int64_t K,
                            uint64_t* counts, uint64_t* points, int32_t on_device);

/* ------------------------------------------------------ Lloyd layer (c) */

/* One layer Z of Sec. 3: K clusters of triangles (the partition of Eq. 11)
 * with their boxes.  assign int32 [n_tris] in [0, K); parent int32 [K]:
 * moves are allowed only between clusters with the same parent (siblings),
 * which keeps the tree nested.  frames (optional, float64 [K][9], rows =
 * axes): when NULL each cluster's frame comes from the eigenvectors of its
 * area-weighted triangle covariance (FP32 compensated sums, FP64 Jacobi).
 * Boxes are the tight slabs of the cluster's vertices; the outer volume of
 * each is counted exactly.  Every cluster must be non-empty
 * (OBB_ERR_EMPTY_CLUSTER). */
obb_status obb_layer_init(obb_ctx* ctx, const obb_lattice* lat, const int32_t* assign,
                          const int32_t* parent, int32_t K, const double* frames, int32_t on_device,
                          obb_layer** out);

typedef struct {
    int32_t rounds;         /* partition rounds per step (stop earlier when a round accepts nothing); <= 0: 16 */
    int32_t refit;          /* box-parameter update after the rounds: 0 none, 1 covariance frame,
                               2 rotation descent, 3 both (covariance first) */
    int32_t descent_steps;  /* descent steps per iteration when refit & 2; <= 0: 2 */
    int32_t graph;          /* 1: run the iteration as one CUDA graph with a device-side round loop
                               (captured on first use per rounds / refit / descent_steps, then
                               relaunched; same kernels, same results, no host round trip per round;
                               ignored while a surrogate is attached).  0: host-driven rounds. */
} obb_step_opts;

typedef struct {
    int32_t rounds_run;
    int32_t refits_accepted;
    int64_t proposals;         /* over all rounds */
    int64_t moves;             /* accepted triangle moves */
    int64_t gain;              /* sum of accepted gains, lattice points */
    int64_t box_evals;         /* exact box counts performed */
    uint64_t points_counted;   /* lattice points inside the boxes counted */
    uint64_t total_obv;        /* sum of the layer's outer volumes after the step */
} obb_step_stats;

/* One Lloyd iteration on the layer (Sec. 4.2.1, Eq. 11-13), in place.
 * Partition rounds: every triangle t of a cluster s with >= 2 triangles that
 * is extremal in s (attains one of s's six slab bounds) evaluates moving to
 * each sibling cluster k of its edge neighbours with the exact gain
 *   [OBV(s) - OBV(s without t)] - [OBV(k with t) - OBV(k)]
 * (boxes keep their frames; bounds follow the new membership); it proposes
 * its best k (largest gain, ties to the smaller k) when the gain is > 0.
 * A proposal is accepted when its key (gain, then smaller t) is the largest
 * among all proposals whose source or target cluster is its source or
 * target, so accepted moves touch disjoint clusters and the layer total
 * drops by exactly the sum of their gains.
 * Box update (opts->refit), each kept only when the exact outer volume
 * strictly drops: (1) covariance frame -- eigenvectors of the cluster's
 * area-weighted covariance, tight bounds, exact count; only clusters whose
 * membership changed since their last try are recomputed (the others would
 * rebuild the frame already tried); (2) rotation descent, the perturbation
 * search of Sec. 4.2.1 step 2 -- six probes per cluster rotate its frame
 * about each of its axes by +-theta, rational rotation cos = (1 - t^2)/(1 +
 * t^2), sin = 2t/(1 + t^2), t = 2^-(5 + level), the best probe kept when it
 * lowers the exact count, else level += 1 (theta halves; clusters at level 8
 * stop; a membership change resets level to 0).
 * stats may be NULL; when given, the call synchronises. */
obb_status obb_lloyd_step(obb_ctx* ctx, obb_layer* layer, const obb_step_opts* opts, obb_step_stats* stats);

/* Read a layer: assign int32 [n_tris], frames float64 [K][9], qboxes [K],
 * boxes [K] (world-space report form of the quantised boxes), obv uint64 [K].
 * Any output may be NULL. */
obb_status obb_layer_read(obb_ctx* ctx, const obb_layer* layer, int32_t* assign, double* frames,
                          obb_qbox* qboxes, obb_box* boxes, uint64_t* obv, int32_t on_device);

/* Moments of the layer's clusters (the input of the covariance refit,
 * Gottschalk-style continuous triangle surface, coordinates relative to the
 * cluster's own origin: the first vertex of its lowest-numbered triangle):
 * out float64 [K][10] = {sum A, sum A m (3),
 * sum A/12 (9 m m^T + p p^T + q q^T + r r^T) (6: xx yy zz xy xz yz)}, host
 * memory.  compensated = 1 sums them as the refit does (FP32 products and
 * sums with error-free transformations, Knuth's TwoSum and Dekker's
 * TwoProduct); 0 sums the same terms in plain FP32 (a diagnostic of what the
 * compensation buys).  Synchronises. */
obb_status obb_layer_moments(obb_ctx* ctx, obb_layer* layer, int32_t compensated, double* out);
int32_t obb_layer_clusters(const obb_layer* layer);

/* The layer's member lists, the order every per-cluster reduction of the
 * Lloyd step (Sec. 4.2.1: extents, covariance sums, tight bounds) walks:
 * members int32 [n_tris] = the triangles sorted by cluster, ascending
 * triangle index within a cluster (a stable sort of the assignment);
 * start int32 [K + 1] = where each cluster's triangles begin (start[K] =
 * n_tris).  Host arrays; either may be NULL.  Rebuilt first if the
 * assignment changed since the last rebuild.  Synchronises. */
obb_status obb_layer_members(obb_ctx* ctx, obb_layer* layer, int32_t* members, int32_t* start);

typedef struct {
    int32_t waves;       /* flooding waves run */
    int32_t reserved;
    int64_t box_evals;   /* grown boxes counted exactly */
} obb_flood_stats;

/* Patch division by flooding (Sec. 4.2.1 step 1, Eq. 12-13): the layer's
 * triangles are re-partitioned among its boxes, whose frames and centres stay
 * fixed; a triangle may only join a box of its group (the parent of its
 * current cluster).  Priority of a triangle: distance from its centroid (FP64
 * mean of its three vertices) to the nearest centre of its group's boxes,
 * rounded to float, ties by triangle index.  Each box first takes the nearest
 * untaken triangle of its group (boxes in index order); then a triangle
 * becomes available once an edge neighbour of its group is assigned, and a
 * taken triangle joins, among the boxes holding such a neighbour, the one
 * whose exact outer volume grows least (ties -> smaller box); a group with no
 * available triangle takes its unassigned triangle of smallest priority with
 * all its boxes as candidates.  mode 0 (exact) takes the available triangle
 * of smallest priority in every group per wave -- the paper's sequential
 * priority-queue order -- and mode 1 (wavefront) every available triangle at
 * once, each evaluated against its boxes as the wave found them.  centres: [K][3]
 * world coordinates (FP64, host or device), or NULL for the current boxes'
 * centres.  The layer's assignment, slabs (tight) and outer volumes are
 * replaced; its frames are kept and every cluster is marked for the next
 * refit.  A group may hold at most 8 boxes (OBB_ERR_STATE beyond).  stats may
 * be NULL.  Synchronises. */
obb_status obb_flood_partition(obb_ctx* ctx, obb_layer* layer, const double* centres, int32_t mode,
                               obb_flood_stats* stats);

typedef struct {
    int32_t kept;            /* 1 if the adjustment lowered the layer's total and was kept */
    int32_t k;               /* the re-seated box (-1: no box has a sibling) */
    int32_t m;               /* the sibling that took k's triangles */
    int32_t j;               /* the sibling that was split to seat k again */
    uint64_t total_before;   /* the layer's total outer volume before and after */
    uint64_t total_after;
} obb_adjust_stats;

/* Adjustment of the layer's boxes out of a local minimum (Sec. 4.2.1 step 3:
 * the least important box is adjusted; kept only if the error drops).  The
 * least important box k is the one with fewest triangles (ties -> smaller
 * index) among boxes with a sibling.  Its triangles go to the sibling m that
 * shares most triangle edges with it (ties -> smaller index), whose slab is
 * recomputed; then the sibling j with the largest outer volume (ties ->
 * smaller index) is split at the median of its triangles along its major axis
 * (key n_0 . (U_p + U_q + U_r), ties by triangle index): the first ceil(n/2)
 * stay in j, the rest become box k with j's frame.  `iters` obb_lloyd_step
 * iterations with `opts` follow; the layer is restored unless its total outer
 * volume is then strictly smaller.  stats may be NULL.  Synchronises. */
obb_status obb_layer_adjust(obb_ctx* ctx, obb_layer* layer, const obb_step_opts* opts, int32_t iters,
                            obb_adjust_stats* stats);

/* The layer's parent map, int32 [K] (host array), as given to obb_layer_init
 * and as changed by obb_unit_step on the layer above.  Synchronises. */
obb_status obb_layer_parents(obb_ctx* ctx, const obb_layer* layer, int32_t* parent);

/* One Lloyd iteration of `upper` whose division units are the boxes of
 * `lower` (Sec. 4.2.2, bottom-up merging: the same-layer method with boxes,
 * not triangles, as the unit).  The two layers must nest: for every triangle
 * t, upper.assign[t] == lower.parent[lower.assign[t]], else OBB_ERR_ARG.
 * A unit u of cluster s moves as a whole to a cluster k != s with the same
 * parent (upper's parent map) that holds a triangle edge-adjacent to one of
 * u's triangles, provided s keeps another unit; the exact gain is
 *   [OBV(s) - OBV(s without u)] - [OBV(k with u) - OBV(k)]
 * with tight slab bounds in the clusters' own frames.  Each unit proposes
 * its best k (gain > 0, ties -> smallest k); proposals are matched as in
 * obb_lloyd_step (key: gain desc, unit asc), so accepted moves touch
 * disjoint clusters and the total falls by exactly the sum of their gains.
 * Rounds repeat up to opts->rounds (<= 0: 16) or until none is accepted.
 * lower's parent map and upper's assignment, boxes and outer volumes change
 * in place; then upper's boxes are updated as opts->refit says (as in
 * obb_lloyd_step).  A unit may border at most 8 sibling clusters
 * (OBB_ERR_STATE beyond).  stats may be NULL.  Synchronises. */
obb_status obb_unit_step(obb_ctx* ctx, obb_layer* upper, obb_layer* lower, const obb_step_opts* opts,
                         obb_step_stats* stats);

/* Median split of every cluster of the layer into two children, the seeding
 * step of the top-down decomposition (Sec. 4.2.2): triangles of cluster c are
 * ordered by key n_0 . (U_p + U_q + U_r) (the cluster's quantised major axis
 * applied to three times the fixed-point centroid, exact int64), ties by
 * triangle index; the first ceil(size / 2) get child[t] = 2c, the rest 2c + 1.
 * child is int32 [n_tris].  OBB_ERR_EMPTY_CLUSTER if a cluster has fewer
 * than two triangles.  Synchronises. */
obb_status obb_layer_split(obb_ctx* ctx, const obb_layer* layer, int32_t* child, int32_t on_device);
void obb_layer_free(obb_layer* layer);

/* --------------------------------------------------------- tree (d) */

typedef struct {
    int32_t depth;    /* levels below the root; 2^depth leaves */
    int32_t iters;    /* Lloyd iterations per level (stop early when one changes nothing) */
    int32_t rounds;   /* partition rounds per iteration; <= 0: 16 */
    int32_t refit;    /* box-parameter update in each iteration (obb_step_opts.refit) */
} obb_tree_opts;

typedef struct {
    int32_t sweeps;   /* reciprocating sweeps (bottom-up pass, then top-down pass) */
    int32_t iters;    /* Lloyd iterations per level visit (stop early when one changes nothing) */
    int32_t rounds;   /* partition rounds per iteration; <= 0: 16 */
    int32_t refit;    /* box-parameter update in each iteration (obb_step_opts.refit) */
} obb_sweep_opts;

typedef struct {
    double eq7_before;        /* Eq. 7 in lattice points before and after the sweeps */
    double eq7_after;
    int64_t unit_moves;       /* moves of whole lower-level boxes */
    int64_t triangle_moves;   /* moves of triangles at the leaf level */
    int32_t level_iters;      /* Lloyd iterations run over all level visits */
    int32_t reserved;
} obb_sweep_stats;

/* Binary OBB tree by top-down decomposition (Sec. 4.2.2): the root box
 * holds every triangle; each level splits every node into two children at
 * the median of its triangles along the node's major axis (key n_0 . (U_p +
 * U_q + U_r), ties by triangle index, first ceil(size/2) to the first child)
 * and then runs `iters` Lloyd iterations restricted to siblings.  Needs
 * n_tris >= 2^depth (OBB_ERR_EMPTY_CLUSTER when a node has fewer than two
 * triangles to split). */
obb_status obb_build_tree(obb_ctx* ctx, const obb_lattice* lat, const obb_tree_opts* opts, obb_tree** out);

/* Layer `level` (0 = root) of a tree, as obb_layer_read (host arrays). */
obb_status obb_tree_read(obb_ctx* ctx, const obb_tree* tree, int32_t level, int32_t* assign,
                         double* frames, obb_qbox* qboxes, obb_box* boxes, uint64_t* obv);
int32_t obb_tree_depth(const obb_tree* tree);
/* Parent map of layer `level` (int32 [2^level], host array; the root's is {0}). */
obb_status obb_tree_parents(obb_ctx* ctx, const obb_tree* tree, int32_t level, int32_t* parent);

/* Eq. 7 with the layer weights of Sec. 5 (a level's weight = its number of
 * levels to the leaves plus one: leaves 1, their parents 2, ...), each layer's
 * OMV replaced by the sum of its boxes' outer volumes (Eq. 6, Eq. 8):
 * *points = weighted sum in lattice points, *volume = the same times
 * h_0 h_1 h_2.  Either pointer may be NULL. */
obb_status obb_tree_score(obb_ctx* ctx, const obb_tree* tree, double* points, double* volume);

/* Reciprocating optimisation between levels (Sec. 4.2.2, Fig. 5): each sweep
 * first merges bottom-up -- for levels depth-1 .. 1, up to opts->iters
 * obb_unit_step iterations with the level below as units, stopping the pass
 * at the first level whose Eq. 7 does not strictly drop -- and then
 * decomposes top-down: levels 1 .. depth again, unit steps at the inner
 * levels and obb_lloyd_step (triangles) at the leaves.  Every step keeps the
 * tree nested and never raises Eq. 7.  stats may be NULL.  Synchronises. */
obb_status obb_tree_sweep(obb_ctx* ctx, obb_tree* tree, const obb_sweep_opts* opts, obb_sweep_stats* stats);
void obb_tree_free(obb_tree* tree);

/* ------------------------------------------------------- batched layers */

/* Many layers stepped together -- of many meshes, each on its own lattice, or
 * several layers of one tree (Sec. 4.2.1 per layer, batched).  A batch holds
 * borrowed layers of this context (each at most once; they must outlive the
 * batch).  obb_batch_lloyd_step runs one Lloyd iteration of every layer: in
 * each partition round the layers still moving run their kernels, and all
 * their exact outer-volume counts go into one counting launch over all their
 * lattices (a device-side gather of every layer's boxes, one multi-lattice
 * count, a scatter back); the covariance refit of all layers likewise shares
 * one counting launch; the rotation descent (refit mode bit 1) runs layer by
 * layer.  Every layer's state and statistics equal those of obb_lloyd_step
 * with the same options (opts->graph is ignored).  stats: [n] or NULL.
 * Synchronises once per round.  The first step captures each layer's round
 * and refit phases as CUDA graphs, and the same phases of the whole batch
 * (a phase every layer runs alike is then one graph launch); a batch holding
 * a surrogate-screened layer runs without graphs. */
obb_status obb_batch_create(obb_ctx* ctx, obb_layer* const* layers, int32_t n, obb_batch** out);
obb_status obb_batch_lloyd_step(obb_ctx* ctx, obb_batch* batch, const obb_step_opts* opts, obb_step_stats* stats);
void obb_batch_free(obb_batch* batch);

/* ---------------------------------------------------- learned surrogate (e) */

/* A learned screen for the partition rounds of obb_lloyd_step (the paper
 * counts every candidate with its GPU estimator, Sec. 4.1 and Sec. 5; here a
 * small network predicts outer volumes so that only the most promising moves
 * are counted exactly -- the exact count still decides every move).
 * Features of a quantised box (OBB_SURROGATE_INPUTS floats): centre of the
 * box in index space / N (3), unit normals of slabs 0 and 1 (6), half widths
 * (H_a - L_a) / (2 |n_a|) / N (3), then an 8^3 patch of occupancy bits sampled
 * at the points M^-1 v, v_a = L_a + (H_a - L_a)(2 s_a + 1) / 16 (x fastest),
 * rounded to the nearest lattice point (0 outside [0, N)^3); L = ceil(lo/256),
 * H = floor(hi/256), M = n.  Arithmetic: the exact integer adjugate and
 * determinant of n, then FP32 with one rounding per operation in a fixed
 * order (centre plus edge vectors times (2 s_a - 7) / 16), so the features are
 * reproducible bit for bit.
 * Network: 524 -> 128 -> 128 -> 128 -> 1, ReLU, sigmoid output = predicted
 * empty fraction; predicted outer volume = fraction x prod(H_a - L_a + 1) /
 * |det n|.  Parameters (flat float32, obb_mlp_num_params()): W1 [524][128],
 * b1, W2 [128][128], b2, W3 [128][128], b3, W4 [128][1], b4.  Training: mean
 * squared error of the fraction, Adam (0.9, 0.999, 1e-8) on FP32 master
 * weights; inference with half_weights uses FP16 weights and activations on
 * the tensor cores with FP32 accumulation (the screening path). */
#define OBB_SURROGATE_INPUTS 524
obb_status obb_mlp_create(obb_ctx* ctx, uint64_t seed, obb_mlp** out);
void obb_mlp_free(obb_mlp* mlp);
int64_t obb_mlp_num_params(void);
obb_status obb_mlp_params(obb_ctx* ctx, const obb_mlp* mlp, float* out, int32_t on_device);
obb_status obb_mlp_set_params(obb_ctx* ctx, obb_mlp* mlp, const float* in, int32_t on_device);
/* Training targets of K quantised boxes with exact outer volumes counts
 * (uint64 [K]): out[k] = counts[k] / (prod_a (H_a - L_a + 1) / |det n|),
 * clipped to [0, 1] -- the empty fraction in the very cell volume the screen
 * multiplies a prediction by (float [K]). */
obb_status obb_surrogate_targets(obb_ctx* ctx, const obb_qbox* boxes, const uint64_t* counts, int64_t K, float* out,
                                 int32_t on_device);
/* features float [K][524] of K quantised boxes on a lattice */
obb_status obb_surrogate_features(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* boxes, int64_t K, float* feats,
                                  int32_t on_device);
/* out float [B]: predicted empty fractions */
obb_status obb_mlp_forward(obb_ctx* ctx, const obb_mlp* mlp, const float* feats, int64_t B, float* out,
                           int32_t half_weights, int32_t on_device);
/* loss and gradients (flat, obb_mlp_num_params() floats) of the mean squared
 * error against target fractions float [B], FP32 weights; no update */
obb_status obb_mlp_gradients(obb_ctx* ctx, obb_mlp* mlp, const float* feats, const float* target, int64_t B,
                             float* grads, float* loss, int32_t on_device);
/* one Adam step on a mini-batch; *loss (optional) = the batch loss before the step */
obb_status obb_mlp_train_step(obb_ctx* ctx, obb_mlp* mlp, const float* feats, const float* target, int64_t B,
                              float lr, float* loss, int32_t on_device);
/* Screen the layer's Lloyd iterations with a surrogate (mlp = NULL turns it
 * off): in the partition rounds keep, per source cluster, the topk candidate
 * moves by predicted gain (topk = 0: no move screening; at most 6,
 * OBB_ERR_ARG beyond); in the refit count
 * exactly only the new boxes whose predicted outer volume is below 1.05 x the
 * current exact one.  Every accepted move and refit is still decided by the
 * exact count.  The surrogate must outlive its use by the layer. */
obb_status obb_layer_set_surrogate(obb_ctx* ctx, obb_layer* layer, const obb_mlp* mlp, int32_t topk);
/* The boxes counted exactly in the layer's last partition round and their
 * exact outer volumes (host arrays, up to cap); *n = how many there were. */
obb_status obb_layer_last_candidates(obb_ctx* ctx, const obb_layer* layer, obb_qbox* boxes, uint64_t* counts,
                                     int64_t cap, int64_t* n);

#ifdef __cplusplus
}
#endif

#endif /* OBBVAR_H */
