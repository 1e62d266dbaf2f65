// Exact outer volume of oriented boxes on the occupancy lattice (Eq. 4).
//
// A box is the integer slab set lo_a <= n_a . (256 p) <= hi_a.  Counting:
//   prep   per box: index-space bounds Lq = ceil(lo / 256), Hq = floor(hi / 256),
//          a conservative (j, k) rectangle (exact integer cofactors, FP32
//          geometry with explicit margins), the row axis (x unless the context
//          counts along the axis of the smallest shadow), the tile shape, the
//          per-row step of each slab's quotient (remainder and 32.32 forms) and
//          three separating bands of the box's shadow on the (j, k) plane; the
//          last block to finish scans the tile counts into per-box offsets and
//          clears the work counter;
//   count  persistent warps take one tile at a time from the counter: wj (y)
//          x wk * tk (z) rows of one box, wj * wk = 32 lanes.  A tile outside
//          the box's shadow is skipped and the rows of a tile are clipped to
//          it.  Each lane owns one j and walks tk rows along z: it divides the
//          six slab bounds exactly once per tile (integer reciprocal) and then
//          steps them as 32.32 fixed-point values (boxes whose three slabs are
//          DDA slabs) or with a remainder carry (the general loop), so each
//          row's exact x-interval costs adds and compares only.  The occupied
//          bits of the interval are popcounted over 64-bit words; outer volume
//          = interval length - occupied bits, and rows or points outside
//          [0, N)^3 are all empty.
// Counts are integer sums (warp reduction + one 64-bit atomic per tile), so
// the result does not depend on scheduling.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

#ifndef OBB_COUNT_UNROLL
#define OBB_COUNT_UNROLL 1
#endif
#ifndef OBB_GRAB
#define OBB_GRAB 1
#endif
// OBB_COUNT_MINB, OBB_COUNT_MINB_SMALL: resident blocks of the counting kernel
// per SM the register budget aims at, on lattices of at least
// OBB_ORDER_MIN_MB MiB and on smaller ones
#ifndef OBB_COUNT_MINB
#define OBB_COUNT_MINB 5
#endif
#ifndef OBB_COUNT_MINB_SMALL
#define OBB_COUNT_MINB_SMALL 4
#endif
// OBB_BIG_TK_ROWS: boxes with at least this many (j, k) rows use tiles twice as tall (0: off)
#ifndef OBB_BIG_TK_ROWS
#define OBB_BIG_TK_ROWS 16384
#endif
// OBB_RANK_MIN_BITS: a box whose rows may be at least this long (in lattice
// points) is counted through the rank table; shorter rows (at most 64 points,
// two words) are counted from their two end words
#ifndef OBB_RANK_MIN_BITS
#define OBB_RANK_MIN_BITS 128
#endif
// OBB_ROW_MARGIN: rows added on each side of a box's (j, k) bounding rectangle
#ifndef OBB_ROW_MARGIN
#define OBB_ROW_MARGIN 1
#endif
// OBB_ORDER_MIN_BOXES, OBB_ORDER_MIN_MB: batches of at least this many boxes on
// lattices of at least this many MiB of occupancy words are counted in spatial order
#ifndef OBB_ORDER_MIN_BOXES
#define OBB_ORDER_MIN_BOXES 1024
#endif
#ifndef OBB_ORDER_MIN_MB
#define OBB_ORDER_MIN_MB 64
#endif
namespace obbv {
constexpr int64_t kOrderMinBoxes = OBB_ORDER_MIN_BOXES;
constexpr int64_t kOrderMinLatticeBytes = int64_t(OBB_ORDER_MIN_MB) << 20;
// tuning parameters: unroll factor of the counting kernel's row loop, tiles per work grab
constexpr int kCountUnroll = OBB_COUNT_UNROLL;
constexpr int kRowMargin = OBB_ROW_MARGIN;
constexpr int kPrepThreads = 32;   // one warp per preparation block: its per-box work spreads over many SMs
constexpr int kGrab = OBB_GRAB;
}  // namespace obbv

namespace obbv {
namespace {

// ---------------------------------------------------------------- quantise

__global__ void k_quantize(const obb_box* __restrict__ boxes, int64_t K, const LatticeFrame* __restrict__ f,
                           obb_qbox* __restrict__ out, int32_t* err)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= K) return;
    const obb_box B = boxes[k];
    const float* raw = reinterpret_cast<const float*>(&B);
    bool bad = false;
    for (int q = 0; q < 12; ++q) bad |= !isfinite(raw[q]);
    double R[9];
    for (int b = 0; b < 3; ++b) {
        R[b] = (double)B.axis0[b];
        R[3 + b] = (double)B.axis1[b];
    }
    R[6] = __dsub_rn(__dmul_rn(R[1], R[5]), __dmul_rn(R[2], R[4]));
    R[7] = __dsub_rn(__dmul_rn(R[2], R[3]), __dmul_rn(R[0], R[5]));
    R[8] = __dsub_rn(__dmul_rn(R[0], R[4]), __dmul_rn(R[1], R[3]));
    const double hm = f->hmax;
    const double s = __ddiv_rn(4294967296.0, hm);
    obb_qbox o;
    o.reserved = 0;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            double t = __dmul_rn(R[3 * a + b], f->h[b]);
            t = __ddiv_rn(t, hm);
            t = __dmul_rn(t, 16777216.0);
            o.n[3 * a + b] = (int32_t)rint(t);
        }
        double half = (double)B.half[a];
        bad |= !(half >= 0.0);
        double m = 0.0;
        for (int b = 0; b < 3; ++b) {
            double d = __dsub_rn((double)B.c[b], f->lo[b]);
            d = __dsub_rn(d, 0.5 * f->h[b]);
            m = __dadd_rn(m, __dmul_rn(R[3 * a + b], d));
        }
        double lo = floor(__dmul_rn(__dsub_rn(m, half), s));
        double hi = ceil(__dmul_rn(__dadd_rn(m, half), s));
        if (!(fabs(lo) < 4.0e18 && fabs(hi) < 4.0e18)) bad = true;
        o.b[2 * a] = bad ? 0 : (int64_t)lo;
        o.b[2 * a + 1] = bad ? -1 : (int64_t)hi;
    }
    if (bad) {
        atomicOr(err, kErrArg);
        for (int q = 0; q < 9; ++q) o.n[q] = (q % 4 == 0) ? 1 : 0;
        for (int a = 0; a < 3; ++a) {
            o.b[2 * a] = 0;
            o.b[2 * a + 1] = -1;   // empty
        }
    }
    out[k] = o;
}

// ------------------------------------------------------------------- prep

// The index axis along which a box is counted with the fewest rows: the one
// whose perpendicular plane receives the box's smallest shadow.  The shadow of
// the parallelepiped with edges e_a (columns of n^-1 scaled by H_a - L_a) on
// the plane of axes (s, t) has area sum_{a<b} |e_a,s e_b,t - e_a,t e_b,s|
// (FP32 from exact cofactors; ties to the lower axis).
__device__ __forceinline__ int choose_axis(const obb_qbox& q)
{
    int64_t m[9];
    for (int i = 0; i < 9; ++i) m[i] = q.n[i];
    const int64_t C[9] = {m[4] * m[8] - m[5] * m[7], m[2] * m[7] - m[1] * m[8], m[1] * m[5] - m[2] * m[4],
                          m[5] * m[6] - m[3] * m[8], m[0] * m[8] - m[2] * m[6], m[2] * m[3] - m[0] * m[5],
                          m[3] * m[7] - m[4] * m[6], m[1] * m[6] - m[0] * m[7], m[0] * m[4] - m[1] * m[3]};
    const __int128 det = (__int128)m[0] * C[0] + (__int128)m[1] * C[3] + (__int128)m[2] * C[6];
    if (det == 0) return 0;
    const float id = 1.0f / i128_to_float(det);
    float E[9];   // E[3 r + a]: component r of edge a
    for (int a = 0; a < 3; ++a) {
        const float d = i64_to_float((q.b[2 * a + 1] >> kS) - (-((-q.b[2 * a]) >> kS)));
        for (int r = 0; r < 3; ++r) E[3 * r + a] = i64_to_float(C[3 * r + a]) * id * d;
    }
    int best = 0;
    float best_area = 0.0f;
    for (int ax = 0; ax < 3; ++ax) {
        const int u = (ax + 1) % 3, v = (ax + 2) % 3;
        float area = 0.0f;
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b) area += fabsf(E[3 * u + a] * E[3 * v + b] - E[3 * v + a] * E[3 * u + b]);
        if (ax == 0 || area < best_area) {
            best = ax;
            best_area = area;
        }
    }
    return best;
}

__device__ __noinline__ void k_prep_box(const obb_qbox* __restrict__ boxes, int64_t k,
                                        const LatRef* __restrict__ lats, int32_t n_lats,
                                        const int32_t* __restrict__ lat_of_box, int32_t tile_k, int32_t axis_mode,
                                        int32_t count_rank, BoxPrep* __restrict__ prep,
                                        int64_t* __restrict__ tiles, int32_t* err)
{
    const obb_qbox q = boxes[k];
    BoxPrep p;
    // count along the chosen axis: the index axes are relabelled (axis, then
    // the other two in order), which permutes the columns of n; the slab
    // bounds are unchanged
    p.axis = 0;
    {
        const int32_t li = lat_of_box ? lat_of_box[k] : 0;
        // a lattice without its y- and z-row copies is counted along x
        if (axis_mode != 0 && li >= 0 && li < n_lats && lats[li].words_y)
            p.axis = axis_mode > 0 ? axis_mode : choose_axis(q);
    }
    p.lat = lat_of_box ? lat_of_box[k] : 0;
    bool bad_lat = p.lat < 0 || p.lat >= n_lats;
    if (bad_lat) {
        atomicOr(err, kErrArg);
        p.lat = 0;
    }
    const LatRef lr = lats[p.lat];
    const int32_t N = lr.N;
    p.words = p.axis == 0 ? lr.words : (p.axis == 1 ? lr.words_y : lr.words_z);
    p.ranks = p.axis == 0 ? lr.rank : (p.axis == 1 ? lr.rank_y : lr.rank_z);
    p.latN = lr.N;
    p.latW = lr.W;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)   // new axis c is old axis (axis, the others in order)[c]
            p.n[3 * a + c] = q.n[3 * a + (c == 0 ? p.axis : (c <= p.axis ? c - 1 : c))];
    bool empty = bad_lat;
    p.mode = 0;
    for (int a = 0; a < 3; ++a) {
        p.Lq[a] = -((-q.b[2 * a]) >> kS);
        p.Hq[a] = q.b[2 * a + 1] >> kS;
        empty |= p.Lq[a] > p.Hq[a];
        const int32_t d = p.n[3 * a];
        p.dd[a] = d >= 0 ? d : -d;
        p.qstep[a] = 0;
        p.rstep[a] = 0;
        p.fmul[a] = 0;
        p.fstep[a] = 0;
        // slab kind: 0 = n_a0 == 0 (a band in (y, z)), 1 = quotient DDA in 32 bits,
        // 2 = quotient DDA in 64 bits (|n_a0| < 32: the slab is almost parallel to x)
        const int kind = d == 0 ? 0 : (p.dd[a] >= 32 ? 1 : 2);
        p.mode |= kind << (2 * a);
    }
    p.i0 = 0;
    p.span = -1;
    p.rank = 0;
    p.j0 = p.k0 = 0;
    p.nj = p.nk = p.ntj = 0;
    for (int a = 0; a < 3; ++a) {
        p.sat_nu[a][0] = p.sat_nu[a][1] = 0.0f;
        p.sat_lo[a] = -1.0f;
        p.sat_hi[a] = 1.0f;
        p.kc_s[a] = 0.0f;
        p.kc_lo[a] = -1e30f;
        p.kc_hi[a] = 1e30f;
    }
    if (!empty) {
        // Exact cofactors of the integer normals (|n| <= 2^24: every product is
        // below 2^48) and the exact determinant in 128 bits; the geometry below
        // is FP32 with explicit margins (FP64 and 64-bit int <-> float
        // conversions issue on the FP64 pipe, a small fraction of the FP32
        // rate on this GPU).
        int64_t m[9];
        for (int i = 0; i < 9; ++i) m[i] = p.n[i];
        // C[3 r + a] = adjugate entry (r, a): M^-1 = C / det
        const int64_t C[9] = {m[4] * m[8] - m[5] * m[7], m[2] * m[7] - m[1] * m[8], m[1] * m[5] - m[2] * m[4],
                              m[5] * m[6] - m[3] * m[8], m[0] * m[8] - m[2] * m[6], m[2] * m[3] - m[0] * m[5],
                              m[3] * m[7] - m[4] * m[6], m[1] * m[6] - m[0] * m[7], m[0] * m[4] - m[1] * m[3]};
        const __int128 det = (__int128)m[0] * C[0] + (__int128)m[1] * C[3] + (__int128)m[2] * C[6];
        if (det == 0) {
            atomicOr(err, kErrArg);
            empty = true;
        } else {
            // FP32 inverse (relative error below 10 * 2^-24 per entry) and the
            // slab bounds: centre (L + H) / 2, half width (H - L) / 2, and
            // max(|L|, |H|), which bounds both
            const float id = 1.0f / i128_to_float(det);
            float mi[9];
            for (int i = 0; i < 9; ++i) mi[i] = i64_to_float(C[i]) * id;
            float yc[3], yh[3], ym[3], yl[3], yu[3];
            for (int a = 0; a < 3; ++a) {
                yc[a] = 0.5f * i64_to_float(p.Lq[a] + p.Hq[a]);
                yh[a] = 0.5f * i64_to_float(p.Hq[a] - p.Lq[a]);
                yl[a] = i64_to_float(p.Lq[a]);
                yu[a] = i64_to_float(p.Hq[a]);
                ym[a] = fmaxf(fabsf(yl[a]), fabsf(yu[a]));
            }
            // the parallelepiped {L <= M p <= H} has centre M^-1 (L + H) / 2 and
            // half extent sum_a |M^-1_ra| (H_a - L_a) / 2 along index axis r; the
            // FP32 error of the two together is below 2e-6 of
            // sum_a |M^-1_ra| max(|L_a|, |H_a|), and the bounds are widened by
            // twice that
            float mn[3], mx[3];
            for (int r = 0; r < 3; ++r) {
                float cen = 0.0f, ext = 0.0f, mag = 0.0f;
                for (int a = 0; a < 3; ++a) {
                    const float w = mi[3 * r + a];
                    cen = fmaf(w, yc[a], cen);
                    ext = fmaf(fabsf(w), yh[a], ext);
                    mag = fmaf(fabsf(w), ym[a], mag);
                }
                const float e = 4e-6f * mag + 1e-3f;
                mn[r] = cen - ext - e;
                mx[r] = cen + ext + e;
            }
            const float lim = (float)kBoxRange;
            for (int r = 0; r < 3; ++r)
                if (!(mn[r] > -lim && mx[r] < lim + (float)N)) {
                    atomicOr(err, kErrRange);
                    empty = true;
                }
            if (!empty) {
                const float span_j = mx[1] - mn[1] + 5.0f, span_k = mx[2] - mn[2] + 5.0f;
                if (span_j * span_k > 2.0e9f) {
                    atomicOr(err, kErrRange);
                    empty = true;
                }
            }
            if (!empty) {
                // beyond the widening above, a margin of two columns along x
                // and kRowMargin rows along y and z
                p.i0 = (int32_t)floorf(mn[0]) - 2;
                p.span = (int32_t)ceilf(mx[0]) + 2 - p.i0;
                p.j0 = (int32_t)floorf(mn[1]) - kRowMargin;
                int32_t j1 = (int32_t)ceilf(mx[1]) + kRowMargin;
                p.k0 = (int32_t)floorf(mn[2]) - kRowMargin;
                int32_t k1 = (int32_t)ceilf(mx[2]) + kRowMargin;
                p.nj = j1 - p.j0 + 1;
                p.nk = k1 - p.k0 + 1;
                // shadow on the (j, k) plane: edge a of the parallelepiped runs
                // along column a of M^-1; its normal nu_a in (j, k) is
                // orthogonal to that edge's shadow, and the shadow's extent
                // along nu_a is the sum over the other two constraints b of
                // nu_a . (column b) times [L_b, H_b].  Widened by two rows plus
                // 4e-6 of the terms' magnitude (the FP32 error, including the
                // neglected term of column a, is below 2e-6 of it).
                for (int a = 0; a < 3; ++a) {
                    float nj_ = -mi[3 * 2 + a], nk_ = mi[3 * 1 + a];
                    const float len2 = nj_ * nj_ + nk_ * nk_;
                    const float emax = fmaxf(fabsf(mi[a]), fmaxf(fabsf(mi[3 + a]), fabsf(mi[6 + a])));
                    if (!(len2 > 1e-12f * emax * emax)) continue;   // edge parallel to x: no axis
                    // (only the direction matters: the band below is computed
                    // with this very normal, whatever its length)
                    const float il = rsqrtf(len2);
                    nj_ *= il;
                    nk_ *= il;
                    float lo = 0.0f, hi = 0.0f, mg = 0.0f;
                    for (int b = 0; b < 3; ++b) {
                        mg = fmaf(fabsf(nj_ * mi[3 * 1 + b]) + fabsf(nk_ * mi[3 * 2 + b]), ym[b], mg);
                        if (b == a) continue;
                        const float w = nj_ * mi[3 * 1 + b] + nk_ * mi[3 * 2 + b];
                        const float x0 = w * yl[b], x1 = w * yu[b];
                        lo += fminf(x0, x1);
                        hi += fmaxf(x0, x1);
                    }
                    const float sm = 2.0f + 4e-6f * mg;
                    p.sat_nu[a][0] = nj_;
                    p.sat_nu[a][1] = nk_;
                    p.sat_lo[a] = lo - sm;
                    p.sat_hi[a] = hi + sm;
                    // solved for k relative to (j0, k0), where the band is not
                    // steep in k (|dk/dj| <= 64, so |nu_k| >= 1/65), with one
                    // row plus 1e-5 of the terms' magnitude (above FP32 rounding
                    // here and in the kernel's evaluation)
                    if (fabsf(nj_) <= 64.0f * fabsf(nk_)) {
                        const float ivk = 1.0f / nk_;
                        const float sl = -nj_ * ivk;
                        const float b0 = (nk_ > 0.0f ? p.sat_lo[a] : p.sat_hi[a]) * ivk;
                        const float b1 = (nk_ > 0.0f ? p.sat_hi[a] : p.sat_lo[a]) * ivk;
                        const float fj0 = (float)p.j0, fk0 = (float)p.k0;
                        const float c0 = b0 + sl * fj0 - fk0, c1 = b1 + sl * fj0 - fk0;
                        const float mm = 1.0f + 1e-5f * (fabsf(sl) * (fabsf(fj0) + (float)p.nj) + fabsf(b0) +
                                                         fabsf(b1) + fabsf(fk0));
                        p.kc_s[a] = sl;
                        p.kc_lo[a] = c0 - mm;
                        p.kc_hi[a] = c1 + mm;
                    }
                }
            }
        }
    }
    // rows per lane per tile: long tiles amortise the exact initial division
    // over more rows (set per context; obb_tune_counting picks it by timing)
    p.tk = tile_k;
#if OBB_BIG_TK_ROWS
    // boxes with many rows take tiles twice as tall (fewer tile setups; the
    // row clipping trims their empty ends)
    if ((int64_t)p.nj * p.nk >= OBB_BIG_TK_ROWS && 2 * tile_k <= 128) p.tk = 2 * tile_k;
#endif
    // row counting: a box's rows are at most ell points long, the smallest of
    // span + 1 and (H_a - L_a) / |n_a0| + 1 over the slabs that step along x.
    // With rank tables, long rows (ell >= OBB_RANK_MIN_BITS) are counted from
    // their two end words and the rank table, and rows of at most 64 points
    // (ell < 63.5, well clear of FP32 rounding) from their two end words; both
    // at a fixed cost per row.
    if (p.nj > 0 && count_rank && p.ranks) {
        float ell = fminf((float)p.span + 1.0f, (float)N);
        for (int a = 0; a < 3; ++a)
            if (p.dd[a] > 0) ell = fminf(ell, i64_to_float(p.Hq[a] - p.Lq[a]) / (float)p.dd[a] + 1.0f);
        p.rank = ell >= (float)OBB_RANK_MIN_BITS ? 1 : (ell < 63.5f ? 2 : 0);
    }
    // tile shape: wj lanes along y, wk = 32 / wj along z; the least padding wins
    // (ties to the wider wj, whose rows sit next to each other in memory)
    int best = 5;
    int64_t best_slots = INT64_MAX;
    if (p.nj > 0) {
        // ceil(nk / ((32 >> l) tk)) = ceil(ceil(nk / tk) / 2^(5 - l)): one division
        const int32_t nkt = (p.nk + p.tk - 1) / p.tk;
        for (int l = 5; l >= 0; --l) {
            const int32_t sh = 5 - l;
            const int64_t slots = (int64_t)(((p.nj + (1 << l) - 1) >> l) << l) *
                                  ((int64_t)((nkt + (1 << sh) - 1) >> sh) * ((32 >> l) * p.tk));
            if (slots < best_slots) {
                best_slots = slots;
                best = l;
            }
        }
    }
    // interior box: its whole index rectangle lies in the lattice, so no row
    // and no x-interval needs clamping to [0, N)
    if (p.nj > 0 && p.i0 >= 0 && p.i0 + p.span <= N - 1 && p.j0 >= 0 && p.j0 + p.nj <= N && p.k0 >= 0 &&
        p.k0 + p.nk <= N)
        p.mode |= 1 << 8;
    p.lwj = best;
    const int32_t wj = 1 << best, wk = 32 >> best;
    p.ntj = p.nj > 0 ? (p.nj + wj - 1) / wj : 0;
    for (int a = 0; a < 3; ++a)
        if ((p.mode >> (2 * a)) & 3) {
            // between a lane's rows k advances by wk: X_lo and X_hi move by -sign(d) * n_a2 * wk
            // |delta| <= 2^24 * 32 and 0 < dd < 2^25: exact in 32 bits
            const int32_t delta = -(p.n[3 * a] > 0 ? 1 : -1) * p.n[3 * a + 2] * wk;
            int32_t qs = delta / p.dd[a];
            if (qs * p.dd[a] > delta) --qs;   // floor
            p.qstep[a] = qs;
            p.rstep[a] = delta - qs * p.dd[a];
            // the same step in 32.32 fixed point, rounded down (exact division:
            // rstep < dd <= 2^24, so rstep * 2^32 < 2^56)
            const uint64_t M = ~0ull / (uint64_t)p.dd[a];
            p.fmul[a] = M;
            // floor(rstep 2^32 / dd) through the reciprocal: rstep M / 2^32 is
            // less than 2^-8 below it, so its floor is exact or one short
            const uint32_t rs = (uint32_t)p.rstep[a];
            uint64_t fr = (uint64_t)rs * (uint32_t)(M >> 32) + __umulhi(rs, (uint32_t)M);
            if ((fr + 1) * (uint64_t)p.dd[a] <= ((uint64_t)rs << 32)) ++fr;
            p.fstep[a] = (int64_t)qs * 4294967296LL + (int64_t)fr;
        }
    // A quotient saturated at +-2^30 must stay outside [0, span] for a whole
    // tile: its tk - 1 steps of at most |qstep| + 1 each stay below 2^29.  With
    // |qstep| <= 2^24 every tk <= 32 qualifies; taller tiles are cut for steep
    // slabs.
    {
        int64_t smax = 0;
        for (int a = 0; a < 3; ++a)
            if (((p.mode >> (2 * a)) & 3) == 1) smax = max(smax, (int64_t)abs(p.qstep[a]) + 1);
        if (smax > 0 && (int64_t)(p.tk - 1) * smax >= (int64_t(1) << 29))
            p.tk = (int32_t)max((int64_t)1, min((int64_t)p.tk, (int64_t(1) << 29) / smax));
    }
    prep[k] = p;
    tiles[k] = p.nj > 0 ? (int64_t)p.ntj * ((p.nk + wk * p.tk - 1) / (wk * p.tk)) : 0;
}

// One box per thread (k_prep_box), counts zeroed on the way; then the last
// block to finish (an atomic ticket, nothing waits) turns the tile counts into
// offsets: off[0..K] exclusive, off[K + 1] = 0 (the counting kernel's work
// counter).
__global__ void __launch_bounds__(kPrepThreads) k_prep(const obb_qbox* __restrict__ boxes,
                                                       const int32_t* __restrict__ d_K,
                                                       const LatRef* __restrict__ lats, int32_t n_lats,
                                                       const int32_t* __restrict__ lat_of_box, int32_t tile_k,
                                                       int32_t axis_mode, int32_t count_rank,
                                                       BoxPrep* __restrict__ prep,
                                                       int64_t* __restrict__ tiles,
                                                       int64_t* __restrict__ off,
                                                       unsigned long long* __restrict__ counts,
                                                       unsigned long long* __restrict__ points,
                                                       unsigned int* __restrict__ ticket,
                                                       uint32_t* __restrict__ bucket, unsigned int* __restrict__ hist,
                                                       int32_t scan_tiles, int32_t* err)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t K = *d_K;
    if (k < K) {
        counts[k] = 0;
        if (points) points[k] = 0;
        k_prep_box(boxes, k, lats, n_lats, lat_of_box, tile_k, axis_mode, count_rank, prep, tiles, err);
        if (bucket) {
            // spatial order: the 16^3 Morton cell of the centre of the box's
            // index-space rectangle (clamped to the lattice)
            const BoxPrep& p = prep[k];
            const int32_t N = max(p.latN, 1);
            const int64_t c[3] = {(int64_t)p.i0 + p.span / 2, (int64_t)p.j0 + p.nj / 2, (int64_t)p.k0 + p.nk / 2};
            uint32_t key = 0;
            for (int a = 0; a < 3; ++a) {
                const uint32_t q = (uint32_t)min(max(c[a] * 16 / N, (int64_t)0), (int64_t)15);
                for (int bit = 0; bit < 4; ++bit) key |= ((q >> bit) & 1u) << (3 * bit + a);
            }
            if (n_lats > 1) {
                // several lattices: lattice-major, each lattice's share of the
                // buckets split by the top bits of the Morton cell
                int sub = 0;
                while (sub < 12 && (n_lats << (sub + 1)) <= kOrderBuckets) ++sub;
                key = (uint32_t)(((int64_t)p.lat * kOrderBuckets) / n_lats) + (key >> (12 - sub));
                key = min(key, (uint32_t)kOrderBuckets - 1);
            }
            bucket[k] = key;
            atomicAdd(&hist[key], 1u);
        }
    }
    // the last block's work: the spatial order's bucket starts, or (scan_tiles)
    // the tile offsets in the caller's order; otherwise the offsets come from
    // k_tile_sums / k_tile_offsets
    if (!bucket && !scan_tiles) return;
    // the block's writes, then one gpu-scope fence before its ticket
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    if (!last) return;
    if (bucket) {
        // spatial order: the bucket counts become bucket starts (exclusive
        // scan, one warp, 128 buckets a lane); k_order_scatter,
        // k_tile_sums and k_tile_offsets follow
        const int lane = threadIdx.x & 31;
        constexpr int per = kOrderBuckets / 32;
        unsigned int run = 0;
        for (int q = 0; q < per; ++q) run += hist[lane * per + q];
        unsigned int x = run;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        unsigned int start = x - run;
        for (int q = 0; q < per; ++q) {
            const unsigned int v = hist[lane * per + q];
            hist[lane * per + q] = start;
            start += v;
        }
        if (threadIdx.x == 0) *ticket = 0;   // ready for the next launch
        return;
    }
    // exclusive scan of tiles[0..K) by the last block (one warp): chunks of
    // 8 x 32 consecutive values, a thread's eight in registers (eight loads in
    // flight), a warp scan of the thread sums, and a running carry
    const int lane = threadIdx.x & 31;
    int64_t carry = 0;
    for (int32_t base = 0; base < K; base += 256) {
        int64_t v[8];
        int64_t sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int32_t i = base + 8 * lane + q;
            v[q] = i < K ? tiles[i] : 0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) sum += v[q];
        int64_t x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        int64_t run = carry + x - sum;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int32_t i = base + 8 * lane + q;
            if (i < K) off[i] = run;
            run += v[q];
        }
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (threadIdx.x == 0) {
        off[K] = carry;
        off[K + 1] = 0;
        *ticket = 0;   // ready for the next launch
    }
}

// ---------------------------------------------------------- spatial order

// perm[start of the box's bucket + its place] = box, and the box's tile count
// at the same place (the place within a bucket depends on scheduling; counts
// do not depend on the order)
__global__ void k_order_scatter(const uint32_t* __restrict__ bucket, const int64_t* __restrict__ tiles,
                                const int32_t* __restrict__ d_K, unsigned int* __restrict__ hist,
                                int32_t* __restrict__ perm, int64_t* __restrict__ ptiles)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t K = *d_K;
    if (k >= K) return;
    const unsigned int pos = atomicAdd(&hist[bucket[k]], 1u);
    if (pos < (unsigned int)K) {
        perm[pos] = (int32_t)k;
        ptiles[pos] = tiles[k];
    }
}

// ---------------------------------------------------------- tile offsets

// Tile offsets in counting order (the boxes' own, or the spatial order's
// permuted copy), in two passes over blocks of 2,048
// positions (256 threads, 8 consecutive positions each): k_tile_sums writes
// each block's total; k_tile_offsets adds up the totals of the blocks before
// its own and scans its positions.  off[i] = tiles of the boxes at positions
// 0..i-1, off[K] = all tiles, off[K + 1] = 0 (the counting kernel's work
// counter).
constexpr int kScanPer = 8;
static_assert(256 * kScanPer == kScanBlock, "offset scan: 256 threads x kScanPer positions per block");

__global__ void __launch_bounds__(256) k_tile_sums(const int64_t* __restrict__ tiles,
                                                    const int32_t* __restrict__ d_K, int64_t* __restrict__ bsum)
{
    __shared__ int64_t ws[8];
    const int32_t K = *d_K;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    int64_t v = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) v += base + q < K ? tiles[base + q] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        bsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) k_tile_offsets(const int64_t* __restrict__ tiles,
                                                       const int64_t* __restrict__ bsum,
                                                       const int32_t* __restrict__ d_K, int64_t* __restrict__ off)
{
    __shared__ int64_t ws[8];
    __shared__ int64_t before;
    const int32_t K = *d_K;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the totals of the blocks before this one
    int64_t p = 0;
    for (int32_t b = threadIdx.x; b < (int32_t)blockIdx.x; b += 256) p += bsum[b];
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0) ws[w] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int i = 0; i < 8; ++i) t += ws[i];
        before = t;
    }
    __syncthreads();
    // this block's positions: a thread's eight in registers, then an exclusive
    // scan of the thread sums (warp shuffles, then across the 8 warps)
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t sum = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        v[q] = base + q < K ? tiles[base + q] : 0;
        sum += v[q];
    }
    int64_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();   // ws is reused
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int64_t wbefore = 0;
    for (int i = 0; i < w; ++i) wbefore += ws[i];
    int64_t run = before + wbefore + x - sum;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < K) off[base + q] = run;
        run += v[q];
    }
    // positions past K hold 0, so the thread whose eight positions include K
    // ends with run = off[K] (the launch has K_cap / 2048 + 1 blocks, so it exists)
    if (base <= K && K < base + kScanPer) {
        off[K] = run;
        off[K + 1] = 0;
    }
}

// ------------------------------------------------------- batched requests

// off[r] = boxes of requests 0..r-1 (each request's count clamped to its
// capacity), off[n] and *d_total = all of them; one block of 1024 threads
__global__ void __launch_bounds__(1024) k_batch_offsets(const BatchReq* __restrict__ reqs, int32_t n,
                                                        int64_t* __restrict__ off, int32_t* __restrict__ d_total)
{
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int32_t per = (n + 1023) / 1024;
    const int32_t b0 = min(n, t * per), b1 = min(n, b0 + per);
    int64_t sum = 0;
    for (int32_t r = b0; r < b1; ++r) sum += min((int64_t)max(*reqs[r].d_K, 0), reqs[r].cap);
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - sum;
    for (int32_t r = b0; r < b1; ++r) {
        off[r] = run;
        run += min((int64_t)max(*reqs[r].d_K, 0), reqs[r].cap);
    }
    if (t == 1023) {
        off[n] = part[1023];
        *d_total = (int32_t)part[1023];
    }
}

// the request of combined position j: the last r with off[r] <= j
__device__ __forceinline__ int32_t batch_request(const int64_t* __restrict__ off, int32_t n, int64_t j)
{
    int32_t lo = 0, hi = n;   // off[lo] <= j < off[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_batch_gather(const BatchReq* __restrict__ reqs, int32_t n, const int64_t* __restrict__ off,
                               obb_qbox* __restrict__ boxes, int32_t* __restrict__ lat_of_box)
{
    const int64_t total = off[n];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = batch_request(off, n, j);
        boxes[j] = reqs[r].boxes[j - off[r]];
        lat_of_box[j] = reqs[r].lat;
    }
}

__global__ void k_batch_scatter(const BatchReq* __restrict__ reqs, int32_t n, const int64_t* __restrict__ off,
                                const uint64_t* __restrict__ counts, const uint64_t* __restrict__ points)
{
    const int64_t total = off[n];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = batch_request(off, n, j);
        const int64_t i = j - off[r];
        reqs[r].counts[i] = counts[j];
        if (reqs[r].points) reqs[r].points[i] = points[j];
    }
}

// ------------------------------------------------------------------- scan

// Exclusive scan of n = *d_n int32 values (n <= cap) into out[0..n]; one block.
// out[0..n] = exclusive scan of in[0..n) (n = *d_n), one block of 1,024
// threads: chunks of 4,096 consecutive values (four per thread), a scan of
// the warp sums, and a running carry.
__global__ void __launch_bounds__(1024) k_scan_i32(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                  const int32_t* __restrict__ d_n)
{
    __shared__ int32_t ws[32];
    __shared__ int32_t chunk_total;
    const int32_t n = *d_n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t carry = 0;
    for (int32_t c = 0; c < n; c += 4096) {
        const int32_t b = c + 4 * threadIdx.x;
        int32_t v[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = b + q < n ? in[b + q] : 0;
            sum += v[q];
        }
        int32_t x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        if (w == 0) {
            const int32_t t = ws[lane];
            int32_t u = t;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, u, o);
                if (lane >= o) u += y;
            }
            ws[lane] = u - t;   // warps before
            if (lane == 31) chunk_total = u;
        }
        __syncthreads();
        int32_t run = carry + ws[w] + x - sum;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (b + q < n) out[b + q] = run;
            run += v[q];
        }
        carry += chunk_total;
        __syncthreads();   // ws and chunk_total are rewritten by the next chunk
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// ------------------------------------------------------------------ count

// 32.32 fixed-point DDA.  A slab bound floor(v), v = q + r / dd, is carried as
// A = q 2^32 + floor(r M / 2^32) + kFixBias with M = floor((2^64 - 1) / dd),
// and steps by floor(s 2^32) per row (s the exact rational step).  The seed is
// at most 1 + 2^-8 units (of 2^-32) below v 2^32 and never above it; each
// step loses less than one unit.  After r <= 127 steps the error lies in
// (kFixBias - 1 - 2^-8 - r, kFixBias] = (1.99, 130]: positive, and below
// 2^32 / dd >= 256, the distance from the largest fraction (dd - 1) / dd to
// the next integer.  So A >> 32 is exactly floor(v) on every row of a tile
// of at most 128 rows (the most obb_set_counting_tile allows).
constexpr int64_t kFixBias = 130;

__device__ __forceinline__ int64_t fixed_frac(int32_t r, uint64_t M)   // 0 <= r < 2^24
{
    const uint32_t ru = (uint32_t)r;
    return (int64_t)((uint64_t)ru * (uint32_t)(M >> 32) + __umulhi(ru, (uint32_t)M));
}

// floor(x / d) and its remainder in [0, d), for 0 < d <= 2^24 and |x| < 2^62,
// by the integer reciprocal M = floor((2^64 - 1) / d): the high half of y M
// is at most one below floor(y / d) (M d > 2^64 - d - 1, y < 2^63), so one
// correction makes it exact.  All integer: 64-bit int <-> float conversions
// issue on the FP64 pipe, a small fraction of the integer rate on this GPU.
__device__ __forceinline__ void floordiv_rcp(int64_t x, int32_t d, uint64_t M, int64_t& q, int32_t& r)
{
    const bool neg = x < 0;
    const uint64_t y = neg ? (uint64_t)(-x) + (uint64_t)(d - 1) : (uint64_t)x;   // x < 0: floor(x/d) = -floor(y/d)
    uint64_t qq = __umul64hi(y, M);
    uint64_t rr = y - qq * (uint64_t)d;
    if (rr >= (uint64_t)d) {
        rr -= (uint64_t)d;
        ++qq;
    }
    q = neg ? -(int64_t)qq : (int64_t)qq;
    r = neg ? d - 1 - (int32_t)rr : (int32_t)rr;
}

// Intersect [lo, hi] with { i : L <= d i + c <= H } exactly (d != 0), by
// integer-reciprocal division (M = floor((2^64 - 1) / |d|)).  Used per row for
// slabs almost parallel to x.
__device__ __forceinline__ void clip_slab_rcp(int32_t d, uint64_t M, int64_t c, int64_t L, int64_t H, int32_t& lo,
                                              int32_t& hi)
{
    const int32_t dd = d > 0 ? d : -d;
    const int64_t A = d > 0 ? L - c : c - H;
    const int64_t B = d > 0 ? H - c : c - L;
    int64_t qn, qb;
    int32_t rem;
    floordiv_rcp(-A, dd, M, qn, rem);   // ceil(A / dd) = -floor(-A / dd)
    floordiv_rcp(B, dd, M, qb, rem);
    const int64_t g = min(max(-qn, (int64_t)lo), (int64_t)hi + 1);
    const int64_t u = max(min(qb, (int64_t)hi), (int64_t)lo - 1);
    lo = (int32_t)g;
    hi = (int32_t)u;
}

// popcount of the occupied bits i in [a, e] of one row (0 <= a <= e < N) of
// a counting copy, the row's word w at row[w ws] (ws = N, the copy's column
// interleave); 64-bit words: the first and last word carry the masks (merged
// without a branch when they are the same word), interior words count whole.
__device__ __forceinline__ uint32_t popc_range(const uint64_t* __restrict__ row, int32_t ws, int32_t a, int32_t e)
{
    const int32_t wa = a >> 6, we = e >> 6;
    const uint64_t first = __ldg(row + wa * ws);
    const uint64_t last = __ldg(row + we * ws);
    uint64_t mlo = ~0ull << (a & 63);
    const uint64_t mhi = ~0ull >> (63 - (e & 63));
    uint32_t cnt = 0;
    for (int32_t w = wa + 1; w < we; ++w) cnt += __popcll(__ldg(row + w * ws));
    const bool one = wa == we;
    mlo = one ? (mlo & mhi) : mlo;
    return cnt + __popcll(first & mlo) + __popcll(last & (one ? 0ull : mhi));
}

// The same count through the row's rank table (rk[w ws] = occupied bits in
// words 0..w-1): the bits before e + 1 minus the bits before a, each a rank
// entry plus the popcount of its word below the bit -- four loads whatever
// the row's length, and no case for an interval inside one word.
__device__ __forceinline__ uint32_t popc_rank(const uint64_t* __restrict__ row, const uint16_t* __restrict__ rk,
                                              int32_t ws, int32_t a, int32_t e)
{
    const int32_t wa = a >> 6, we = e >> 6;
    const uint64_t first = __ldg(row + wa * ws);
    const uint64_t last = __ldg(row + we * ws);
    const uint32_t ra = __ldg(rk + wa * ws), rb = __ldg(rk + we * ws);
    return rb - ra + (uint32_t)__popcll(last & (~0ull >> (63 - (e & 63)))) -
           (uint32_t)__popcll(first & ~(~0ull << (a & 63)));
}

// occupied bits of [a, e] when it lies within two consecutive words
__device__ __forceinline__ uint32_t popc_short(const uint64_t* __restrict__ row, int32_t ws, int32_t a, int32_t e)
{
    const int32_t wa = a >> 6, we = e >> 6;
    const uint64_t first = __ldg(row + wa * ws);
    const uint64_t last = __ldg(row + we * ws);
    uint64_t mlo = ~0ull << (a & 63);
    const uint64_t mhi = ~0ull >> (63 - (e & 63));
    const bool one = wa == we;
    mlo = one ? (mlo & mhi) : mlo;
    return __popcll(first & mlo) + __popcll(last & (one ? 0ull : mhi));
}

// Row counting modes of a box (BoxPrep::rank).
enum { kRowWalk = 0, kRowRank = 1, kRowShort = 2 };

// algorithmic bytes of one counted row [a, e]: every 16-byte chunk the
// interval touches; through the rank table, the end words' chunks and two
// 2-byte rank entries
template <int kMode>
__device__ __forceinline__ uint32_t row_bytes(int32_t a, int32_t e)
{
    const int32_t ca = a >> 7, ce = e >> 7;
    return kMode == kRowRank ? (ca == ce ? 16u : 32u) + 4u : (uint32_t)(ce - ca + 1) * 16u;
}

// occupied bits of [a, e] by the box's row counting mode
template <int kMode>
__device__ __forceinline__ uint32_t popc_mode(const uint64_t* __restrict__ row, const uint16_t* __restrict__ rk,
                                              int32_t ws, int32_t a, int32_t e)
{
    if constexpr (kMode == kRowRank) return popc_rank(row, rk, ws, a, e);
    else if constexpr (kMode == kRowShort) return popc_short(row, ws, a, e);
    else return popc_range(row, ws, a, e);
}

// One pass of a lane over its rows r0..r1 of a tile of a box whose three
// slabs all step by DDA: each of the six bounds is a 32.32 fixed-point value
// whose integer part is the quotient, so a bound costs one 64-bit add per
// row.  kMode: how a row's occupied bits are counted; kInterior: the tile's
// rows and x-intervals all lie in the lattice (no clamps); kProf: algorithmic
// bytes and rows are added up.
template <int kMode, bool kInterior, bool kProf>
__device__ __forceinline__ void dda_rows(int64_t (&Al)[3], int64_t (&Ah)[3], const int64_t (&Bs)[3],
                                         const uint64_t* __restrict__ rowp, const uint16_t* __restrict__ rkp,
                                         int64_t rstride, int32_t r0, int32_t r1, int32_t k, int32_t wk, int32_t kend,
                                         bool jvalid, bool jin, int32_t i0, int32_t span, int32_t N,
                                         uint32_t& empty, uint32_t& inbox, uint32_t& my_bytes, uint32_t& my_rows,
                                         uint32_t& my_rank, uint32_t& my_dom)
{
    const int32_t spanl = kInterior ? (jvalid ? span : -1) : span;
#pragma unroll kCountUnroll
    for (int r = r0; r <= r1; ++r, k += wk, rowp += rstride, rkp += rstride) {
        const int32_t lo = max(max((int32_t)(Al[0] >> 32), (int32_t)(Al[1] >> 32)), max((int32_t)(Al[2] >> 32), 0));
        const int32_t hi = min(min((int32_t)(Ah[0] >> 32), (int32_t)(Ah[1] >> 32)), min((int32_t)(Ah[2] >> 32), spanl));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Al[a] += Bs[a];
            Ah[a] += Bs[a];
        }
        if (kInterior) {
            if (lo <= hi) {
                const int32_t a = i0 + lo, e = i0 + hi;
                const uint32_t len = (uint32_t)(hi - lo + 1);
                empty += len - popc_mode<kMode>(rowp, rkp, N, a, e);
                inbox += len;
                my_dom += len;
                if (kProf) {
                    my_bytes += row_bytes<kMode>(a, e);
                    my_rows += 1;
                    my_rank += kMode == kRowRank ? 1u : 0u;
                }
            }
        } else if (jvalid && k < kend && lo <= hi) {
            const uint32_t len = (uint32_t)(hi - lo + 1);
            uint32_t occ = 0;
            if (jin && (uint32_t)k < (uint32_t)N) {
                const int32_t a = max(i0 + lo, 0), e = min(i0 + hi, N - 1);
                if (a <= e) {
                    occ = popc_mode<kMode>(rowp, rkp, N, a, e);
                    my_dom += (uint32_t)(e - a + 1);
                    if (kProf) my_bytes += row_bytes<kMode>(a, e);
                }
            }
            empty += len - occ;
            inbox += len;
            if (kProf) {
                my_rows += 1;
                my_rank += kMode == kRowRank ? 1u : 0u;
            }
        }
    }
}

// kProf: the launch adds up its algorithmic bytes, rows and rank rows into
// acc[0], acc[1], acc[3]; every launch adds its in-domain points into *dom.
// kMinB: resident blocks per SM the register budget aims at.
template <bool kProf, int kMinB>
__global__ void __launch_bounds__(256, kMinB) k_count(const BoxPrep* __restrict__ prep,
                                               const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ d_K,
                                               unsigned long long* __restrict__ counts,
                                               unsigned long long* __restrict__ points,
                                               unsigned long long* __restrict__ acc,
                                               unsigned long long* __restrict__ dom,
                                               const int32_t* __restrict__ perm)
{
    uint32_t my_bytes = 0, my_rows = 0, my_rank = 0, my_dom = 0;
    const int lane = threadIdx.x & 31;
    const int32_t K = *d_K;
    const int64_t total = off[K];
    unsigned long long* next = reinterpret_cast<unsigned long long*>(const_cast<int64_t*>(off + K + 1));
    // warps take runs of kGrab consecutive tiles from a global counter; within a
    // run the box and the tile coordinates advance incrementally
    // b: position in the launch's order; bi: the box there (perm[b], or b)
    int64_t c = 0, c_end = 0, box_end = 0;
    int32_t b = 0, bi = 0, tj = 0, tk = 0;
    for (;;) {
        if (c == c_end) {
            unsigned long long g = 0;
            if (lane == 0) g = atomicAdd(next, (unsigned long long)kGrab);
            c = (int64_t)__shfl_sync(0xffffffffu, g, 0);
            if (c >= total) break;
            c_end = min(c + (int64_t)kGrab, total);
            // the last box b with off[b] <= c: a 32-way search, one probe per lane
            int32_t lo = 0, hi = K;   // off[lo] <= c < off[hi]
            while (hi - lo > 1) {
                const int32_t st = (hi - lo + 31) >> 5;
                const int32_t idx = lo + lane * st;
                const unsigned m = __ballot_sync(0xffffffffu, idx < hi && off[idx] <= c);
                lo += (31 - __clz(m)) * st;
                hi = min(hi, lo + st);
            }
            b = lo;
            bi = perm ? perm[b] : b;
            box_end = off[b + 1];
            const int32_t u = (int32_t)(c - off[b]);
            const int32_t ntj0 = prep[bi].ntj;
            tk = u / ntj0;
            tj = u - tk * ntj0;
        } else if (c >= box_end) {
            ++b;
            while (off[b + 1] <= c) ++b;   // skip boxes without tiles
            bi = perm ? perm[b] : b;
            box_end = off[b + 1];
            tj = tk = 0;
        }
        const BoxPrep& p = prep[bi];
        {
            // skip a tile whose rectangle misses the box's shadow on (j, k)
            const int32_t lw = p.lwj, hk = (32 >> lw) * p.tk;
            const float hj = 0.5f * (float)((1 << lw) - 1), hkf = 0.5f * (float)(hk - 1);
            const float jc = (float)(p.j0 + (tj << lw)) + hj, kc = (float)(p.k0 + tk * hk) + hkf;
            bool out = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float u = p.sat_nu[a][0], v = p.sat_nu[a][1];
                const float cc = u * jc + v * kc, e = fabsf(u) * hj + fabsf(v) * hkf;
                out |= cc + e < p.sat_lo[a] || cc - e > p.sat_hi[a];
            }
            if (out) {
                if (++tj == p.ntj) {
                    tj = 0;
                    ++tk;
                }
                ++c;
                continue;
            }
        }
        const uint64_t* __restrict__ words = p.words;
        const int32_t N = p.latN, W = p.latW;
        const int32_t mode = p.mode;
        const int32_t lwj = p.lwj;
        const int32_t wk = 32 >> lwj;
        const int32_t jl = (tj << lwj) + (lane & ((1 << lwj) - 1));
        const int32_t j = p.j0 + jl;
        const bool jvalid = jl < p.nj;
        const int32_t tkr = p.tk;
        const int32_t kb = p.k0 + tk * (wk * tkr) + (lane >> lwj);   // this lane's first row
        const int32_t kend = p.k0 + p.nk;
        // rows r0..r1 (warp-uniform) of the tile's tkr are visited
        int32_t r0 = 0, r1 = tkr - 1;
        if ((mode & 0xff) == 0x15) {
            // each lane's column meets the shadow in a k-range (the separating
            // bands solved for k); the warp visits the union of its lanes'
            // ranges, which skips the empty ends of a tile the shadow crosses
            const float jr = (float)(j - p.j0);
            float klo = -1e30f, khi = 1e30f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                klo = fmaxf(klo, fmaf(p.kc_s[a], jr, p.kc_lo[a]));
                khi = fminf(khi, fmaf(p.kc_s[a], jr, p.kc_hi[a]));
            }
            int32_t rl = tkr, rh = -1;
            if (jvalid && klo <= khi) {
                const int32_t lwk = 5 - lwj;   // wk = 2^lwk
                const int32_t kbr = kb - p.k0;
                const int32_t kl = (int32_t)floorf(fmaxf(klo, -1e9f));
                const int32_t kh = (int32_t)ceilf(fminf(khi, 1e9f));
                rl = max(0, -((kbr - kl) >> lwk));    // first r with kb + r wk >= kl
                rh = min(tkr - 1, (kh - kbr) >> lwk);  // last r with kb + r wk <= kh
                if (rl > rh) {
                    rl = tkr;
                    rh = -1;
                }
            }
            r0 = __reduce_min_sync(0xffffffffu, rl);
            r1 = __reduce_max_sync(0xffffffffu, rh);
            if (r0 > r1) {
                if (++tj == p.ntj) {
                    tj = 0;
                    ++tk;
                }
                ++c;
                continue;
            }
        }
        const int32_t kb0 = kb + r0 * wk;   // the first row this lane visits
        const int32_t i0 = p.i0, span = p.span;
        // Kind-1 slabs carry exact quotient bounds relative to i0 in 32 bits,
        // saturated at +-2^30: a bound that far out moves less than 2^29 within a
        // tile, so it stays outside [0, span].  Kind 0 (n_a0 = 0) and kind 2
        // (|n_a0| < 32) slabs are evaluated from scratch on each row.
        int32_t qa[3], qb[3], ra[3], rb[3], dd[3], rs[3], qs[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            qa[a] = qb[a] = ra[a] = rb[a] = rs[a] = qs[a] = 0;
            dd[a] = 1;
            if (((mode >> (2 * a)) & 3) == 1) {
                dd[a] = p.dd[a];
                rs[a] = p.rstep[a];
                qs[a] = p.qstep[a];
                const int64_t cc = (int64_t)p.n[3 * a + 1] * j + (int64_t)p.n[3 * a + 2] * kb0;
                const int64_t xlo = p.n[3 * a] > 0 ? p.Lq[a] - cc : cc - p.Hq[a];
                const int64_t xhi = p.n[3 * a] > 0 ? p.Hq[a] - cc : cc - p.Lq[a];
                int64_t wlo, whi;
                floordiv_rcp(xlo + dd[a] - 1, dd[a], p.fmul[a], wlo, ra[a]);   // ceil(xlo / dd)
                floordiv_rcp(xhi, dd[a], p.fmul[a], whi, rb[a]);               // floor(xhi / dd)
                const int64_t lim = int64_t(1) << 30;
                qa[a] = (int32_t)min(max(wlo - i0, -lim), lim);
                qb[a] = (int32_t)min(max(whi - i0, -lim), lim);
            }
        }
        uint32_t empty = 0, inbox = 0;
        const bool jin = j >= 0 && j < N;
        if ((mode & 0xff) == 0x15) {
            // all three slabs step by DDA (any rotated box): the 32.32
            // fixed-point bounds, seeded exactly at the first visited row
            int64_t Al[3], Ah[3], Bs[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const uint64_t M = p.fmul[a];
                Al[a] = (int64_t)qa[a] * 4294967296LL + fixed_frac(ra[a], M) + kFixBias;
                Ah[a] = (int64_t)qb[a] * 4294967296LL + fixed_frac(rb[a], M) + kFixBias;
                Bs[a] = p.fstep[a];
            }
            // count copies interleave the rows of a slice by column: word w of
            // row (slice k, column j) at (k W + w) N + j
            const int64_t roff = (int64_t)kb0 * W * N + j;
            const int64_t rstride = (int64_t)wk * W * N;
            // an interior box's full-height tile: every row is in the lattice
            // and so is every x-interval; an idle lane gets an empty range
            const bool interior = (mode & 0x100) && (tk + 1) * wk * tkr <= p.nk;
#define OBB_DDA_ROWS(MODE, INTERIOR)                                                                             \
    dda_rows<MODE, INTERIOR, kProf>(Al, Ah, Bs, words + roff, p.ranks + roff, rstride, r0, r1, kb0, wk, kend, jvalid, \
                                    jin, i0, span, N, empty, inbox, my_bytes, my_rows, my_rank, my_dom)
            if (p.rank == kRowRank) {
                if (interior) OBB_DDA_ROWS(kRowRank, true);
                else OBB_DDA_ROWS(kRowRank, false);
            } else if (p.rank == kRowShort) {
                if (interior) OBB_DDA_ROWS(kRowShort, true);
                else OBB_DDA_ROWS(kRowShort, false);
            } else {
                if (interior) OBB_DDA_ROWS(kRowWalk, true);
                else OBB_DDA_ROWS(kRowWalk, false);
            }
#undef OBB_DDA_ROWS
        } else
#pragma unroll kCountUnroll
        for (int r = 0; r < tkr; ++r) {
            const int32_t k = kb + r * wk;
            int32_t lo = 0, hi = span;
            bool ok = jvalid && k < kend;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int kind = (mode >> (2 * a)) & 3;
                if (kind == 1) {
                    lo = max(lo, qa[a]);
                    hi = min(hi, qb[a]);
                    qa[a] += qs[a];
                    ra[a] += rs[a];
                    if (ra[a] >= dd[a]) {
                        ra[a] -= dd[a];
                        qa[a] += 1;
                    }
                    qb[a] += qs[a];
                    rb[a] += rs[a];
                    if (rb[a] >= dd[a]) {
                        rb[a] -= dd[a];
                        qb[a] += 1;
                    }
                } else if (ok && lo <= hi) {
                    const int64_t cc = (int64_t)p.n[3 * a + 1] * j + (int64_t)p.n[3 * a + 2] * k;
                    if (kind == 0) {
                        ok = cc >= p.Lq[a] && cc <= p.Hq[a];
                    } else {
                        int32_t l2 = i0 + lo, h2 = i0 + hi;
                        clip_slab_rcp(p.n[3 * a], p.fmul[a], cc, p.Lq[a], p.Hq[a], l2, h2);
                        lo = l2 - i0;
                        hi = h2 - i0;
                    }
                }
            }
            if (ok && lo <= hi) {
                const int32_t ia = i0 + lo, ie = i0 + hi;
                const uint32_t len = (uint32_t)(hi - lo + 1);
                uint32_t occ = 0;
                if (jin && k >= 0 && k < N) {
                    const int32_t a = max(ia, 0), e = min(ie, N - 1);
                    if (a <= e) {
                        const int64_t roff = (int64_t)k * W * N + j;
                        if (p.rank == kRowRank) {
                            occ = popc_rank(words + roff, p.ranks + roff, N, a, e);
                            if (kProf) my_bytes += row_bytes<kRowRank>(a, e);
                        } else {
                            occ = popc_range(words + roff, N, a, e);
                            if (kProf) my_bytes += row_bytes<kRowWalk>(a, e);
                        }
                        my_dom += (uint32_t)(e - a + 1);
                    }
                }
                empty += len - occ;
                inbox += len;
                if (kProf) {
                    my_rows += 1;
                    my_rank += p.rank == kRowRank ? 1u : 0u;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            empty += __shfl_xor_sync(0xffffffffu, empty, o);
            inbox += __shfl_xor_sync(0xffffffffu, inbox, o);
        }
        if (lane == 0) {
            if (empty) atomicAdd(&counts[bi], (unsigned long long)empty);
            if (points && inbox) atomicAdd(&points[bi], (unsigned long long)inbox);
        }
        if (++tj == p.ntj) {
            tj = 0;
            ++tk;
        }
        ++c;
    }
    // in-domain points of this launch (always), and with profiling its
    // algorithmic bytes, non-empty rows and rank rows: block sums, one atomic
    // each
    if (kProf || dom) {
        __shared__ unsigned long long sh[4];
        if (threadIdx.x < 4) sh[threadIdx.x] = 0;
        __syncthreads();
        unsigned long long v[4] = {my_bytes, my_rows, my_dom, my_rank};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (!kProf && i != 2) continue;
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
            if (lane == 0 && v[i]) atomicAdd(&sh[i], v[i]);
        }
        __syncthreads();
        if (kProf && threadIdx.x < 4 && threadIdx.x != 2 && acc && sh[threadIdx.x])
            atomicAdd(&acc[threadIdx.x], sh[threadIdx.x]);
        if (threadIdx.x == 2 && dom && sh[2]) atomicAdd(dom, sh[2]);
    }
}

// ---------------------------------------------------------------- report

__global__ void k_report(const LatticeFrame* __restrict__ f, const double* __restrict__ frames,
                         const obb_qbox* __restrict__ q, int32_t K, obb_box* __restrict__ out)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double* R = frames + 9 * (int64_t)k;
    const double s = 4294967296.0 / f->hmax;
    double c[3] = {0, 0, 0};
    obb_box o;
    for (int a = 0; a < 3; ++a) {
        double base = 0.0;
        for (int b = 0; b < 3; ++b) base += R[3 * a + b] * (f->lo[b] + 0.5 * f->h[b]);
        double lo = (double)q[k].b[2 * a] / s + base;
        double hi = (double)q[k].b[2 * a + 1] / s + base;
        double mid = 0.5 * (lo + hi);
        for (int b = 0; b < 3; ++b) c[b] += R[3 * a + b] * mid;
        o.half[a] = (float)(0.5 * (hi - lo));
    }
    for (int b = 0; b < 3; ++b) {
        o.c[b] = (float)c[b];
        o.axis0[b] = (float)R[b];
        o.axis1[b] = (float)R[3 + b];
    }
    out[k] = o;
}

__global__ void k_set_i32(int32_t* dst, int32_t v)
{
    *dst = v;
}

}  // namespace

obb_status set_device_int(obb_ctx* ctx, int32_t* d_dst, int32_t value)
{
    k_set_i32<<<1, 1, 0, ctx->stream>>>(d_dst, value);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

void launch_scan_i32(obb_ctx* ctx, const int32_t* in, int32_t* out, const int32_t* d_n)
{
    k_scan_i32<<<1, 1024, 0, ctx->stream>>>(in, out, d_n);
    note_launch(ctx);
}

void launch_box_report(obb_ctx* ctx, const obb_lattice* lat, const double* d_frames, const obb_qbox* d_q, int32_t K,
                       obb_box* d_out)
{
    if (K > 0) {
        k_report<<<(K + 31) / 32, 32, 0, ctx->stream>>>(lat->d_frame, d_frames, d_q, K, d_out);
        note_launch(ctx);
    }
}

obb_status quantize_boxes(obb_ctx* ctx, const obb_lattice* lat, const obb_box* d_boxes, int64_t K,
                          obb_qbox* d_out)
{
    if (K <= 0) return OBB_OK;
    k_quantize<<<(unsigned)((K + 31) / 32), 32, 0, ctx->stream>>>(d_boxes, K, lat->d_frame, d_out,
                                                                    ctx->d_err);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

// The counting kernel as a persistent grid (every resident block of every
// SM), in the register budget for the lattices' size: 5 blocks per SM for
// lattices of at least kOrderMinLatticeBytes (DRAM-resident: more warps to
// cover the loads), 4 below (L2-resident: more registers per thread).
template <bool kProf, int kMinB>
static void launch_count_v(obb_ctx* ctx, cudaStream_t s, const BoxPrep* prep, const int64_t* off, const int32_t* d_K,
                           uint64_t* counts, uint64_t* points, unsigned long long* acc, unsigned long long* dom,
                           const int32_t* perm)
{
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_count<kProf, kMinB>, 256, 0) != cudaSuccess ||
            nb < 1)
            nb = 1;
        blocks_per_sm = nb;
    }
    k_count<kProf, kMinB><<<blocks_per_sm * ctx->num_sms, 256, 0, s>>>(
        prep, off, d_K, reinterpret_cast<unsigned long long*>(counts), reinterpret_cast<unsigned long long*>(points),
        acc, dom, perm);
}

static void launch_count(obb_ctx* ctx, cudaStream_t s, bool prof, int64_t lattice_bytes, const BoxPrep* prep,
                         const int64_t* off, const int32_t* d_K, uint64_t* counts, uint64_t* points,
                         unsigned long long* acc, unsigned long long* dom, const int32_t* perm)
{
    constexpr int kLarge = OBB_COUNT_MINB, kSmall = OBB_COUNT_MINB_SMALL;
    const bool large = lattice_bytes >= kOrderMinLatticeBytes;
    if (prof) {
        if (large) launch_count_v<true, kLarge>(ctx, s, prep, off, d_K, counts, points, acc, dom, perm);
        else launch_count_v<true, kSmall>(ctx, s, prep, off, d_K, counts, points, acc, dom, perm);
    } else {
        if (large) launch_count_v<false, kLarge>(ctx, s, prep, off, d_K, counts, points, acc, dom, perm);
        else launch_count_v<false, kSmall>(ctx, s, prep, off, d_K, counts, points, acc, dom, perm);
    }
}

obb_status count_boxes(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* d_boxes, const int32_t* d_K,
                       int64_t K_cap, uint64_t* d_counts, uint64_t* d_points)
{
    if (ctx->count_defer) {
        // a batched step counts every layer's requests together (count_flush)
        ctx->count_defer->push_back(CountReq{lat, d_boxes, d_K, K_cap, d_counts, d_points});
        return OBB_OK;
    }
    return count_boxes_multi(ctx, lat->d_ref, 1, nullptr, d_boxes, d_K, K_cap, d_counts, d_points,
                             (int64_t)lat->n_words * 8);
}

obb_status count_boxes_multi(obb_ctx* ctx, const LatRef* d_lats, int32_t n_lats, const int32_t* d_lat_of_box,
                             const obb_qbox* d_boxes, const int32_t* d_K, int64_t K_cap, uint64_t* d_counts,
                             uint64_t* d_points, int64_t lattice_bytes)
{
    cudaStream_t s = ctx->stream;
    if (K_cap <= 0) return OBB_OK;
    if (K_cap > (int64_t(1) << 30)) return fail(ctx, OBB_ERR_RANGE, "too many boxes in one call");
    BoxPrep* prep;
    int64_t *tiles, *off;
    unsigned int* ticket = ctx->d_ticket;
    uint32_t* bucket = nullptr;
    int32_t* perm = nullptr;
    int64_t *ptiles = nullptr, *bsum = nullptr;
    if (ctx->count_scratch) {
        // fixed scratch of a step being captured into a graph: its addresses must not move
        const CountScratch& cs = *ctx->count_scratch;
        if (K_cap > cs.cap) return fail(ctx, OBB_ERR_STATE, "count scratch of a captured step too small");
        prep = cs.prep;
        tiles = cs.tiles;
        off = cs.tiles + cs.cap;
        bsum = cs.bsum;
    } else {
        const int64_t nb = K_cap / kScanBlock + 1;
        OBB_CK(ctx, ctx->prep.reserve(sizeof(BoxPrep) * K_cap, s));
        OBB_CK(ctx, ctx->chunk_off.reserve(sizeof(int64_t) * (2 * K_cap + 2 + nb), s));
        prep = ctx->prep.as<BoxPrep>();
        tiles = ctx->chunk_off.as<int64_t>();
        off = tiles + K_cap;
        bsum = off + K_cap + 2;
        if (ctx->count_order && K_cap >= kOrderMinBoxes && lattice_bytes >= kOrderMinLatticeBytes) {
            // large batches on lattices too large for L2 are counted in
            // spatial order (boxes of every size over one region together, so
            // the region's lattice words are reused from L2)
            OBB_CK(ctx, ctx->order.reserve((2 * sizeof(int32_t) + sizeof(int64_t)) * K_cap, s));
            ptiles = reinterpret_cast<int64_t*>(ctx->order.as<char>());
            bucket = reinterpret_cast<uint32_t*>(ptiles + K_cap);
            perm = reinterpret_cast<int32_t*>(bucket + K_cap);
            OBB_CK(ctx, cudaMemsetAsync(ctx->d_order_hist, 0, kOrderBuckets * sizeof(unsigned int), s));
        }
    }
    // the preparation kernel also zeroes counts and points (accumulated with atomics)
    k_prep<<<(unsigned)((K_cap + kPrepThreads - 1) / kPrepThreads), kPrepThreads, 0, s>>>(
        d_boxes, d_K, d_lats, n_lats, d_lat_of_box, ctx->tile_k, ctx->count_axis, ctx->count_rank, prep, tiles, off,
        reinterpret_cast<unsigned long long*>(d_counts), reinterpret_cast<unsigned long long*>(d_points), ticket,
        bucket, bucket ? ctx->d_order_hist : nullptr, 0, ctx->d_err);
    note_launch(ctx);
    // tile offsets: an exclusive scan of the tile counts in counting order
    // (the spatial order's permuted copy, else the boxes' own order)
    const int64_t* scan_in = tiles;
    if (perm) {
        k_order_scatter<<<(unsigned)((K_cap + 255) / 256), 256, 0, s>>>(bucket, tiles, d_K, ctx->d_order_hist, perm,
                                                                      ptiles);
        note_launch(ctx);
        scan_in = ptiles;
    }
    const unsigned nsb = (unsigned)(K_cap / kScanBlock + 1);
    k_tile_sums<<<nsb, 256, 0, s>>>(scan_in, d_K, bsum);
    k_tile_offsets<<<nsb, 256, 0, s>>>(scan_in, bsum, d_K, off);
    note_launch(ctx, 2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->prof) {
        OBB_CK(ctx, cudaEventCreate(&e0));
        OBB_CK(ctx, cudaEventCreate(&e1));
        OBB_CK(ctx, cudaEventRecord(e0, s));
    }
    launch_count(ctx, s, ctx->prof == 1, lattice_bytes, prep, off, d_K, d_counts, d_points,
                 ctx->prof == 1 ? ctx->d_prof : nullptr, ctx->d_prof + 2, perm);
    note_launch(ctx);
    if (ctx->prof) {
        OBB_CK(ctx, cudaEventRecord(e1, s));
        ctx->prof_ev.emplace_back(e0, e1);
    }
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

obb_status count_flush(obb_ctx* ctx, const std::vector<CountReq>& reqs, DevBuf& tables, DevBuf& scratch)
{
    cudaStream_t s = ctx->stream;
    const int32_t n = (int32_t)reqs.size();
    if (n == 0) return OBB_OK;
    if (n > (1 << 20)) return fail(ctx, OBB_ERR_RANGE, "too many counting requests in one batch");
    // lattice table and request table (host), uploaded into `tables`
    std::vector<const obb_lattice*> lats;
    std::vector<BatchReq> hreq(n);
    int64_t cap = 0, lattice_bytes = 0;
    for (int32_t r = 0; r < n; ++r) {
        const CountReq& q = reqs[r];
        int32_t li = 0;
        while (li < (int32_t)lats.size() && lats[li] != q.lat) ++li;
        if (li == (int32_t)lats.size()) {
            lats.push_back(q.lat);
            lattice_bytes += (int64_t)q.lat->n_words * 8;
        }
        hreq[r] = BatchReq{q.boxes, q.d_K, q.counts, q.points, q.K_cap, li, 0};
        cap += q.K_cap;
    }
    if (cap > (int64_t(1) << 30)) return fail(ctx, OBB_ERR_RANGE, "too many boxes in one batch");
    const size_t req_bytes = (sizeof(BatchReq) * n + 255) / 256 * 256;
    const size_t lat_bytes = (sizeof(LatRef) * lats.size() + 255) / 256 * 256;
    OBB_CK(ctx, tables.reserve(req_bytes + lat_bytes, s));
    BatchReq* d_req = tables.as<BatchReq>();
    LatRef* d_lat = reinterpret_cast<LatRef*>(tables.as<char>() + req_bytes);
    std::vector<LatRef> hlat(lats.size());
    for (size_t i = 0; i < lats.size(); ++i) hlat[i] = lats[i]->ref;
    // pinned staging keeps the copies asynchronous (the tables are small)
    void* h = nullptr;
    OBB_CK(ctx, cudaMallocHost(&h, req_bytes + lat_bytes));
    memcpy(h, hreq.data(), sizeof(BatchReq) * n);
    memcpy(static_cast<char*>(h) + req_bytes, hlat.data(), sizeof(LatRef) * hlat.size());
    cudaError_t e = cudaMemcpyAsync(d_req, h, req_bytes + lat_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the staging is freed below
    cudaFreeHost(h);
    OBB_CK(ctx, e);
    // combined scratch: offsets [n + 1], total, boxes [cap], lattice of box [cap], counts and points [cap]
    const size_t off_b = (sizeof(int64_t) * (n + 1) + 255) / 256 * 256;
    const size_t box_b = (sizeof(obb_qbox) * cap + 255) / 256 * 256;
    const size_t li_b = (sizeof(int32_t) * cap + 255) / 256 * 256;
    const size_t cnt_b = (sizeof(uint64_t) * cap + 255) / 256 * 256;
    OBB_CK(ctx, scratch.reserve(off_b + 256 + box_b + li_b + 2 * cnt_b, s));
    char* b = scratch.as<char>();
    int64_t* off = reinterpret_cast<int64_t*>(b);
    int32_t* d_total = reinterpret_cast<int32_t*>(b + off_b);
    obb_qbox* boxes = reinterpret_cast<obb_qbox*>(b + off_b + 256);
    int32_t* lat_of_box = reinterpret_cast<int32_t*>(b + off_b + 256 + box_b);
    uint64_t* counts = reinterpret_cast<uint64_t*>(b + off_b + 256 + box_b + li_b);
    uint64_t* points = counts + cnt_b / sizeof(uint64_t);
    k_batch_offsets<<<1, 1024, 0, s>>>(d_req, n, off, d_total);
    const unsigned gb = (unsigned)std::min<int64_t>((cap + 255) / 256, 4 * (int64_t)ctx->num_sms);
    k_batch_gather<<<std::max(gb, 1u), 256, 0, s>>>(d_req, n, off, boxes, lat_of_box);
    note_launch(ctx, 2);
    OBB_TRY(count_boxes_multi(ctx, d_lat, (int32_t)lats.size(), lat_of_box, boxes, d_total, cap, counts, points,
                              lattice_bytes));
    k_batch_scatter<<<std::max(gb, 1u), 256, 0, s>>>(d_req, n, off, counts, points);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}

}  // namespace obbv

// ---------------------------------------------------------------------------
// Outer volume without device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// real-time collision or physics loop that works inside a fixed memory
// budget, or a host framework that owns the whole device memory pool and
// forbids allocations outside it.  This variant of the counting path takes
// its per-box scratch (count preparation, chunk counts and offsets, the box
// count) from one file-scope device array of fixed size instead of the
// context's growable buffers.  Every GPU that loads the library holds the
// array until the process exits.
// ---------------------------------------------------------------------------
namespace obbv {
namespace {

constexpr int64_t kNoAllocMaxBoxes = 4096;   // OBB_NOALLOC_MAX_BOXES in obbvar.h
constexpr size_t kNoAllocPrepBytes = sizeof(BoxPrep) * kNoAllocMaxBoxes;
constexpr size_t kNoAllocChunkBytes = sizeof(int64_t) * kNoAllocMaxBoxes;
constexpr size_t kNoAllocOffBytes = sizeof(int64_t) * (kNoAllocMaxBoxes + 2);
constexpr size_t kNoAllocOffsetChunks = (kNoAllocPrepBytes + 255) / 256 * 256;
constexpr size_t kNoAllocOffsetOff = kNoAllocOffsetChunks + (kNoAllocChunkBytes + 255) / 256 * 256;
constexpr size_t kNoAllocOffsetK = kNoAllocOffsetOff + (kNoAllocOffBytes + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocOffsetK + 256;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the array on `device` (looked up once per device, with
// that device current).  In host code the array's name is only a stand-in.
obb_status noalloc_scratch(obb_ctx* ctx, unsigned char** out)
{
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices) return fail(ctx, OBB_ERR_ARG, "device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[ctx->device]) {
        int prev = -1;
        OBB_CK(ctx, cudaGetDevice(&prev));
        if (prev != ctx->device) OBB_CK(ctx, cudaSetDevice(ctx->device));
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (prev != ctx->device) cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[ctx->device] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_ptr[ctx->device];
    return OBB_OK;
}

}  // namespace
}  // namespace obbv

extern "C" obb_status obb_outer_volume_q_noalloc(obb_ctx* ctx, const obb_lattice* lat, const obb_qbox* d_boxes,
                                                 int64_t K, uint64_t* d_counts, uint64_t* d_points)
{
    using namespace obbv;
    if (!ctx || !lat) return fail(ctx, OBB_ERR_ARG, "null argument");
    if (lat->ctx != ctx) return fail(ctx, OBB_ERR_STATE, "lattice belongs to another context");
    if (K < 0) return fail(ctx, OBB_ERR_ARG, "negative K");
    if (K > kNoAllocMaxBoxes)
        return fail(ctx, OBB_ERR_RANGE,
                    "obb_outer_volume_q_noalloc takes at most " + std::to_string(kNoAllocMaxBoxes) +
                        " boxes per call (got " + std::to_string(K) + "); split the batch or use obb_outer_volume_q");
    if (K == 0) return OBB_OK;
    if (!d_boxes || !d_counts) return fail(ctx, OBB_ERR_ARG, "null argument");
    unsigned char* base = nullptr;
    OBB_TRY(noalloc_scratch(ctx, &base));
    BoxPrep* prep = reinterpret_cast<BoxPrep*>(base);
    int64_t* chunks = reinterpret_cast<int64_t*>(base + kNoAllocOffsetChunks);
    int64_t* off = reinterpret_cast<int64_t*>(base + kNoAllocOffsetOff);
    int32_t* dK = reinterpret_cast<int32_t*>(base + kNoAllocOffsetK);
    cudaStream_t s = ctx->stream;
    // the last 128 bytes of the count's slot hold the preparation blocks' ticket
    // (zero at load; every launch leaves it at zero again)
    unsigned int* ticket = reinterpret_cast<unsigned int*>(base + kNoAllocOffsetK + 128);
    k_set_i32<<<1, 1, 0, s>>>(dK, (int32_t)K);
    note_launch(ctx);
    // the preparation kernel also zeroes counts and points (accumulated with atomics)
    k_prep<<<(unsigned)((K + kPrepThreads - 1) / kPrepThreads), kPrepThreads, 0, s>>>(
        d_boxes, dK, lat->d_ref, 1, nullptr, ctx->tile_k, ctx->count_axis, ctx->count_rank, prep, chunks, off,
        reinterpret_cast<unsigned long long*>(d_counts), reinterpret_cast<unsigned long long*>(d_points), ticket,
        nullptr, nullptr, 1, ctx->d_err);
    note_launch(ctx);
    launch_count(ctx, s, false, (int64_t)lat->n_words * 8, prep, off, dK, d_counts, d_points, nullptr, nullptr,
                 nullptr);
    note_launch(ctx);
    OBB_CK(ctx, cudaGetLastError());
    return OBB_OK;
}
