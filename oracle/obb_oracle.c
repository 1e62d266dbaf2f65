/*
 * CPU oracle for the outer-volume / Lloyd path of "Variational Hierarchical
 * Directed Bounding Box Construction for Solid Mesh Models" (arXiv 2203.10521).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement that the CUDA path is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header or constant table with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -shared -fPIC (see oracle/build.py).
 * -ffp-contract=off matters: the fixed-point snap and the box quantisation are
 * defined as sequences of correctly rounded IEEE-754 double operations.
 *
 * Readings of the paper used here (the paper's own error method is ray
 * integration on a rasteriser, Sec. 4.1; the lattice count below is the exact
 * discretisation of Eq. 4 that replaces it):
 *   - lattice: N points per axis, cell centred over the vertex AABB,
 *     x_b(i) = lo_b + (i + 1/2) h_b, h_b = (hi_b - lo_b) / N;
 *   - fixed point: U_b = rint(((x_b - lo_b) / h_b - 1/2) * 2^S), S = 8, so
 *     lattice point i sits at U = 2^S i;
 *   - solid Omega(X) (Sec. 3): point inside iff the +x ray from it crosses the
 *     surface an odd number of times; crossings of a column are decided with
 *     Simulation of Simplicity on the (y, z) projection, perturbing the query
 *     point by (eps, eps^2); a crossing at x* counts for point x iff x* <= x;
 *   - outer volume of one box, Eq. 4: number of lattice points of Z^3 inside
 *     the closed box and outside the solid (points outside [0,N)^3 are
 *     outside the solid);
 *   - box: frame R (rows = axes), quantised normals
 *     n_ab = rint(2^Q R_ab h_b / h_max), Q = 24, and integer slab bounds
 *     lo_a <= n_a . U <= hi_a (Sec. 4.2.1: the shape follows from the
 *     enclosure once centre and axes are fixed; here it is the tight slab);
 *   - Lloyd partition step (Sec. 4.2.1, Eq. 11-13): exact integer gains,
 *     locally dominant matching of proposals;
 *   - refit: area-weighted covariance, cyclic Jacobi in FP64.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_S 8
#define ORC_Q 24

/* ------------------------------------------------------------------------- */
/* Lattice frame and fixed-point snap                                        */
/* ------------------------------------------------------------------------- */

/* lo_b, h_b of the N^3 cell-centred lattice over the vertex AABB. */
void orc_lattice_frame(const float* V, int64_t nv, int32_t N, double* lo, double* h)
{
    for (int b = 0; b < 3; ++b) {
        float mn = V[b], mx = V[b];
        for (int64_t v = 1; v < nv; ++v) {
            float x = V[3 * v + b];
            if (x < mn) mn = x;
            if (x > mx) mx = x;
        }
        lo[b] = (double)mn;
        h[b] = ((double)mx - (double)mn) / (double)N;
    }
}

/* U_b = rint(((x_b - lo_b) / h_b - 1/2) * 2^S), evaluated in this order. */
void orc_snap(const float* V, int64_t nv, const double* lo, const double* h, int32_t* U)
{
    for (int64_t v = 0; v < nv; ++v)
        for (int b = 0; b < 3; ++b) {
            double d = (double)V[3 * v + b] - lo[b];
            double q = d / h[b];
            q = q - 0.5;
            q = q * 256.0;
            U[3 * v + b] = (int32_t)nearbyint(q);
        }
}

/* ------------------------------------------------------------------------- */
/* Solid occupancy by crossing parity, one lattice point at a time           */
/* ------------------------------------------------------------------------- */

/* orient2d of (a, b, p) in the (y, z) plane, exact in int64. */
static int64_t orient_yz(int64_t ay, int64_t az, int64_t by, int64_t bz, int64_t py, int64_t pz)
{
    return (by - ay) * (pz - az) - (bz - az) * (py - ay);
}

/* Sign of orient2d(a, b, p') with p' = p + (eps, eps^2), eps -> 0+. */
static int sos_sign(int64_t ay, int64_t az, int64_t by, int64_t bz, int64_t py, int64_t pz)
{
    int64_t o = orient_yz(ay, az, by, bz, py, pz);
    if (o > 0) return 1;
    if (o < 0) return -1;
    /* d/d eps of orient = -(bz - az); d/d eps^2 = (by - ay) */
    if (bz != az) return (bz - az) > 0 ? -1 : 1;
    if (by != ay) return (by - ay) > 0 ? 1 : -1;
    return 0;
}

/* Does the perturbed column point (py, pz) lie in the (y,z) projection of the
 * triangle?  If so, return 1 and the crossing as the exact fraction num/den
 * (den > 0) of the triangle's plane x at (py, pz). */
static int column_crossing(const int32_t* A, const int32_t* B, const int32_t* C,
                           int64_t py, int64_t pz, int64_t* num, int64_t* den)
{
    int sa = sos_sign(B[1], B[2], C[1], C[2], py, pz);
    int sb = sos_sign(C[1], C[2], A[1], A[2], py, pz);
    int sc = sos_sign(A[1], A[2], B[1], B[2], py, pz);
    if (sa == 0 || sb == 0 || sc == 0) return 0;
    if (!(sa == sb && sb == sc)) return 0;
    /* barycentric weights at the unperturbed point */
    int64_t wa = orient_yz(B[1], B[2], C[1], C[2], py, pz);
    int64_t wb = orient_yz(C[1], C[2], A[1], A[2], py, pz);
    int64_t wc = orient_yz(A[1], A[2], B[1], B[2], py, pz);
    int64_t d = wa + wb + wc;
    if (d == 0) return 0; /* cannot happen when all three SoS signs agree */
    int64_t n = wa * (int64_t)A[0] + wb * (int64_t)B[0] + wc * (int64_t)C[0];
    if (d < 0) { d = -d; n = -n; }
    *num = n;
    *den = d;
    return 1;
}

/* Threads of the loops below that run over independent columns or slices
 * (OpenMP when built with it; 1 by default, so the oracle is single threaded
 * unless a caller asks otherwise).  No result depends on the thread count:
 * every column and every point is computed on its own, and counts are
 * integer sums. */
void orc_set_threads(int32_t n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int32_t orc_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORC_BLOCK 32

static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : (x > y);
}

/*
 * Occupancy of the requested columns.  occ is N*N*N bytes indexed
 * ((k*N)+j)*N+i; colmask is N*N bytes indexed k*N+j and is set to 1 for
 * every column written.  For each point, the number of crossings with
 * x* <= 2^S i is counted over all triangles; the point is inside iff odd.
 * The columns are taken in blocks of 32 x 32; for each block only the
 * triangles whose (y, z) bounding box meets the block's rectangle are
 * examined (a triangle outside it cannot contain any of its column points).
 */
void orc_occupancy_columns(const int32_t* U, const int32_t* F, int64_t nt, int32_t N,
                           const int32_t* cols, int64_t ncols, uint8_t* occ, uint8_t* colmask)
{
    if (ncols <= 0) return;
    /* order the columns by block: key = block id * 2^32 + column index */
    const int64_t nbj = (N + ORC_BLOCK - 1) / ORC_BLOCK;
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncols);
    for (int64_t c = 0; c < ncols; ++c) {
        const int64_t blk = (int64_t)(cols[2 * c + 1] / ORC_BLOCK) * nbj + cols[2 * c] / ORC_BLOCK;
        key[c] = (blk << 32) | c;
    }
    qsort(key, (size_t)ncols, sizeof(int64_t), cmp_i64);
    int64_t nblk = 0;
    int64_t* bstart = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncols + 1));
    for (int64_t c = 0; c < ncols; ++c)
        if (c == 0 || (key[c] >> 32) != (key[c - 1] >> 32)) bstart[nblk++] = c;
    bstart[nblk] = ncols;
    int64_t b;
#pragma omp parallel for schedule(dynamic, 1)
    for (b = 0; b < nblk; ++b) {
        int64_t* tl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
        int64_t* nums = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
        int64_t* dens = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
        /* the block's column rectangle in fixed point */
        int64_t y0 = INT64_MAX, y1 = INT64_MIN, z0 = INT64_MAX, z1 = INT64_MIN;
        for (int64_t q = bstart[b]; q < bstart[b + 1]; ++q) {
            const int64_t c = key[q] & 0xffffffffLL;
            const int64_t py = (int64_t)cols[2 * c] << ORC_S, pz = (int64_t)cols[2 * c + 1] << ORC_S;
            if (py < y0) y0 = py;
            if (py > y1) y1 = py;
            if (pz < z0) z0 = pz;
            if (pz > z1) z1 = pz;
        }
        int64_t ntl = 0;
        for (int64_t t = 0; t < nt; ++t) {
            const int32_t* A = U + 3 * (int64_t)F[3 * t];
            const int32_t* B = U + 3 * (int64_t)F[3 * t + 1];
            const int32_t* C = U + 3 * (int64_t)F[3 * t + 2];
            int32_t ymin = A[1], ymax = A[1], zmin = A[2], zmax = A[2];
            if (B[1] < ymin) ymin = B[1];
            if (B[1] > ymax) ymax = B[1];
            if (C[1] < ymin) ymin = C[1];
            if (C[1] > ymax) ymax = C[1];
            if (B[2] < zmin) zmin = B[2];
            if (B[2] > zmax) zmax = B[2];
            if (C[2] < zmin) zmin = C[2];
            if (C[2] > zmax) zmax = C[2];
            if (ymax < y0 || ymin > y1 || zmax < z0 || zmin > z1) continue;
            tl[ntl++] = t;
        }
        for (int64_t q = bstart[b]; q < bstart[b + 1]; ++q) {
            const int64_t c = key[q] & 0xffffffffLL;
            int32_t j = cols[2 * c], k = cols[2 * c + 1];
            int64_t py = (int64_t)j << ORC_S, pz = (int64_t)k << ORC_S;
            int64_t m = 0;
            for (int64_t u = 0; u < ntl; ++u) {
                const int64_t t = tl[u];
                const int32_t* A = U + 3 * (int64_t)F[3 * t];
                const int32_t* B = U + 3 * (int64_t)F[3 * t + 1];
                const int32_t* C = U + 3 * (int64_t)F[3 * t + 2];
                /* closed yz-bbox reject: a point outside it is outside the
                 * perturbed projection as well */
                int32_t ymin = A[1], ymax = A[1], zmin = A[2], zmax = A[2];
                if (B[1] < ymin) ymin = B[1];
                if (B[1] > ymax) ymax = B[1];
                if (C[1] < ymin) ymin = C[1];
                if (C[1] > ymax) ymax = C[1];
                if (B[2] < zmin) zmin = B[2];
                if (B[2] > zmax) zmax = B[2];
                if (C[2] < zmin) zmin = C[2];
                if (C[2] > zmax) zmax = C[2];
                if (py < ymin || py > ymax || pz < zmin || pz > zmax) continue;
                int64_t n, d;
                if (column_crossing(A, B, C, py, pz, &n, &d)) {
                    nums[m] = n;
                    dens[m] = d;
                    ++m;
                }
            }
            uint8_t* row = occ + ((int64_t)k * N + j) * (int64_t)N;
            for (int32_t i = 0; i < N; ++i) {
                int64_t x = (int64_t)i << ORC_S;
                int cnt = 0;
                for (int64_t q2 = 0; q2 < m; ++q2)
                    if (nums[q2] <= x * dens[q2]) ++cnt;
                row[i] = (uint8_t)(cnt & 1);
            }
            colmask[(int64_t)k * N + j] = 1;
        }
        free(tl);
        free(nums);
        free(dens);
    }
    free(key);
    free(bstart);
}

/* Number of crossings of each requested column (used by the even-count pin). */
void orc_column_crossing_counts(const int32_t* U, const int32_t* F, int64_t nt,
                                const int32_t* cols, int64_t ncols, int64_t* out)
{
    for (int64_t c = 0; c < ncols; ++c) {
        int64_t py = (int64_t)cols[2 * c] << ORC_S, pz = (int64_t)cols[2 * c + 1] << ORC_S;
        int64_t m = 0;
        for (int64_t t = 0; t < nt; ++t) {
            int64_t n, d;
            if (column_crossing(U + 3 * (int64_t)F[3 * t], U + 3 * (int64_t)F[3 * t + 1],
                                U + 3 * (int64_t)F[3 * t + 2], py, pz, &n, &d))
                ++m;
        }
        out[c] = m;
    }
}

/* ------------------------------------------------------------------------- */
/* Boxes: frames, quantisation, bounds                                        */
/* ------------------------------------------------------------------------- */

static double hmax3(const double* h)
{
    double m = h[0];
    if (h[1] > m) m = h[1];
    if (h[2] > m) m = h[2];
    return m;
}

/* n_ab = rint(2^Q * ((R_ab * h_b) / h_max)), frames R row-major [K][9]. */
void orc_frame_normals(const double* R, int64_t K, const double* h, int32_t* n)
{
    double hm = hmax3(h);
    for (int64_t k = 0; k < K; ++k)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double t = R[9 * k + 3 * a + b] * h[b];
                t = t / hm;
                t = t * 16777216.0;
                n[9 * k + 3 * a + b] = (int32_t)nearbyint(t);
            }
}

/*
 * A user box {c[3], axis0[3], axis1[3], half[3]} (float32) becomes the slab
 * set lo_a <= n_a . U <= hi_a.  axis2 = axis0 x axis1 in FP64.  With
 * m_a = sum_b R_ab ((c_b - lo_b) - h_b / 2) and s = 2^(Q+S) / h_max:
 *   lo_a = floor((m_a - half_a) * s),  hi_a = ceil((m_a + half_a) * s).
 * Returns 0, or -1 for a non-finite box or a negative half extent.
 */
int orc_quantize_boxes(const float* boxes, int64_t K, const double* lo, const double* h,
                       int32_t* n, int64_t* bnd)
{
    double hm = hmax3(h);
    double s = 4294967296.0 / hm;
    for (int64_t k = 0; k < K; ++k) {
        const float* B = boxes + 12 * k;
        for (int q = 0; q < 12; ++q)
            if (!isfinite(B[q])) return -1;
        double R[9];
        for (int b = 0; b < 3; ++b) {
            R[b] = (double)B[3 + b];
            R[3 + b] = (double)B[6 + b];
        }
        R[6] = R[1] * R[5] - R[2] * R[4];
        R[7] = R[2] * R[3] - R[0] * R[5];
        R[8] = R[0] * R[4] - R[1] * R[3];
        orc_frame_normals(R, 1, h, n + 9 * k);
        for (int a = 0; a < 3; ++a) {
            double half = (double)B[9 + a];
            if (half < 0.0) return -1;
            double m = 0.0;
            for (int b = 0; b < 3; ++b) {
                double d = (double)B[b] - lo[b];
                d = d - 0.5 * h[b];
                m = m + R[3 * a + b] * d;
            }
            bnd[6 * k + 2 * a] = (int64_t)floor((m - half) * s);
            bnd[6 * k + 2 * a + 1] = (int64_t)ceil((m + half) * s);
        }
    }
    return 0;
}

static int64_t floordiv64(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

/*
 * Integer AABB of the box in lattice-index space, found from the FP64
 * corners of the parallelepiped and then widened until no lattice point on
 * its boundary layer is inside the box.  out = {i0, i1, j0, j1, k0, k1}.
 */
static int inside_box(const int32_t* n, const int64_t* Lq, const int64_t* Hq, int64_t i, int64_t j, int64_t k)
{
    for (int a = 0; a < 3; ++a) {
        int64_t v = (int64_t)n[3 * a] * i + (int64_t)n[3 * a + 1] * j + (int64_t)n[3 * a + 2] * k;
        if (v < Lq[a] || v > Hq[a]) return 0;
    }
    return 1;
}

static void index_bounds(const int64_t* bnd, int64_t* Lq, int64_t* Hq)
{
    /* lo <= n.(2^S p) <= hi  <=>  ceil(lo/2^S) <= n.p <= floor(hi/2^S) */
    for (int a = 0; a < 3; ++a) {
        Lq[a] = -floordiv64(-bnd[2 * a], 256);
        Hq[a] = floordiv64(bnd[2 * a + 1], 256);
    }
}

static int box_aabb(const int32_t* n, const int64_t* bnd, int64_t* out)
{
    int64_t Lq[3], Hq[3];
    index_bounds(bnd, Lq, Hq);
    for (int a = 0; a < 3; ++a)
        if (Lq[a] > Hq[a]) { /* empty box */
            out[0] = 0; out[1] = -1; out[2] = 0; out[3] = -1; out[4] = 0; out[5] = -1;
            return 0;
        }
    double M[9];
    for (int q = 0; q < 9; ++q) M[q] = (double)n[q];
    double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    if (det == 0.0) return -1;
    double inv[9] = {c00 / det, (M[2] * M[7] - M[1] * M[8]) / det, (M[1] * M[5] - M[2] * M[4]) / det,
                     c01 / det, (M[0] * M[8] - M[2] * M[6]) / det, (M[2] * M[3] - M[0] * M[5]) / det,
                     c02 / det, (M[1] * M[6] - M[0] * M[7]) / det, (M[0] * M[4] - M[1] * M[3]) / det};
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int c = 0; c < 8; ++c) {
        double b[3] = {(double)((c & 1) ? Hq[0] : Lq[0]), (double)((c & 2) ? Hq[1] : Lq[1]),
                       (double)((c & 4) ? Hq[2] : Lq[2])};
        for (int r = 0; r < 3; ++r) {
            double p = inv[3 * r] * b[0] + inv[3 * r + 1] * b[1] + inv[3 * r + 2] * b[2];
            if (p < mn[r]) mn[r] = p;
            if (p > mx[r]) mx[r] = p;
        }
    }
    for (int r = 0; r < 3; ++r) {
        out[2 * r] = (int64_t)floor(mn[r]) - 2;
        out[2 * r + 1] = (int64_t)ceil(mx[r]) + 2;
    }
    /* widen until the boundary layer holds no box point */
    for (int guard = 0; guard < 64; ++guard) {
        int grew = 0;
        for (int r = 0; r < 3 && !grew; ++r)
            for (int side = 0; side < 2 && !grew; ++side) {
                int64_t fixed = out[2 * r + side];
                int r1 = (r + 1) % 3, r2 = (r + 2) % 3;
                for (int64_t u = out[2 * r1]; u <= out[2 * r1 + 1] && !grew; ++u)
                    for (int64_t w = out[2 * r2]; w <= out[2 * r2 + 1]; ++w) {
                        int64_t p[3];
                        p[r] = fixed; p[r1] = u; p[r2] = w;
                        if (inside_box(n, Lq, Hq, p[0], p[1], p[2])) {
                            out[2 * r + side] += side ? 1 : -1;
                            grew = 1;
                            break;
                        }
                    }
            }
        if (!grew) return 0;
    }
    return -2;
}

/* Exposed for tests: the index-space AABB the oracle enumerates. */
int orc_box_aabb(const int32_t* n, const int64_t* bnd, int64_t* out) { return box_aabb(n, bnd, out); }

/*
 * Eq. 4 on the lattice, one point at a time: counts[k] = number of lattice
 * points p in Z^3 inside box k that are not occupied (points outside [0,N)^3
 * are unoccupied); npts[k] = number of lattice points inside box k; ndom[k]
 * (if ndom is not NULL) = those of them inside [0, N)^3.
 * occ/colmask as in orc_occupancy_columns.  Returns 0, -1 for a singular box,
 * -3 when an in-domain column needed has not been computed.
 */
int orc_outer_volume(const uint8_t* occ, const uint8_t* colmask, int32_t N,
                     const int32_t* n, const int64_t* bnd, int64_t K,
                     uint64_t* counts, uint64_t* npts, uint64_t* ndom)
{
    for (int64_t b = 0; b < K; ++b) {
        const int32_t* nb = n + 9 * b;
        int64_t Lq[3], Hq[3], ab[6];
        index_bounds(bnd + 6 * b, Lq, Hq);
        int rc = box_aabb(nb, bnd + 6 * b, ab);
        if (rc) return rc == -1 ? -1 : -2;
        uint64_t cnt = 0, tot = 0, dom = 0;
        int missing = 0;
        int64_t k;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : cnt, tot, dom) reduction(| : missing)
        for (k = ab[4]; k <= ab[5]; ++k)
            for (int64_t j = ab[2]; j <= ab[3]; ++j) {
                int incol = (j >= 0 && j < N && k >= 0 && k < N);
                for (int64_t i = ab[0]; i <= ab[1]; ++i) {
                    if (!inside_box(nb, Lq, Hq, i, j, k)) continue;
                    ++tot;
                    int filled = 0;
                    if (incol && i >= 0 && i < N) {
                        if (!colmask[k * N + j]) {
                            missing = 1;
                            continue;
                        }
                        ++dom;
                        filled = occ[(k * N + j) * (int64_t)N + i];
                    }
                    if (!filled) ++cnt;
                }
            }
        if (missing) return -3;
        counts[b] = cnt;
        npts[b] = tot;
        if (ndom) ndom[b] = dom;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Cluster boxes                                                             */
/* ------------------------------------------------------------------------- */

/* Tight slab bounds of each cluster: min / max of n_a . U over the vertices
 * of its triangles.  Clusters with no triangle get lo = +inf-ish, hi = -inf-ish. */
void orc_tight_bounds(const int32_t* U, const int32_t* F, int64_t nt, const int32_t* assign,
                      int32_t K, const int32_t* n, int64_t* bnd)
{
    for (int32_t k = 0; k < K; ++k)
        for (int a = 0; a < 3; ++a) {
            bnd[6 * k + 2 * a] = INT64_MAX;
            bnd[6 * k + 2 * a + 1] = INT64_MIN;
        }
    for (int64_t t = 0; t < nt; ++t) {
        int32_t k = assign[t];
        for (int v = 0; v < 3; ++v) {
            const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
            for (int a = 0; a < 3; ++a) {
                const int32_t* na = n + 9 * k + 3 * a;
                int64_t d = (int64_t)na[0] * P[0] + (int64_t)na[1] * P[1] + (int64_t)na[2] * P[2];
                if (d < bnd[6 * k + 2 * a]) bnd[6 * k + 2 * a] = d;
                if (d > bnd[6 * k + 2 * a + 1]) bnd[6 * k + 2 * a + 1] = d;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Lloyd partition step (Sec. 4.2.1, Eq. 12-13), restated data-parallel      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t proposals;
    int64_t accepted;
    int64_t gain;       /* sum of accepted gains (exact lattice points) */
    int64_t evals;      /* box counts performed */
} orc_round_stats;

static void bounds_without(const int32_t* U, const int32_t* F, const int32_t* members, int64_t nm,
                           int64_t skip, const int32_t* n, int64_t* out)
{
    for (int a = 0; a < 3; ++a) {
        out[2 * a] = INT64_MAX;
        out[2 * a + 1] = INT64_MIN;
    }
    for (int64_t q = 0; q < nm; ++q) {
        int64_t t = members[q];
        if (t == skip) continue;
        for (int v = 0; v < 3; ++v) {
            const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
            for (int a = 0; a < 3; ++a) {
                int64_t d = (int64_t)n[3 * a] * P[0] + (int64_t)n[3 * a + 1] * P[1] + (int64_t)n[3 * a + 2] * P[2];
                if (d < out[2 * a]) out[2 * a] = d;
                if (d > out[2 * a + 1]) out[2 * a + 1] = d;
            }
        }
    }
}

static void bounds_with(const int32_t* U, const int32_t* F, int64_t t, const int32_t* n,
                        const int64_t* cur, int64_t* out)
{
    memcpy(out, cur, sizeof(int64_t) * 6);
    for (int v = 0; v < 3; ++v) {
        const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
        for (int a = 0; a < 3; ++a) {
            int64_t d = (int64_t)n[3 * a] * P[0] + (int64_t)n[3 * a + 1] * P[1] + (int64_t)n[3 * a + 2] * P[2];
            if (d < out[2 * a]) out[2 * a] = d;
            if (d > out[2 * a + 1]) out[2 * a + 1] = d;
        }
    }
}

static int same6(const int64_t* a, const int64_t* b)
{
    for (int q = 0; q < 6; ++q)
        if (a[q] != b[q]) return 0;
    return 1;
}

static int count_one(const uint8_t* occ, const uint8_t* colmask, int32_t N, const int32_t* n,
                     const int64_t* bnd, uint64_t* c)
{
    uint64_t tot;
    return orc_outer_volume(occ, colmask, N, n, bnd, 1, c, &tot, NULL);
}

/*
 * Partition rounds.  In each round every triangle t whose cluster s has at
 * least two triangles looks at the clusters of its edge neighbours that share
 * s's parent (adj: [nt][3] triangle ids).  For each such k:
 *   gain = [OBV(s) - OBV(s without t)] - [OBV(k with t) - OBV(k)]
 * with boxes recomputed from scratch (tight slab of the members in the
 * cluster's own frame).  t proposes its best k (max gain, ties -> smallest k)
 * when the gain is > 0.  A proposal is accepted when its key (gain desc,
 * t asc) is the largest among all proposals whose source or target is its
 * source or target; accepted moves therefore touch disjoint clusters and the
 * total decreases by exactly the sum of their gains.  Rounds repeat until no
 * move is accepted or `rounds` is reached.  stats: one entry per round run.
 * Returns the number of rounds run, or a negative error.
 */
int orc_lloyd_moves(const int32_t* U, const int32_t* F, const int32_t* adj, int64_t nt,
                    int32_t* assign, const int32_t* parent, int32_t K, const int32_t* n,
                    int64_t* bnd, uint64_t* obv, const uint8_t* occ, const uint8_t* colmask,
                    int32_t N, int32_t rounds, orc_round_stats* stats)
{
    int64_t* size = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    int64_t* start = (int64_t*)calloc((size_t)K + 1, sizeof(int64_t));
    int32_t* members = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
    int64_t* fill = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    int32_t* pdst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
    int64_t* pgain = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
    int64_t* pnewsrc = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)(nt > 0 ? nt : 1));
    int64_t* pnewdst = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)(nt > 0 ? nt : 1));
    uint64_t* pobvsrc = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nt > 0 ? nt : 1));
    uint64_t* pobvdst = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nt > 0 ? nt : 1));
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    int ran = 0, err = 0;
    for (int r = 0; r < rounds && !err; ++r) {
        orc_round_stats st = {0, 0, 0, 0};
        /* cluster member lists, ascending triangle order */
        memset(size, 0, sizeof(int64_t) * (size_t)K);
        for (int64_t t = 0; t < nt; ++t) size[assign[t]]++;
        start[0] = 0;
        for (int32_t k = 0; k < K; ++k) start[k + 1] = start[k] + size[k];
        memset(fill, 0, sizeof(int64_t) * (size_t)K);
        for (int64_t t = 0; t < nt; ++t) {
            int32_t k = assign[t];
            members[start[k] + fill[k]++] = (int32_t)t;
        }
        /* proposals */
        for (int64_t t = 0; t < nt && !err; ++t) {
            pdst[t] = -1;
            int32_t s = assign[t];
            if (size[s] < 2) continue;
            int32_t cand[3];
            int nc = 0;
            for (int e = 0; e < 3; ++e) {
                int32_t k = assign[adj[3 * t + e]];
                if (k == s || parent[k] != parent[s]) continue;
                int dup = 0;
                for (int q = 0; q < nc; ++q) dup |= (cand[q] == k);
                if (!dup) cand[nc++] = k;
            }
            if (nc == 0) continue;
            int64_t shr[6];
            bounds_without(U, F, members + start[s], size[s], t, n + 9 * s, shr);
            if (same6(shr, bnd + 6 * s)) continue; /* removal gain 0, add cost >= 0 */
            uint64_t obv_shr;
            if (count_one(occ, colmask, N, n + 9 * s, shr, &obv_shr)) { err = -3; break; }
            st.evals++;
            int64_t remove_gain = (int64_t)obv[s] - (int64_t)obv_shr;
            int64_t bestg = 0;
            int32_t bestk = -1;
            int64_t bestb[6];
            uint64_t besto = 0;
            for (int q = 0; q < nc; ++q) {
                int32_t k = cand[q];
                int64_t gro[6];
                bounds_with(U, F, t, n + 9 * k, bnd + 6 * k, gro);
                uint64_t obv_gro = obv[k];
                if (!same6(gro, bnd + 6 * k)) {
                    if (count_one(occ, colmask, N, n + 9 * k, gro, &obv_gro)) { err = -3; break; }
                    st.evals++;
                }
                int64_t g = remove_gain - ((int64_t)obv_gro - (int64_t)obv[k]);
                if (g > 0 && (bestk < 0 || g > bestg || (g == bestg && k < bestk))) {
                    bestg = g;
                    bestk = k;
                    memcpy(bestb, gro, sizeof(bestb));
                    besto = obv_gro;
                }
            }
            if (bestk < 0) continue;
            pdst[t] = bestk;
            pgain[t] = bestg;
            memcpy(pnewsrc + 6 * t, shr, sizeof(shr));
            memcpy(pnewdst + 6 * t, bestb, sizeof(bestb));
            pobvsrc[t] = obv_shr;
            pobvdst[t] = besto;
            st.proposals++;
        }
        if (err) break;
        /* locally dominant matching: best proposal touching each cluster */
        for (int32_t k = 0; k < K; ++k) best[k] = -1;
        for (int64_t t = 0; t < nt; ++t) {
            if (pdst[t] < 0) continue;
            int32_t ends[2] = {assign[t], pdst[t]};
            for (int e = 0; e < 2; ++e) {
                int32_t c = ends[e];
                int32_t o = best[c];
                if (o < 0 || pgain[t] > pgain[o] || (pgain[t] == pgain[o] && t < o)) best[c] = (int32_t)t;
            }
        }
        int64_t acc = 0;
        /* decide first, then apply (decisions use the state at round start) */
        for (int64_t t = 0; t < nt; ++t) {
            if (pdst[t] < 0) continue;
            if (best[assign[t]] == t && best[pdst[t]] == t) pgain[t] = -pgain[t] - 1; /* mark */
        }
        for (int64_t t = 0; t < nt; ++t) {
            if (pdst[t] < 0 || pgain[t] >= 0) continue;
            int64_t g = -(pgain[t] + 1);
            int32_t s = assign[t], k = pdst[t];
            memcpy(bnd + 6 * s, pnewsrc + 6 * t, sizeof(int64_t) * 6);
            memcpy(bnd + 6 * k, pnewdst + 6 * t, sizeof(int64_t) * 6);
            obv[s] = pobvsrc[t];
            obv[k] = pobvdst[t];
            assign[t] = k;
            acc++;
            st.gain += g;
        }
        st.accepted = acc;
        if (stats) stats[r] = st;
        ran = r + 1;
        if (acc == 0) break;
    }
    free(size); free(start); free(members); free(fill); free(pdst); free(pgain);
    free(pnewsrc); free(pnewdst); free(pobvsrc); free(pobvdst); free(best);
    return err ? err : ran;
}

/*
 * Partition rounds between levels (Sec. 4.2.2, bottom-up merging): the units
 * are the clusters of the level below (unit_of_tri: [nt] unit ids, Ku units);
 * cluster_of_unit: [Ku] the cluster of this level each unit belongs to (the
 * lower level's parent map, updated in place).  A unit u of cluster s moves as
 * a whole; it may go to a cluster k != s that shares s's parent (parent: [K])
 * and holds a triangle edge-adjacent to one of u's triangles, if s keeps at
 * least one other unit.  For each such k:
 *   gain = [OBV(s) - OBV(s without u)] - [OBV(k with u) - OBV(k)]
 * with both boxes recomputed from scratch (tight slab of all member
 * triangles in the cluster's own frame).  u proposes its best k (max gain,
 * ties -> smallest k) when the gain is > 0, and proposals are matched exactly
 * as in orc_lloyd_moves (key: gain desc, unit asc).  With one triangle per
 * unit this is the triangle step.  Returns the number of rounds run, or a
 * negative error (-3: a needed occupancy column is missing).
 */
static void cluster_bounds(const int32_t* U, const int32_t* F, int64_t nt, const int32_t* unit_of_tri,
                           const int32_t* cluster_of_unit, int32_t k, int32_t skip_unit, int32_t add_unit,
                           const int32_t* n, int64_t* out)
{
    for (int a = 0; a < 3; ++a) {
        out[2 * a] = INT64_MAX;
        out[2 * a + 1] = INT64_MIN;
    }
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t u = unit_of_tri[t];
        const int member = (cluster_of_unit[u] == k && u != skip_unit) || u == add_unit;
        if (!member) continue;
        for (int v = 0; v < 3; ++v) {
            const int32_t* P = U + 3 * (int64_t)F[3 * t + v];
            for (int a = 0; a < 3; ++a) {
                int64_t d = (int64_t)n[3 * a] * P[0] + (int64_t)n[3 * a + 1] * P[1] + (int64_t)n[3 * a + 2] * P[2];
                if (d < out[2 * a]) out[2 * a] = d;
                if (d > out[2 * a + 1]) out[2 * a + 1] = d;
            }
        }
    }
}

int orc_unit_moves(const int32_t* U, const int32_t* F, const int32_t* adj, int64_t nt,
                   const int32_t* unit_of_tri, int32_t Ku, int32_t* cluster_of_unit, const int32_t* parent,
                   int32_t K, const int32_t* n, int64_t* bnd, uint64_t* obv, const uint8_t* occ,
                   const uint8_t* colmask, int32_t N, int32_t rounds, orc_round_stats* stats)
{
    int64_t* usize = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    uint8_t* cand = (uint8_t*)calloc((size_t)K, 1);
    int32_t* pdst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(Ku > 0 ? Ku : 1));
    int64_t* pgain = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Ku > 0 ? Ku : 1));
    int64_t* pnewsrc = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)(Ku > 0 ? Ku : 1));
    int64_t* pnewdst = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)(Ku > 0 ? Ku : 1));
    uint64_t* pobvsrc = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(Ku > 0 ? Ku : 1));
    uint64_t* pobvdst = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(Ku > 0 ? Ku : 1));
    int32_t* best = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
    int ran = 0, err = 0;
    for (int r = 0; r < rounds && !err; ++r) {
        orc_round_stats st = {0, 0, 0, 0};
        memset(usize, 0, sizeof(int64_t) * (size_t)K);
        for (int32_t u = 0; u < Ku; ++u) usize[cluster_of_unit[u]]++;
        for (int32_t u = 0; u < Ku && !err; ++u) {
            pdst[u] = -1;
            const int32_t s = cluster_of_unit[u];
            if (usize[s] < 2) continue;
            /* candidate clusters: siblings of s next to one of u's triangles */
            memset(cand, 0, (size_t)K);
            int nc = 0;
            for (int64_t t = 0; t < nt; ++t) {
                if (unit_of_tri[t] != u) continue;
                for (int e = 0; e < 3; ++e) {
                    const int32_t k = cluster_of_unit[unit_of_tri[adj[3 * t + e]]];
                    if (k == s || parent[k] != parent[s] || cand[k]) continue;
                    cand[k] = 1;
                    ++nc;
                }
            }
            if (nc == 0) continue;
            int64_t shr[6];
            cluster_bounds(U, F, nt, unit_of_tri, cluster_of_unit, s, u, -1, n + 9 * s, shr);
            if (same6(shr, bnd + 6 * s)) continue; /* removal gain 0, add cost >= 0 */
            uint64_t obv_shr;
            if (count_one(occ, colmask, N, n + 9 * s, shr, &obv_shr)) { err = -3; break; }
            st.evals++;
            const int64_t remove_gain = (int64_t)obv[s] - (int64_t)obv_shr;
            int64_t bestg = 0;
            int32_t bestk = -1;
            int64_t bestb[6];
            uint64_t besto = 0;
            for (int32_t k = 0; k < K; ++k) {   /* ascending k: ties keep the smallest */
                if (!cand[k]) continue;
                int64_t gro[6];
                cluster_bounds(U, F, nt, unit_of_tri, cluster_of_unit, k, -1, u, n + 9 * k, gro);
                uint64_t obv_gro = obv[k];
                if (!same6(gro, bnd + 6 * k)) {
                    if (count_one(occ, colmask, N, n + 9 * k, gro, &obv_gro)) { err = -3; break; }
                    st.evals++;
                }
                const int64_t g = remove_gain - ((int64_t)obv_gro - (int64_t)obv[k]);
                if (g > 0 && (bestk < 0 || g > bestg)) {
                    bestg = g;
                    bestk = k;
                    memcpy(bestb, gro, sizeof(bestb));
                    besto = obv_gro;
                }
            }
            if (err || bestk < 0) continue;
            pdst[u] = bestk;
            pgain[u] = bestg;
            memcpy(pnewsrc + 6 * u, shr, sizeof(shr));
            memcpy(pnewdst + 6 * u, bestb, sizeof(bestb));
            pobvsrc[u] = obv_shr;
            pobvdst[u] = besto;
            st.proposals++;
        }
        if (err) break;
        for (int32_t k = 0; k < K; ++k) best[k] = -1;
        for (int32_t u = 0; u < Ku; ++u) {
            if (pdst[u] < 0) continue;
            const int32_t ends[2] = {cluster_of_unit[u], pdst[u]};
            for (int e = 0; e < 2; ++e) {
                const int32_t c = ends[e];
                const int32_t o = best[c];
                if (o < 0 || pgain[u] > pgain[o] || (pgain[u] == pgain[o] && u < o)) best[c] = u;
            }
        }
        int64_t acc = 0;
        for (int32_t u = 0; u < Ku; ++u) {
            if (pdst[u] < 0) continue;
            if (best[cluster_of_unit[u]] == u && best[pdst[u]] == u) pgain[u] = -pgain[u] - 1; /* mark */
        }
        for (int32_t u = 0; u < Ku; ++u) {
            if (pdst[u] < 0 || pgain[u] >= 0) continue;
            const int64_t g = -(pgain[u] + 1);
            const int32_t s = cluster_of_unit[u], k = pdst[u];
            memcpy(bnd + 6 * s, pnewsrc + 6 * u, sizeof(int64_t) * 6);
            memcpy(bnd + 6 * k, pnewdst + 6 * u, sizeof(int64_t) * 6);
            obv[s] = pobvsrc[u];
            obv[k] = pobvdst[u];
            cluster_of_unit[u] = k;
            acc++;
            st.gain += g;
        }
        st.accepted = acc;
        if (stats) stats[r] = st;
        ran = r + 1;
        if (acc == 0) break;
    }
    free(usize); free(cand); free(pdst); free(pgain); free(pnewsrc); free(pnewdst);
    free(pobvsrc); free(pobvdst); free(best);
    return err ? err : ran;
}

/* ------------------------------------------------------------------------- */
/* Flooding partition (Sec. 4.2.1 step 1), sequential, in the paper's order  */
/* ------------------------------------------------------------------------- */

/* Priority of a triangle: distance from its centroid (world FP64, the mean of
 * its three float vertices) to the nearest centre of the boxes it may join,
 * rounded to float; packed with the triangle index as (bits << 32 | t), so
 * equal distances pop in triangle order. */
static uint64_t tri_box_key(const float* V, const int32_t* F, int64_t t, const double* c)
{
    double d2 = 0.0;
    for (int b = 0; b < 3; ++b) {
        double m = (double)V[3 * (int64_t)F[3 * t] + b] + (double)V[3 * (int64_t)F[3 * t + 1] + b];
        m = m + (double)V[3 * (int64_t)F[3 * t + 2] + b];
        m = m / 3.0;
        const double d = m - c[b];
        d2 = d2 + d * d;
    }
    const float f = (float)sqrt(d2);
    uint32_t bits;
    memcpy(&bits, &f, 4);
    return ((uint64_t)bits << 32) | (uint64_t)(uint32_t)t;
}

static void heap_push(uint64_t* h, int64_t* n, uint64_t v)
{
    int64_t i = (*n)++;
    h[i] = v;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p] <= h[i]) break;
        uint64_t tmp = h[p]; h[p] = h[i]; h[i] = tmp;
        i = p;
    }
}

static uint64_t heap_pop(uint64_t* h, int64_t* n)
{
    uint64_t top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *n && h[l] < h[m]) m = l;
        if (r < *n && h[r] < h[m]) m = r;
        if (m == i) break;
        uint64_t tmp = h[m]; h[m] = h[i]; h[i] = tmp;
        i = m;
    }
    return top;
}

/*
 * Patch division by flooding.  group[t] is the set triangle t must stay in
 * (its cluster one level up); box k (frame n_k, centre centre_k in world
 * coordinates) takes triangles of group box_group[k] only.  Centres and
 * frames stay fixed.  Every box first takes as seed the triangle of its group
 * nearest its centre (boxes in index order; a triangle already taken is
 * skipped).  Then the triangle with the smallest priority (distance to the
 * nearest centre of its group's boxes) among those edge-adjacent to an
 * assigned triangle of the same group is taken; it joins, among the boxes
 * holding such a neighbour, the one whose exact outer volume grows least
 * (Eq. 12-13: dOBV = OBV(box with t) - OBV(box); ties -> smaller box), and
 * its unassigned neighbours of the same group become available.  When none is
 * available but triangles remain (a group in several pieces), the remaining
 * triangle of smallest priority is taken with every box of its group as a
 * candidate (an empty box has OBV 0 and grows to the triangle's own slab).
 * Out: assign [nt], bnd [K][6] (tight slabs; empty boxes lo > hi), obv [K].
 * Returns 0, -1 (a box without any triangle of its group), -3 (an occupancy
 * column the count needs is missing).
 */
int orc_flood_partition(const float* V, const int32_t* U, const int32_t* F, const int32_t* adj, int64_t nt,
                        const int32_t* group, int32_t K, const int32_t* box_group, const int32_t* n,
                        const double* centre, const uint8_t* occ, const uint8_t* colmask, int32_t N,
                        int32_t* assign, int64_t* bnd, uint64_t* obv)
{
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nt > 0 ? nt : 1));
    uint64_t* heap = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nt > 0 ? nt : 1));
    uint8_t* queued = (uint8_t*)calloc((size_t)(nt > 0 ? nt : 1), 1);
    uint8_t* cand = (uint8_t*)calloc((size_t)(K > 0 ? K : 1), 1);
    int64_t hn = 0, left = nt;
    int err = 0;
    for (int64_t t = 0; t < nt; ++t) {
        assign[t] = -1;
        key[t] = UINT64_MAX;
        for (int32_t k = 0; k < K; ++k) {
            if (box_group[k] != group[t]) continue;
            const uint64_t kk = tri_box_key(V, F, t, centre + 3 * k);
            if (kk < key[t]) key[t] = kk;
        }
    }
    for (int32_t k = 0; k < K; ++k) {
        for (int a = 0; a < 3; ++a) {
            bnd[6 * k + 2 * a] = INT64_MAX;
            bnd[6 * k + 2 * a + 1] = INT64_MIN;
        }
        obv[k] = 0;
    }
    /* seeds */
    for (int32_t k = 0; k < K && !err; ++k) {
        int64_t best = -1;
        uint64_t bk = UINT64_MAX;
        for (int64_t t = 0; t < nt; ++t) {
            if (group[t] != box_group[k] || assign[t] >= 0) continue;
            const uint64_t kk = tri_box_key(V, F, t, centre + 3 * k);
            if (kk < bk) { bk = kk; best = t; }
        }
        if (best < 0) { err = -1; break; }
        int64_t g[6];
        bounds_with(U, F, best, n + 9 * k, bnd + 6 * k, g);
        memcpy(bnd + 6 * k, g, sizeof(g));
        if (count_one(occ, colmask, N, n + 9 * k, g, obv + k)) { err = -3; break; }
        assign[best] = k;
        queued[best] = 1;
        --left;
    }
    for (int32_t k = 0; k < K && !err; ++k)   /* neighbours of the seeds */
        for (int64_t t = 0; t < nt; ++t) {
            if (assign[t] != k) continue;
            for (int e = 0; e < 3; ++e) {
                const int32_t u = adj[3 * t + e];
                if (queued[u] || group[u] != group[t]) continue;
                queued[u] = 1;
                heap_push(heap, &hn, key[u]);
            }
        }
    while (left > 0 && !err) {
        int64_t t = -1;
        if (hn > 0) {
            t = (int64_t)(uint32_t)(heap_pop(heap, &hn) & 0xffffffffu);
        } else {
            uint64_t bk = UINT64_MAX;
            for (int64_t u = 0; u < nt; ++u)
                if (assign[u] < 0 && key[u] < bk) { bk = key[u]; t = u; }
            queued[t] = 1;
        }
        memset(cand, 0, (size_t)K);
        int nc = 0;
        for (int e = 0; e < 3; ++e) {
            const int32_t u = adj[3 * t + e];
            if (assign[u] >= 0 && group[u] == group[t] && !cand[assign[u]]) { cand[assign[u]] = 1; ++nc; }
        }
        if (nc == 0)
            for (int32_t k = 0; k < K; ++k)
                if (box_group[k] == group[t]) { cand[k] = 1; ++nc; }
        int32_t bestk = -1;
        int64_t bestc = 0;
        int64_t bestb[6];
        uint64_t besto = 0;
        for (int32_t k = 0; k < K && !err; ++k) {
            if (!cand[k]) continue;
            int64_t g[6];
            bounds_with(U, F, t, n + 9 * k, bnd + 6 * k, g);
            uint64_t o = obv[k];
            if (!same6(g, bnd + 6 * k) && count_one(occ, colmask, N, n + 9 * k, g, &o)) { err = -3; break; }
            const int64_t c = (int64_t)o - (int64_t)obv[k];
            if (bestk < 0 || c < bestc) { bestk = k; bestc = c; memcpy(bestb, g, sizeof(g)); besto = o; }
        }
        if (err) break;
        assign[t] = bestk;
        memcpy(bnd + 6 * bestk, bestb, sizeof(bestb));
        obv[bestk] = besto;
        --left;
        for (int e = 0; e < 3; ++e) {
            const int32_t u = adj[3 * t + e];
            if (queued[u] || group[u] != group[t]) continue;
            queued[u] = 1;
            heap_push(heap, &hn, key[u]);
        }
    }
    free(key); free(heap); free(queued); free(cand);
    return err;
}

/* ------------------------------------------------------------------------- */
/* Refit: area-weighted covariance and cyclic Jacobi (FP64)                  */
/* ------------------------------------------------------------------------- */

/*
 * Per cluster moments of the continuous triangle surface, coordinates taken
 * relative to `center`:  mom[k] = {sum A, sum A m (3), sum M (6: xx yy zz xy xz yz)}
 * with A the area, m the centroid and M = A/12 (9 m m^T + p p^T + q q^T + r r^T).
 */
void orc_moments(const float* V, const int32_t* F, int64_t nt, const int32_t* assign, int32_t K,
                 const double* center, double* mom)
{
    memset(mom, 0, sizeof(double) * 10 * (size_t)K);
    for (int64_t t = 0; t < nt; ++t) {
        double P[3][3];
        for (int v = 0; v < 3; ++v)
            for (int b = 0; b < 3; ++b) P[v][b] = (double)V[3 * (int64_t)F[3 * t + v] + b] - center[b];
        double e1[3], e2[3];
        for (int b = 0; b < 3; ++b) {
            e1[b] = P[1][b] - P[0][b];
            e2[b] = P[2][b] - P[0][b];
        }
        double cx = e1[1] * e2[2] - e1[2] * e2[1];
        double cy = e1[2] * e2[0] - e1[0] * e2[2];
        double cz = e1[0] * e2[1] - e1[1] * e2[0];
        double A = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
        double m[3];
        for (int b = 0; b < 3; ++b) m[b] = (P[0][b] + P[1][b] + P[2][b]) / 3.0;
        static const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
        double* o = mom + 10 * assign[t];
        o[0] += A;
        for (int b = 0; b < 3; ++b) o[1 + b] += A * m[b];
        for (int q = 0; q < 6; ++q) {
            int x = ia[q], y = ib[q];
            double s = 9.0 * m[x] * m[y] + P[0][x] * P[0][y] + P[1][x] * P[1][y] + P[2][x] * P[2][y];
            o[4 + q] += A / 12.0 * s;
        }
    }
}

/* Covariance C = sum M / sum A - mu mu^T, mu = sum A m / sum A. cov: xx yy zz xy xz yz.
 * Returns 0, or -1 if sum A == 0. */
int orc_covariance_from_moments(const double* mom, double* cov)
{
    double A = mom[0];
    if (!(A > 0.0)) return -1;
    double mu[3] = {mom[1] / A, mom[2] / A, mom[3] / A};
    static const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) cov[q] = mom[4 + q] / A - mu[ia[q]] * mu[ib[q]];
    return 0;
}

/*
 * Cyclic Jacobi on a symmetric 3x3 matrix (packed xx yy zz xy xz yz).
 * Pivots in the order (0,1), (0,2), (1,2); rotation angle from the stable
 * tangent t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), theta = (a_qq - a_pp) / (2 a_pq).
 * Stops when the off-diagonal square sum is <= 1e-30 * ||A||_F^2 or after 16
 * sweeps.  Eigenvalues sorted descending; frame rows = eigenvectors; the
 * largest-magnitude component of rows 0 and 1 made positive (first index on
 * ties); row 2 = row 0 x row 1.  evals receives the sorted eigenvalues.
 */
void orc_jacobi3(const double* cov, double* R, double* evals)
{
    double A[3][3] = {{cov[0], cov[3], cov[4]}, {cov[3], cov[1], cov[5]}, {cov[4], cov[5], cov[2]}};
    double Vm[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double fro = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) fro += A[i][j] * A[i][j];
    static const int PP[3] = {0, 0, 1}, QQ[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = 2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]);
        if (off <= 1e-30 * fro) break;
        for (int r = 0; r < 3; ++r) {
            int p = PP[r], q = QQ[r];
            if (A[p][q] == 0.0) continue;
            double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
            double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0);
            double s = t * c;
            /* A <- J^T A J with J the rotation in the (p, q) plane */
            for (int k = 0; k < 3; ++k) {
                double akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - s * akq;
                A[k][q] = s * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                double apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - s * aqk;
                A[q][k] = s * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                double vkp = Vm[k][p], vkq = Vm[k][q];
                Vm[k][p] = c * vkp - s * vkq;
                Vm[k][q] = s * vkp + c * vkq;
            }
        }
    }
    double ev[3] = {A[0][0], A[1][1], A[2][2]};
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (ev[ord[j]] > ev[ord[i]]) {
                int tmp = ord[i];
                ord[i] = ord[j];
                ord[j] = tmp;
            }
    for (int a = 0; a < 2; ++a) {
        double row[3] = {Vm[0][ord[a]], Vm[1][ord[a]], Vm[2][ord[a]]};
        int big = 0;
        for (int b = 1; b < 3; ++b)
            if (fabs(row[b]) > fabs(row[big])) big = b;
        double sg = row[big] < 0.0 ? -1.0 : 1.0;
        for (int b = 0; b < 3; ++b) R[3 * a + b] = sg * row[b];
        evals[a] = ev[ord[a]];
    }
    evals[2] = ev[ord[2]];
    R[6] = R[1] * R[5] - R[2] * R[4];
    R[7] = R[2] * R[3] - R[0] * R[5];
    R[8] = R[0] * R[4] - R[1] * R[3];
}

/*
 * Refit (box parameter update): for each cluster, covariance -> Jacobi frame
 * -> quantised normals -> tight bounds -> exact outer volume; the new box is
 * kept iff its outer volume is strictly smaller.  frames/n/bnd/obv updated in
 * place; accepted[k] = 1 where kept.  Returns the number kept or < 0.
 */
int orc_refit(const float* V, const int32_t* U, const int32_t* F, int64_t nt, const int32_t* assign,
              int32_t K, const double* center, const double* h, double* frames, int32_t* n,
              int64_t* bnd, uint64_t* obv, const uint8_t* occ, const uint8_t* colmask, int32_t N,
              uint8_t* accepted)
{
    double* mom = (double*)malloc(sizeof(double) * 10 * (size_t)K);
    double* Rn = (double*)malloc(sizeof(double) * 9 * (size_t)K);
    int32_t* nn = (int32_t*)malloc(sizeof(int32_t) * 9 * (size_t)K);
    int64_t* bn = (int64_t*)malloc(sizeof(int64_t) * 6 * (size_t)K);
    orc_moments(V, F, nt, assign, K, center, mom);
    int kept = 0, err = 0;
    for (int32_t k = 0; k < K; ++k) {
        double cov[6], ev[3];
        accepted[k] = 0;
        if (orc_covariance_from_moments(mom + 10 * k, cov)) {
            memcpy(Rn + 9 * k, frames + 9 * k, sizeof(double) * 9);
            continue;
        }
        orc_jacobi3(cov, Rn + 9 * k, ev);
    }
    orc_frame_normals(Rn, K, h, nn);
    orc_tight_bounds(U, F, nt, assign, K, nn, bn);
    for (int32_t k = 0; k < K && !err; ++k) {
        uint64_t c;
        if (count_one(occ, colmask, N, nn + 9 * k, bn + 6 * k, &c)) { err = -3; break; }
        if (c < obv[k]) {
            memcpy(frames + 9 * k, Rn + 9 * k, sizeof(double) * 9);
            memcpy(n + 9 * k, nn + 9 * k, sizeof(int32_t) * 9);
            memcpy(bnd + 6 * k, bn + 6 * k, sizeof(int64_t) * 6);
            obv[k] = c;
            accepted[k] = 1;
            ++kept;
        }
    }
    free(mom); free(Rn); free(nn); free(bn);
    return err ? err : kept;
}

/*
 * Frames of clusters straight from their covariance (no acceptance test),
 * used to seed a new layer.  Clusters with zero area keep fallback[k].
 */
void orc_cluster_frames(const float* V, const int32_t* F, int64_t nt, const int32_t* assign, int32_t K,
                        const double* center, const double* fallback, double* frames)
{
    double* mom = (double*)malloc(sizeof(double) * 10 * (size_t)K);
    orc_moments(V, F, nt, assign, K, center, mom);
    for (int32_t k = 0; k < K; ++k) {
        double cov[6], ev[3];
        if (orc_covariance_from_moments(mom + 10 * k, cov))
            memcpy(frames + 9 * k, fallback + 9 * k, sizeof(double) * 9);
        else
            orc_jacobi3(cov, frames + 9 * k, ev);
    }
    free(mom);
}

/*
 * Median split of every cluster into two children (initial seeds of the next
 * layer): triangles of cluster k are ordered by key = n0_k . (U_p + U_q + U_r)
 * (the major axis of k's quantised frame applied to three times the centroid,
 * exact in int64), ties by triangle index; the first ceil(size/2) go to child
 * 2k, the rest to child 2k+1.  Returns -4 if a cluster has fewer than 2 triangles.
 */
typedef struct { int64_t key; int64_t t; } orc_kt;

static int cmp_kt(const void* a, const void* b)
{
    const orc_kt* x = (const orc_kt*)a;
    const orc_kt* y = (const orc_kt*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->t < y->t ? -1 : (x->t > y->t ? 1 : 0);
}

int orc_median_split(const int32_t* U, const int32_t* F, int64_t nt, const int32_t* assign, int32_t K,
                     const int32_t* n, int32_t* child)
{
    int64_t* size = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    for (int64_t t = 0; t < nt; ++t) size[assign[t]]++;
    for (int32_t k = 0; k < K; ++k)
        if (size[k] < 2) { free(size); return -4; }
    orc_kt* buf = (orc_kt*)malloc(sizeof(orc_kt) * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        int32_t k = assign[t];
        const int32_t* na = n + 9 * k;
        int64_t s[3] = {0, 0, 0};
        for (int v = 0; v < 3; ++v)
            for (int b = 0; b < 3; ++b) s[b] += U[3 * (int64_t)F[3 * t + v] + b];
        buf[t].key = (int64_t)na[0] * s[0] + (int64_t)na[1] * s[1] + (int64_t)na[2] * s[2];
        buf[t].t = t;
    }
    /* per cluster: collect, sort, split */
    int64_t* start = (int64_t*)calloc((size_t)K + 1, sizeof(int64_t));
    for (int32_t k = 0; k < K; ++k) start[k + 1] = start[k] + size[k];
    int64_t* fill = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    orc_kt* grp = (orc_kt*)malloc(sizeof(orc_kt) * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        int32_t k = assign[t];
        grp[start[k] + fill[k]++] = buf[t];
    }
    for (int32_t k = 0; k < K; ++k) {
        qsort(grp + start[k], (size_t)size[k], sizeof(orc_kt), cmp_kt);
        int64_t half = (size[k] + 1) / 2;
        for (int64_t q = 0; q < size[k]; ++q) child[grp[start[k] + q].t] = 2 * k + (q < half ? 0 : 1);
    }
    free(size); free(buf); free(start); free(fill); free(grp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Surrogate features (the learned screen's inputs), from their definition   */
/* ------------------------------------------------------------------------- */

/* floor(y / z) for z > 0, 128-bit */
static __int128 floordiv128(__int128 y, __int128 z)
{
    __int128 q = y / z;
    if ((y % z != 0) && (y < 0)) q -= 1;
    return q;
}

/*
 * For each quantised box (normals n, integer slab bounds L <= n . p <= H in
 * index units, L = ceil(lo / 256), H = floor(hi / 256)) the surrogate's 524
 * inputs, computed from what they mean:
 *   params   centre of the parallelepiped {L <= n p <= H} divided by N
 *            (n^-1 (L + H) / 2), the unit normals n_0 / |n_0| and n_1 / |n_1|,
 *            and the half widths ((H_a - L_a) / 2) / |n_a| / N, in FP64 from
 *            exact integers, rounded once to FP32;
 *   patch    the occupancy at the centres of an 8 x 8 x 8 subdivision of the
 *            box in its own frame, p = n^-1 v with v_a = L_a + (H_a - L_a)
 *            (2 s_a + 1) / 16 (s_a = 0..7, x fastest), rounded to the nearest
 *            lattice point, floor(p + 1/2), and 0 outside [0, N)^3.
 * The sample points are exact rationals: with the adjugate A of n (int64)
 * and det (128 bits), p_r + 1/2 = (sum_a A_ra (16 v_a) + 8 det) / (16 det), an
 * exact 128-bit quotient.  If `tie` is given, tie[512 b + s] = 1 when some
 * coordinate of point s lies within 10^-3 of a rounding tie (a half-integer),
 * where a computation in floating point may round either way.  det = 0 gives
 * zero parameters and bits.  Returns 0, or -3 if an in-domain column needed
 * is not computed.
 */
int orc_surrogate_features(const uint8_t* occ, const uint8_t* colmask, int32_t N, const int32_t* n,
                           const int64_t* bnd, int64_t K, float* feats, uint8_t* tie)
{
    for (int64_t b = 0; b < K; ++b) {
        const int32_t* nb = n + 9 * b;
        int64_t m[9], L[3], H[3];
        for (int i = 0; i < 9; ++i) m[i] = nb[i];
        for (int a = 0; a < 3; ++a) {
            L[a] = -floordiv64(-bnd[6 * b + 2 * a], 256);
            H[a] = floordiv64(bnd[6 * b + 2 * a + 1], 256);
        }
        /* A[3 r + a]: adjugate entry, n^-1 = A / det */
        const int64_t A[9] = {m[4] * m[8] - m[5] * m[7], m[2] * m[7] - m[1] * m[8], m[1] * m[5] - m[2] * m[4],
                              m[5] * m[6] - m[3] * m[8], m[0] * m[8] - m[2] * m[6], m[2] * m[3] - m[0] * m[5],
                              m[3] * m[7] - m[4] * m[6], m[1] * m[6] - m[0] * m[7], m[0] * m[4] - m[1] * m[3]};
        const __int128 det = (__int128)m[0] * A[0] + (__int128)m[1] * A[3] + (__int128)m[2] * A[6];
        float* f = feats + 524 * b;
        uint8_t* tb = tie ? tie + 512 * b : NULL;
        for (int r = 0; r < 3; ++r) {
            double c = 0.0;
            if (det != 0) {
                __int128 num = 0;
                for (int a = 0; a < 3; ++a) num += (__int128)A[3 * r + a] * (__int128)(L[a] + H[a]);
                c = ((double)num / (2.0 * (double)det)) / (double)N;
            }
            f[r] = (float)c;
        }
        for (int a = 0; a < 3; ++a) {
            const double n0 = (double)nb[3 * a], n1 = (double)nb[3 * a + 1], n2 = (double)nb[3 * a + 2];
            const double nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);   /* exact sum below 2^53 */
            if (a < 2) {
                f[3 + 3 * a] = nn > 0.0 ? (float)(n0 / nn) : 0.0f;
                f[4 + 3 * a] = nn > 0.0 ? (float)(n1 / nn) : 0.0f;
                f[5 + 3 * a] = nn > 0.0 ? (float)(n2 / nn) : 0.0f;
            }
            f[9 + a] = nn > 0.0 ? (float)((0.5 * (double)(H[a] - L[a]) / nn) / (double)N) : 0.0f;
        }
        /* denominator 16 det made positive */
        const __int128 Z = det < 0 ? -16 * det : 16 * det;
        const __int128 sg = det < 0 ? -1 : 1;
        for (int s = 0; s < 512; ++s) {
            const int sv[3] = {s & 7, (s >> 3) & 7, s >> 6};
            int64_t idx[3];
            int near = 0;
            for (int r = 0; r < 3; ++r) {
                idx[r] = -1;
                if (det == 0) continue;
                __int128 X = 8 * det;
                for (int a = 0; a < 3; ++a) {
                    const __int128 v16 = (__int128)16 * L[a] + (__int128)(H[a] - L[a]) * (2 * sv[a] + 1);
                    X += (__int128)A[3 * r + a] * v16;
                }
                const __int128 Y = sg * X;
                const __int128 q = floordiv128(Y, Z);
                const __int128 fr = Y - q * Z;             /* in [0, Z) */
                const __int128 dist = fr < Z - fr ? fr : Z - fr;
                if (1000 * dist < Z) near = 1;
                idx[r] = (q >= -1 && q <= (__int128)N) ? (int64_t)q : -1;
            }
            float bit = 0.f;
            if (idx[0] >= 0 && idx[0] < N && idx[1] >= 0 && idx[1] < N && idx[2] >= 0 && idx[2] < N) {
                if (!colmask[idx[2] * N + idx[1]]) return -3;
                bit = (float)occ[(idx[2] * N + idx[1]) * (int64_t)N + idx[0]];
            }
            f[12 + s] = bit;
            if (tb) tb[s] = (uint8_t)near;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Box-parameter descent: rotation probes (the perturbation search of the   */
/* box update, Sec. 4.2.1 step 2)                                             */
/* ------------------------------------------------------------------------- */

/* Frame of probe p (axis p / 2, sign + for even p) rotated by the rational
 * rotation cos = (1 - t^2)/(1 + t^2), sin = 2t/(1 + t^2), t = 2^-(5 + level). */
void orc_probe_frame(const double* R, int32_t level, int32_t p, double* O)
{
    double t = ldexp(1.0, -(5 + level));
    double t2 = t * t;
    double den = 1.0 + t2;
    double c = (1.0 - t2) / den;
    double sn = (2.0 * t) / den;
    double ss = (p & 1) ? -sn : sn;
    int a = p >> 1, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    for (int j = 0; j < 3; ++j) {
        O[3 * a + j] = R[3 * a + j];
        O[3 * b1 + j] = c * R[3 * b1 + j] + ss * R[3 * b2 + j];
        O[3 * b2 + j] = c * R[3 * b2 + j] - ss * R[3 * b1 + j];
    }
}

/*
 * One descent step for every cluster below level 8: the six probes' tight
 * boxes are counted exactly; the lowest count (ties -> smaller probe index)
 * replaces the cluster's box when strictly below its outer volume, otherwise
 * the cluster's level rises by one.  Returns the number of boxes replaced.
 */
int orc_descent_step(const int32_t* U, const int32_t* F, int64_t nt, const int32_t* assign, int32_t K,
                     const double* h, double* frames, int32_t* n, int64_t* bnd, uint64_t* obv, int32_t* level,
                     const uint8_t* occ, const uint8_t* colmask, int32_t N)
{
    int64_t* size = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    int64_t* start = (int64_t*)calloc((size_t)K + 1, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    int32_t* members = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
    for (int64_t t = 0; t < nt; ++t) size[assign[t]]++;
    for (int32_t k = 0; k < K; ++k) start[k + 1] = start[k] + size[k];
    for (int64_t t = 0; t < nt; ++t) members[start[assign[t]] + fill[assign[t]]++] = (int32_t)t;
    int kept = 0, err = 0;
    for (int32_t k = 0; k < K && !err; ++k) {
        if (level[k] >= 8) continue;
        uint64_t best = UINT64_MAX;
        int bp = -1;
        double bR[9];
        int32_t bn[9];
        int64_t bb[6];
        for (int p = 0; p < 6; ++p) {
            double R[9];
            int32_t nn[9];
            int64_t b6[6];
            orc_probe_frame(frames + 9 * k, level[k], p, R);
            orc_frame_normals(R, 1, h, nn);
            bounds_without(U, F, members + start[k], size[k], -1, nn, b6);
            uint64_t c;
            if (count_one(occ, colmask, N, nn, b6, &c)) { err = -3; break; }
            if (c < best) {
                best = c;
                bp = p;
                memcpy(bR, R, sizeof(bR));
                memcpy(bn, nn, sizeof(bn));
                memcpy(bb, b6, sizeof(bb));
            }
        }
        if (err) break;
        if (bp >= 0 && best < obv[k]) {
            memcpy(frames + 9 * k, bR, sizeof(bR));
            memcpy(n + 9 * k, bn, sizeof(bn));
            memcpy(bnd + 6 * k, bb, sizeof(bb));
            obv[k] = best;
            ++kept;
        } else {
            level[k] += 1;
        }
    }
    free(size); free(start); free(fill); free(members);
    return err ? err : kept;
}
