"""Pins of the oracle's per-box outer volume (Eq. 4 on the lattice) and of
the box quantisation."""
import numpy as np
import pytest

import oracle as O
from synth import meshes as M
from tests import pins


def _aabb_box_bounds(P, n):
    """Tight slab bounds of all vertices of the mesh under normals n."""
    d = P.U.astype(np.int64) @ n.reshape(3, 3).astype(np.int64).T
    return np.stack([d.min(0), d.max(0)], -1).reshape(-1)


def test_axis_aligned_cube_in_its_own_box_is_zero():
    """Outer volume of an axis-aligned cube mesh in its own tight box is 0."""
    for N, hi in ((16, (1.0, 2.0, 3.0)), (21, (3.0, 1.0, 0.5))):
        m = M.cube((0, 0, 0), hi)
        P = O.Problem(m.verts, m.tris, N)
        n = O.frame_normals(np.eye(3).reshape(1, 9), P.h)
        bnd = _aabb_box_bounds(P, n[0]).reshape(1, 6)
        cnt, tot = O.outer_volume(P.occ, n, bnd)
        assert cnt[0] == 0 and tot[0] == N ** 3


def test_sphere_in_bounding_cube():
    """Icosphere of radius r in its axis-aligned tight box: OBV h^3 ~ box
    volume - polyhedron volume, within sqrt(3) h (A_box + A_poly)."""
    m = M.icosphere(3, radius=1.0)
    N = 48
    P = O.Problem(m.verts, m.tris, N)
    n = O.frame_normals(np.eye(3).reshape(1, 9), P.h)
    bnd = _aabb_box_bounds(P, n[0]).reshape(1, 6)
    cnt, tot = O.outer_volume(P.occ, n, bnd)
    Vw = pins.fixed_to_world(P.U, P.lo, P.h)
    F = P.F.astype(np.int64)
    ext = Vw.max(0) - Vw.min(0)
    box_vol = float(np.prod(ext))
    box_area = 2.0 * (ext[0] * ext[1] + ext[1] * ext[2] + ext[0] * ext[2])
    poly = abs(pins.polyhedron_volume(Vw, F))
    area = pins.surface_area(Vw, F)
    cell = float(np.prod(P.h))
    bound = np.sqrt(3.0) * P.h.max() * (box_area + area)
    assert abs(float(cnt[0]) * cell - (box_vol - poly)) <= bound
    assert abs(float(tot[0]) * cell - box_vol) <= np.sqrt(3.0) * P.h.max() * box_area


def _rand_box(rng, center, half):
    R = pins.random_rotation(rng)
    return np.concatenate([center, R[0], R[1], half]).astype(np.float32), R


def test_rotated_box_point_count_matches_volume():
    """Quantised FP32 box on an anisotropic lattice: the number of lattice
    points inside approaches the box volume / cell volume (a transposed or
    mis-scaled normal would miss by a large factor)."""
    m = M.cube((0, 0, 0), (4.0, 2.0, 1.0))     # anisotropic h = (4, 2, 1) / N
    N = 64
    P = O.Problem(m.verts, m.tris, N)
    rng = np.random.Generator(np.random.PCG64(3))
    cell = float(np.prod(P.h))
    for _ in range(6):
        half = rng.uniform(0.2, 0.6, 3)
        box, R = _rand_box(rng, rng.uniform([1, 0.5, 0.3], [3, 1.5, 0.7]), half)
        n, bnd = O.quantize_boxes(box[None], P.lo, P.h)
        cnt, tot = O.outer_volume(P.occ, n, bnd)
        vol = 8.0 * np.prod(half)
        area = 8.0 * (half[0] * half[1] + half[1] * half[2] + half[0] * half[2])
        assert abs(float(tot[0]) * cell - vol) <= np.sqrt(3.0) * P.h.max() * area
        # inside-the-solid points never count, points outside [0,N)^3 always do
        assert cnt[0] <= tot[0]


def test_box_outside_domain_counts_every_point():
    """A box beyond the lattice: every point is outside the solid; for an
    axis-aligned box the count is the product of the index ranges."""
    m = M.cube((0, 0, 0), (1.0, 1.0, 1.0))
    N = 16
    P = O.Problem(m.verts, m.tris, N)
    n = O.frame_normals(np.eye(3).reshape(1, 9), P.h)
    # n = 2^24 e_a (h isotropic): slab lo <= 2^24 U_a <= hi, U = 256 i
    lo_i = np.array([20, -9, 3])
    hi_i = np.array([25, -2, 30])
    bnd = np.stack([lo_i * 256 * 2 ** 24, hi_i * 256 * 2 ** 24], -1).reshape(1, 6)
    cnt, tot = O.outer_volume(P.occ, n, bnd)
    assert cnt[0] == tot[0] == np.prod(hi_i - lo_i + 1)


def test_box_inside_solid_is_zero():
    m = M.icosphere(3, radius=1.0)
    N = 40
    P = O.Problem(m.verts, m.tris, N)
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(4):
        box, _ = _rand_box(rng, rng.uniform(-0.1, 0.1, 3), np.full(3, 0.45))
        n, bnd = O.quantize_boxes(box[None], P.lo, P.h)
        cnt, tot = O.outer_volume(P.occ, n, bnd)
        assert tot[0] > 1000 and cnt[0] == 0


def test_monotone_under_growth_and_bounds():
    """Growing a box with fixed axes never lowers its outer volume (the
    property behind Eq. 12); 0 <= OBV <= points in box."""
    m = M.torus_4096()
    N = 48
    P = O.Problem(m.verts, m.tris, N)
    rng = np.random.Generator(np.random.PCG64(9))
    for _ in range(5):
        box, _ = _rand_box(rng, rng.uniform(-0.8, 0.8, 3) * [1, 1, 0.2], rng.uniform(0.1, 0.4, 3))
        n, bnd = O.quantize_boxes(box[None], P.lo, P.h)
        prev = None
        for grow in range(4):
            b2 = bnd.copy()
            b2[0, 0::2] -= grow * 3 * 2 ** 30
            b2[0, 1::2] += grow * 3 * 2 ** 30
            cnt, tot = O.outer_volume(P.occ, n, b2)
            assert 0 <= cnt[0] <= tot[0]
            if prev is not None:
                assert cnt[0] >= prev[0] and tot[0] >= prev[1]
            prev = (cnt[0], tot[0])


def test_sum_obv_bounds_union_omv():
    """Eq. 5-6: sum_j OBV_j >= OMV(union), equal for disjoint boxes.  The
    union count is an independent numpy mask over a region."""
    m = M.torus_4096()
    N = 40
    P = O.Problem(m.verts, m.tris, N)
    P.occ.fill_all()
    rng = np.random.Generator(np.random.PCG64(13))
    boxes = []
    for _ in range(5):
        box, _ = _rand_box(rng, rng.uniform(-0.9, 0.9, 3) * [1, 1, 0.3], rng.uniform(0.15, 0.5, 3))
        boxes.append(box)
    n, bnd = O.quantize_boxes(np.stack(boxes), P.lo, P.h)
    cnt, _ = O.outer_volume(P.occ, n, bnd)
    # union over a region well beyond every box (checked below: no box point
    # on the region's outer layer)
    ab = np.stack([O.box_aabb(n[b], bnd[b]) for b in range(n.shape[0])])
    rlo = ab[:, 0::2].min(0) - 6
    rhi = ab[:, 1::2].max(0) + 6
    K_, J_, I_ = np.meshgrid(np.arange(rlo[2], rhi[2] + 1), np.arange(rlo[1], rhi[1] + 1),
                             np.arange(rlo[0], rhi[0] + 1), indexing="ij")
    pts = np.stack([I_, J_, K_], -1).reshape(-1, 3).astype(np.int64) * 256
    edge = np.any((pts // 256 == rlo) | (pts // 256 == rhi), axis=1)
    inside_any = np.zeros(pts.shape[0], dtype=bool)
    per_box = []
    for b in range(n.shape[0]):
        d = pts @ n[b].reshape(3, 3).astype(np.int64).T
        ins = np.all((d >= bnd[b, 0::2]) & (d <= bnd[b, 1::2]), axis=1)
        per_box.append(ins)
        inside_any |= ins
        assert not np.any(ins & edge)
    p = pts // 256
    indom = np.all((p >= 0) & (p < N), axis=1)
    occ = np.zeros(pts.shape[0], dtype=bool)
    occ[indom] = P.occ.occ[p[indom, 2], p[indom, 1], p[indom, 0]] == 1
    omv = int((inside_any & ~occ).sum())
    for b in range(n.shape[0]):
        assert int((per_box[b] & ~occ).sum()) == int(cnt[b])   # region covers the box
    assert int(cnt.sum()) >= omv
    overlap = int(sum((pb & ~occ).sum() for pb in per_box)) - omv
    assert overlap == int(cnt.sum()) - omv and overlap >= 0


def test_quantize_rejects_bad_boxes():
    m = M.cube()
    P = O.Problem(m.verts, m.tris, 8)
    bad = np.zeros((1, 12), dtype=np.float32)
    bad[0, 3] = 1
    bad[0, 7] = 1
    bad[0, 9] = -0.1
    with pytest.raises(ValueError):
        O.quantize_boxes(bad, P.lo, P.h)
    bad[0, 9] = np.nan
    with pytest.raises(ValueError):
        O.quantize_boxes(bad, P.lo, P.h)


def _axis_box(lo, h, a, b):
    """FP32 axis-aligned box whose faces sit at lo + a h and lo + b h (per axis)."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    c = lo + 0.5 * (a + b) * h
    half = 0.5 * (b - a) * h
    box = np.concatenate([c, [1, 0, 0], [0, 1, 0], half]).astype(np.float32)
    assert np.array_equal(box.astype(np.float64)[[0, 1, 2, 9, 10, 11]], np.concatenate([c, half]))
    return box


def test_axis_aligned_box_counts_closed_form_on_anisotropic_lattice():
    """Axis-aligned FP32 boxes on an anisotropic lattice (h = 1/16, 1/32, 1/64; every value dyadic, so
    the quantisation is exact).  Lattice point i sits at lo + (i + 1/2) h (R1), so a box with faces at
    lo + a h and lo + b h holds the indices a..b-1 per axis, and a face through lattice points
    (a = i + 1/2) keeps them (closed box, R7).  The cube mesh fills every in-domain point, so the outer
    volume is exactly the box's points outside [0, N)^3 (R2).  A transposed or inverted h_b / h_max scale
    in the normals, an open box or a half-cell offset in the snap changes these products."""
    m = M.cube((0, 0, 0), (4.0, 2.0, 1.0))
    N = 64
    P = O.Problem(m.verts, m.tris, N)
    assert np.array_equal(P.h, [1 / 16, 1 / 32, 1 / 64]) and np.array_equal(P.lo, [0, 0, 0])
    n, _ = O.quantize_boxes(_axis_box(P.lo, P.h, [1, 1, 1], [2, 2, 2])[None], P.lo, P.h)
    assert np.array_equal(n[0], [2 ** 24, 0, 0, 0, 2 ** 23, 0, 0, 0, 2 ** 22])
    cases = [([3, 5, 7], [10, 9, 40]),          # inside the domain: no outer volume
             ([-4, 2, 60], [5, 70, 71]),        # poking out on three sides
             ([-9, -3, -7], [-1, -1, -2]),      # entirely outside
             ([2.5, 0.5, 10.5], [6.5, 3.5, 12.5])]  # faces through lattice points: closed
    for a, b in cases:
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        qn, bnd = O.quantize_boxes(_axis_box(P.lo, P.h, a, b)[None], P.lo, P.h)
        cnt, tot = O.outer_volume(P.occ, qn, bnd)
        first = np.ceil(a - 0.5).astype(np.int64)       # smallest i with i + 1/2 >= a
        last = np.floor(b - 0.5).astype(np.int64)       # largest i with i + 1/2 <= b
        ext = np.maximum(last - first + 1, 0)
        indom = np.maximum(np.minimum(last, N - 1) - np.maximum(first, 0) + 1, 0)
        assert int(tot[0]) == int(np.prod(ext)), (a, b)
        assert int(cnt[0]) == int(np.prod(ext)) - int(np.prod(indom)), (a, b)
