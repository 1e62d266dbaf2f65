"""Pins of the oracle's solid occupancy (the Omega(X) of Sec. 3, discretised on
the lattice) against geometry it does not compute itself."""
import numpy as np
import pytest

import oracle as O
from synth import meshes as M
from tests import pins


def _two_cubes(N, inner_lo, inner_hi, offset=(0, 0, 0)):
    """Outer cube [0, N]^3 (so lo = 0, h = 1: lattice point i at x = i + 1/2,
    fixed point U = 256 (x - 1/2)) and an inner cube whose corners sit exactly
    on lattice points: world corner a + 1/2 snaps to U = 256 a."""
    outer = M.cube((0, 0, 0), (N, N, N))
    lo = np.asarray(inner_lo) + 0.5 + np.asarray(offset)
    hi = np.asarray(inner_hi) + 0.5 + np.asarray(offset)
    inner = M.cube(tuple(lo), tuple(hi))
    V = np.concatenate([outer.verts, inner.verts])
    F = np.concatenate([outer.tris, inner.tris + 8])
    return V, F


def test_cube_all_inside():
    """A closed cube over its own AABB: every cell-centred point is inside."""
    for N, hi in ((8, (1.0, 2.0, 3.0)), (13, (0.7, 0.7, 5.0))):
        m = M.cube((0, 0, 0), hi)
        P = O.Problem(m.verts, m.tris, N)
        P.occ.fill_all()
        assert P.occ.occ.sum() == N ** 3


def test_faces_on_lattice_points_half_open():
    """Tie rules: a face through lattice points.  The crossing at x* = x counts
    (x* <= x), and the (y, z) query point is perturbed by (+eps, +eps^2); so
    an inner cube with corners on lattice planes a..b removes exactly the
    half-open index box [a0, b0) x [a1, b1) x [a2, b2) from the outer solid."""
    N = 12
    a, b = (2, 3, 4), (7, 9, 8)
    V, F = _two_cubes(N, a, b)
    P = O.Problem(V, F, N)
    assert np.allclose(P.lo, 0.0) and np.allclose(P.h, 1.0)
    P.occ.fill_all()
    expect = np.ones((N, N, N), dtype=np.uint8)
    expect[a[2]:b[2], a[1]:b[1], a[0]:b[0]] = 0   # [k, j, i]
    assert np.array_equal(P.occ.occ, expect)


def test_translation_by_whole_cells():
    """Moving an inner solid by one cell along each axis shifts its bits by one."""
    N = 16
    rng = np.random.Generator(np.random.PCG64(7))
    ico = M.icosphere(1, center=(0, 0, 0), radius=2.6)
    base = np.round((ico.verts.astype(np.float64) + 7.3) * 1024) / 1024   # dyadic: exact in float32
    outer = M.cube((0, 0, 0), (N, N, N))
    occs = []
    for d in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)):
        V = np.concatenate([outer.verts, (base + np.asarray(d)).astype(np.float32)])
        F = np.concatenate([outer.tris, ico.tris + 8])
        P = O.Problem(V, F, N)
        P.occ.fill_all()
        occs.append(P.occ.occ.astype(np.int8))
    o0 = occs[0]
    assert (1 - o0).sum() > 50                        # the inner solid is non-trivial
    assert np.array_equal(np.roll(o0, 1, axis=2), occs[1])   # x -> i (last axis)
    assert np.array_equal(np.roll(o0, 1, axis=1), occs[2])
    assert np.array_equal(np.roll(o0, 1, axis=0), occs[3])


@pytest.mark.parametrize("name", ["torus", "icosphere", "sdf"])
def test_parity_matches_winding_number(name):
    """Away from the surface, inside-ness by crossing parity equals the
    generalised winding number (solid-angle sum / 4 pi) of the snapped mesh."""
    rng = np.random.Generator(np.random.PCG64(11))
    if name == "torus":
        m, N = M.torus_4096(), 64
    elif name == "icosphere":
        m, N = M.icosphere(3, radius=1.0), 40
    else:
        m, N = M.sdf_union_mesh(5, 24, 6, 3, 0), 48
    P = O.Problem(m.verts, m.tris, N)
    cols = rng.integers(0, N, size=(60, 2))
    P.occ.fill_columns(cols)
    Vw = pins.fixed_to_world(P.U, P.lo, P.h)
    pts, bits = [], []
    for j, k in np.unique(cols, axis=0):
        i = np.arange(N)
        pts.append(np.stack([P.lo[0] + (i + 0.5) * P.h[0],
                             np.full(N, P.lo[1] + (j + 0.5) * P.h[1]),
                             np.full(N, P.lo[2] + (k + 0.5) * P.h[2])], -1))
        bits.append(P.occ.occ[k, j, :])
    pts = np.concatenate(pts)
    bits = np.concatenate(bits)
    w = pins.winding_numbers(pts, Vw, P.F.astype(np.int64))
    clean = np.abs(w - np.round(w)) < 1e-6
    assert clean.mean() > 0.99
    wb = (np.abs(np.round(w[clean])).astype(np.int64) & 1).astype(np.uint8)
    assert np.array_equal(wb, bits[clean])
    assert bits.sum() > 0 and bits.sum() < bits.size


def test_even_crossings_per_column():
    """A closed surface crosses every column an even number of times."""
    m = M.torus_4096()
    P = O.Problem(m.verts, m.tris, 64)
    j, k = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    cnt = O.column_crossings(P.U, P.F, np.stack([j.ravel(), k.ravel()], -1))
    assert cnt.max() >= 4          # columns through both sides of the ring
    assert np.all(cnt % 2 == 0)


@pytest.mark.parametrize("name", ["torus", "icosphere"])
def test_volume_against_divergence_theorem(name):
    """sum(occ) * cell volume vs the exact polyhedron volume of the snapped
    mesh: only cells cut by the surface can be wrong, all of which lie within
    half a cell diagonal of it, so |dV| <= sqrt(3) h_max A."""
    if name == "torus":
        m, N = M.torus_4096(), 64
    else:
        m, N = M.icosphere(3, radius=1.0), 48
    P = O.Problem(m.verts, m.tris, N)
    P.occ.fill_all()
    Vw = pins.fixed_to_world(P.U, P.lo, P.h)
    vol = abs(pins.polyhedron_volume(Vw, P.F.astype(np.int64)))
    area = pins.surface_area(Vw, P.F.astype(np.int64))
    got = P.occ.occ.sum() * np.prod(P.h)
    bound = np.sqrt(3.0) * P.h.max() * area
    assert abs(got - vol) <= bound
    # and the estimate is far better than the bound in practice
    assert abs(got - vol) <= 0.1 * bound


def test_snap_definition_values():
    """The fixed-point snap of Sec. 3's lattice reading: the AABB corners land
    on -2^(S-1) and N 2^S - 2^(S-1), the AABB centre on (N-1) 2^(S-1)."""
    m = M.cube((-1.0, 0.0, 2.0), (1.0, 4.0, 2.5))
    for N in (8, 64, 512):
        P = O.Problem(m.verts, m.tris, N)
        assert P.U.min() == -128 and P.U.max() == 256 * N - 128
        c = O.snap(np.array([[0.0, 2.0, 2.25]], dtype=np.float32), P.lo, P.h)
        assert np.all(c == (N - 1) * 128)
