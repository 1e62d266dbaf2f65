"""Pins of the oracle's box adjustment for local minima (Sec. 4.2.1 step 3)."""
import numpy as np

import oracle as O
from synth import meshes as M


def _flat_layer(K=8, iters=6):
    """K boxes under one parent on a union of 6 spheres and 3 capsules, after
    Lloyd iterations from a median-split seeding."""
    m = M.sdf_union_mesh(7, 14, n_spheres=6, n_capsules=3)
    P = O.Problem(m.verts, m.tris, 32)
    depth = int(np.log2(K))
    seed = O.build_tree(P, depth, iters=0)[depth]
    L = O.layer_init(P, seed.assign, np.zeros(K, np.int32))
    for _ in range(iters):
        O.lloyd_step(P, L, 16, 1)
    return P, L


def _consistent(P, L):
    assert np.all(np.bincount(L.assign, minlength=L.K) > 0)
    assert np.array_equal(L.n, O.frame_normals(L.frames, P.h))
    assert np.array_equal(L.bnd, O.tight_bounds(P.U, P.F, L.assign, L.K, L.n))
    assert np.array_equal(L.obv, O.outer_volume(P.occ, L.n, L.bnd)[0])


def test_adjustment_escapes_a_lloyd_fixed_point():
    P, L = _flat_layer()
    before = int(L.obv.astype(np.int64).sum())
    size = np.bincount(L.assign, minlength=L.K)
    kept, k, j = O.adjust_step(P, L, iters=3)
    assert k == int(np.lexsort((np.arange(L.K), size))[0])       # fewest triangles
    assert kept and int(L.obv.astype(np.int64).sum()) < before
    _consistent(P, L)


def test_rejected_adjustment_restores_the_layer():
    P, L = _flat_layer()
    O.adjust_step(P, L, iters=3)
    ref = L.copy()
    for _ in range(3):
        kept, k, j = O.adjust_step(P, L, iters=3)
        if kept:
            ref = L.copy()
            continue
        assert np.array_equal(L.assign, ref.assign) and np.array_equal(L.frames, ref.frames)
        assert np.array_equal(L.bnd, ref.bnd) and np.array_equal(L.obv, ref.obv)
    _consistent(P, L)


def test_adjustment_keeps_triangles_in_their_group():
    m = M.sdf_union_mesh(3, 12, n_spheres=5, n_capsules=2)
    P = O.Problem(m.verts, m.tris, 28)
    layers = O.build_tree(P, 3, iters=1)
    L = layers[3]
    group = L.parent[L.assign].copy()
    for _ in range(4):
        O.adjust_step(P, L, iters=2)
        assert np.array_equal(L.parent[L.assign], group)
        _consistent(P, L)
