"""Pins of the oracle's moves between levels (Sec. 4.2.2, bottom-up merging
with boxes as the division unit) and of the reciprocating sweeps."""
import numpy as np

import oracle as O
from synth import meshes as M


def _problem(nu=32, nv=16, N=40, seed=3):
    m = M.torus(1.0, 0.3, nu, nv, jitter=0.01, seed=seed)
    return O.Problem(m.verts, m.tris, N)


def _blobs(seed=7, grid=14, N=32):
    """A union of 6 spheres and 3 capsules, about 2k triangles."""
    m = M.sdf_union_mesh(seed, grid, n_spheres=6, n_capsules=3)
    return O.Problem(m.verts, m.tris, N)


def _singletons(up: O.Layer):
    """A level below `up` whose units are single triangles."""
    T = up.assign.shape[0]
    z = np.zeros((T, 9))
    return O.Layer(np.arange(T, dtype=np.int32), up.assign.copy(), z, np.zeros((T, 9), np.int32),
                   np.zeros((T, 6), np.int64), np.zeros(T, np.uint64))


def test_single_triangle_units_reduce_to_the_triangle_step():
    P = _problem()
    layers = O.build_tree(P, 3, iters=0)
    moved = 0
    for up0 in layers[1:]:
        a, b = up0.copy(), up0.copy()
        st_t = O.lloyd_moves(P, a, 8)
        low = _singletons(b)
        st_u = O.unit_moves(P, b, low, 8)
        assert st_t == st_u
        moved += sum(s["accepted"] for s in st_t)
        assert np.array_equal(a.assign, b.assign) and np.array_equal(low.parent, b.assign)
        assert np.array_equal(a.bnd, b.bnd) and np.array_equal(a.obv, b.obv)
    assert moved > 0


def _brute_gain(P, up, low, u, k):
    """Exact gain of moving unit u into cluster k, from tight bounds and the
    per-point count of the whole changed assignment."""
    cl = low.parent.copy()
    s = cl[u]
    before = O.outer_volume(P.occ, up.n[[s, k]], up.bnd[[s, k]])[0].astype(np.int64).sum()
    cl[u] = k
    assign = cl[low.assign]
    bnd = O.tight_bounds(P.U, P.F, assign, up.K, up.n)
    after = O.outer_volume(P.occ, up.n[[s, k]], bnd[[s, k]])[0].astype(np.int64).sum()
    return before - after


def test_converged_units_admit_no_improving_move():
    P = _blobs()
    P.occ.fill_all()
    layers = O.build_tree(P, 5, iters=0)
    up, low = layers[4], layers[5]
    tot0 = int(up.obv.astype(np.int64).sum())
    st = O.unit_moves(P, up, low, 64)
    assert st[-1]["accepted"] == 0                      # converged within the cap
    tot1 = int(up.obv.astype(np.int64).sum())
    assert tot0 - tot1 == sum(s["gain"] for s in st)    # exact bookkeeping
    assert sum(s["accepted"] for s in st) > 0
    # nesting and state consistency
    assert np.array_equal(up.assign, low.parent[low.assign])
    assert np.array_equal(up.bnd, O.tight_bounds(P.U, P.F, up.assign, up.K, up.n))
    assert np.array_equal(up.obv, O.outer_volume(P.occ, up.n, up.bnd)[0])
    # local optimality certificate, by brute force over every legal unit move
    usize = np.bincount(low.parent, minlength=up.K)
    checked = 0
    for u in range(low.K):
        s = low.parent[u]
        if usize[s] < 2:
            continue
        tris = np.nonzero(low.assign == u)[0]
        ks = {int(low.parent[low.assign[t2]]) for t in tris for t2 in P.adj[t]}
        for k in sorted(ks):
            if k == s or up.parent[k] != up.parent[s]:
                continue
            assert _brute_gain(P, up, low, u, k) <= 0
            checked += 1
    assert checked > 0


def test_sweeps_never_raise_eq7_and_keep_the_tree_nested():
    P = _blobs()
    layers = O.build_tree(P, 5, iters=1)
    hist = O.tree_sweeps(P, layers, sweeps=2, iters=2, rounds=8)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < hist[0]
    for lev in range(1, len(layers)):
        up, low = layers[lev - 1], layers[lev]
        assert np.array_equal(up.assign, low.parent[low.assign])
        assert np.all(np.bincount(low.assign, minlength=low.K) > 0)
        assert np.array_equal(low.obv, O.outer_volume(P.occ, low.n, low.bnd)[0])
    assert np.isclose(hist[-1], O.tree_eq7(layers))
