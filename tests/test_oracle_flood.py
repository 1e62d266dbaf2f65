"""Pins of the oracle's flooding partition (Sec. 4.2.1 step 1, Eq. 12-13)."""
import heapq

import numpy as np

import oracle as O
from synth import meshes as M


def _two_spheres():
    a = M.icosphere(2, center=(0.0, 0.0, 0.0), radius=0.5)
    b = M.icosphere(2, center=(3.0, 0.2, -0.1), radius=0.6)
    V = np.concatenate([a.verts, b.verts]).astype(np.float32)
    F = np.concatenate([a.tris, b.tris + len(a.verts)]).astype(np.int32)
    return O.Problem(V, F, 40), len(a.tris)


def _eye_n(P, K):
    return O.frame_normals(np.tile(np.eye(3).reshape(1, 9), (K, 1)), P.h)


def test_separated_components_fill_their_own_box():
    P, na = _two_spheres()
    T = P.F.shape[0]
    centre = np.array([[0.0, 0.0, 0.0], [3.0, 0.2, -0.1]])
    assign, bnd, obv = O.flood_partition(P, np.zeros(T, np.int32), np.zeros(2, np.int32), _eye_n(P, 2), centre)
    assert np.all(assign[:na] == 0) and np.all(assign[na:] == 1)


def _components(F, adj, tris):
    sel = set(int(t) for t in tris)
    seen, comps = set(), 0
    for t0 in sel:
        if t0 in seen:
            continue
        comps += 1
        stack = [t0]
        seen.add(t0)
        while stack:
            t = stack.pop()
            for u in adj[t]:
                if int(u) in sel and int(u) not in seen:
                    seen.add(int(u))
                    stack.append(int(u))
    return comps


def test_flood_invariants_on_a_tree_level():
    m = M.sdf_union_mesh(7, 14, n_spheres=6, n_capsules=3)
    P = O.Problem(m.verts, m.tris, 32)
    layers = O.build_tree(P, 3, iters=1)
    up, L = layers[2], layers[3]
    group = up.assign
    centre = O.box_centres(P, L)
    assign, bnd, obv = O.flood_partition(P, group, L.parent, L.n, centre)
    T = P.F.shape[0]
    assert np.all(assign >= 0) and np.all(L.parent[assign] == group)      # every triangle, own group
    assert np.all(np.bincount(assign, minlength=L.K) > 0)                  # every box seeded
    assert np.array_equal(bnd, O.tight_bounds(P.U, P.F, assign, L.K, L.n))
    assert np.array_equal(obv, O.outer_volume(P.occ, L.n, bnd)[0])
    # a box grows from its seed through edge neighbours: within a connected
    # group every region is edge-connected
    for g in range(up.K):
        if _components(P.F, P.adj, np.nonzero(group == g)[0]) != 1:
            continue
        for k in np.nonzero(L.parent == g)[0]:
            assert _components(P.F, P.adj, np.nonzero(assign == k)[0]) == 1
    # the first box's seed is the triangle of its group nearest its centre
    c = P.V[P.F].astype(np.float64).sum(1) / 3.0
    d = np.sqrt(((c - centre[0]) ** 2).sum(1)).astype(np.float32)
    d[group != L.parent[0]] = np.inf
    assert assign[int(np.argmin(d))] == 0
    assert T == assign.shape[0]


def test_one_box_per_group_keeps_the_groups():
    m = M.sdf_union_mesh(3, 12, n_spheres=5, n_capsules=2)
    P = O.Problem(m.verts, m.tris, 28)
    layers = O.build_tree(P, 2, iters=0)
    L = layers[2]
    assign, _, obv = O.flood_partition(P, L.assign, np.arange(L.K, dtype=np.int32), L.n, O.box_centres(P, L))
    assert np.array_equal(assign, L.assign) and np.array_equal(obv, L.obv)


def _flood_py(P, group, box_group, n, centre):
    """The same procedure in plain Python (heapq), for a cross-check on tiny meshes."""
    V, F, adj = P.V.astype(np.float64), P.F, P.adj
    T, K = F.shape[0], len(box_group)

    def key(t, k):
        m = (V[F[t, 0]] + V[F[t, 1]]) + V[F[t, 2]]
        m = m / 3.0
        d = m - centre[k]
        d2 = ((0.0 + d[0] * d[0]) + d[1] * d[1]) + d[2] * d[2]
        return float(np.float32(np.sqrt(d2)))

    kt = [min((key(t, k) for k in range(K) if box_group[k] == group[t]), default=np.inf) for t in range(T)]
    assign = -np.ones(T, np.int32)
    members = [[] for _ in range(K)]

    def obv_of(k, tris):
        if not tris:
            return 0
        a = np.full(T, -1, np.int32)
        a[tris] = 0
        b = O.tight_bounds(P.U, P.F, np.where(a >= 0, 0, 1).astype(np.int32), 2, np.stack([n[k], n[k]]))[:1]
        return int(O.outer_volume(P.occ, n[k:k + 1], b)[0][0])

    for k in range(K):
        cands = [(key(t, k), t) for t in range(T) if group[t] == box_group[k] and assign[t] < 0]
        t = min(cands)[1]
        assign[t] = k
        members[k].append(t)
    queued = assign >= 0
    heap = []
    for k in range(K):
        for t in members[k]:
            for u in adj[t]:
                if not queued[u] and group[u] == group[t]:
                    queued[u] = True
                    heapq.heappush(heap, (kt[u], u))
    while (assign < 0).any():
        if heap:
            _, t = heapq.heappop(heap)
        else:
            t = min((kt[u], u) for u in range(T) if assign[u] < 0)[1]
            queued[t] = True
        ks = sorted({int(assign[u]) for u in adj[t] if assign[u] >= 0 and group[u] == group[t]})
        if not ks:
            ks = [k for k in range(K) if box_group[k] == group[t]]
        costs = [obv_of(k, members[k] + [t]) - obv_of(k, members[k]) for k in ks]
        k = ks[int(np.argmin(costs))]
        assign[t] = k
        members[k].append(t)
        for u in adj[t]:
            if not queued[u] and group[u] == group[t]:
                queued[u] = True
                heapq.heappush(heap, (kt[u], u))
    return assign


def test_flood_matches_a_plain_python_restatement():
    m = M.subdivided_tetrahedron(jitter=0.05, seed=2)
    P = O.Problem(m.verts, m.tris, 12)
    P.occ.fill_all()
    T = P.F.shape[0]
    rng = np.random.Generator(np.random.PCG64(9))
    for K in (2, 3):
        R = np.stack([np.linalg.qr(rng.normal(size=(3, 3)))[0] for _ in range(K)])
        R = R * np.sign(np.linalg.det(R))[:, None, None]
        n = O.frame_normals(R.reshape(K, 9), P.h)
        centre = rng.uniform(P.lo, P.lo + P.N * P.h, size=(K, 3))
        got, _, _ = O.flood_partition(P, np.zeros(T, np.int32), np.zeros(K, np.int32), n, centre)
        ref = _flood_py(P, np.zeros(T, np.int32), np.zeros(K, np.int32), n, centre)
        assert np.array_equal(got, ref)
