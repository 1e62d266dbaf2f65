"""Pins of the oracle's Lloyd step (Sec. 4.2.1, Eq. 11-13), refit pieces and
tree score: brute-force partitions, closed forms, invariants."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O
from synth import meshes as M
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Jacobi ---

def test_jacobi_recovers_known_spectrum():
    rng = np.random.Generator(np.random.PCG64(21))
    for _ in range(50):
        Q = pins.random_rotation(rng)
        d = np.sort(rng.uniform(-3, 5, 3))[::-1]
        A = Q @ np.diag(d) @ Q.T
        R, ev = O.jacobi3([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])
        assert np.allclose(ev, d, rtol=0, atol=1e-14 * np.abs(d).max())
        for a in range(3):
            assert np.linalg.norm(A @ R[a] - ev[a] * R[a]) <= 1e-12 * np.linalg.norm(A)
            assert abs(abs(R[a] @ Q[:, a]) - 1.0) < 1e-12
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert np.linalg.det(R) > 0.999
        for a in range(2):                          # sign canonicalisation
            assert R[a, np.argmax(np.abs(R[a]))] > 0


def test_jacobi_diagonal_input():
    R, ev = O.jacobi3([1.0, 3.0, 2.0, 0.0, 0.0, 0.0])
    assert np.array_equal(ev, [3.0, 2.0, 1.0])
    assert np.array_equal(np.abs(R), np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=float))


# ------------------------------------------------------------- covariance ---

def test_triangle_second_moment_matches_quadrature():
    """A/12 (9 m m^T + p p^T + q q^T + r r^T) equals the edge-midpoint rule,
    which integrates quadratics over a triangle exactly."""
    rng = np.random.Generator(np.random.PCG64(4))
    V = rng.normal(size=(3, 3)).astype(np.float32)
    F = np.array([[0, 1, 2]], dtype=np.int32)
    mom = O.moments(V, F, np.zeros(1, np.int32), 1, np.zeros(3))[0]
    P = V.astype(np.float64)
    A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    mids = [(P[0] + P[1]) / 2, (P[1] + P[2]) / 2, (P[2] + P[0]) / 2]
    S = sum(np.outer(x, x) for x in mids) * A / 3.0
    first = sum(mids) * A / 3.0
    assert np.isclose(mom[0], A, rtol=1e-14)
    assert np.allclose(mom[1:4], first, rtol=1e-13, atol=1e-15)
    packed = [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]
    assert np.allclose(mom[4:], packed, rtol=1e-12, atol=1e-14)


def test_covariance_frame_of_flat_cluster_has_normal_last():
    """A planar patch has zero variance along its normal: third axis = normal."""
    rng = np.random.Generator(np.random.PCG64(8))
    Q = pins.random_rotation(rng)
    pts = np.concatenate([rng.uniform(-1, 1, (30, 2)) * [3, 1], np.zeros((30, 1))], 1) @ Q.T
    F = np.array([[i, i + 1, i + 2] for i in range(0, 27, 3)], dtype=np.int32)
    fr = O.cluster_frames(pts.astype(np.float32), F, np.zeros(len(F), np.int32), 1, np.zeros(3))
    R = fr[0].reshape(3, 3)
    assert abs(abs(R[2] @ Q[:, 2]) - 1) < 1e-6


# ---------------------------------------------------------- brute force ---

def _tiny_problem(name, N):
    if name == "tetra16":
        m = M.subdivided_tetrahedron(jitter=0.15, seed=3)
    else:
        m = M.octahedron(radius=1.0)
        m.verts = (m.verts * np.array([1.0, 0.7, 0.45], dtype=np.float32)
                   + np.random.Generator(np.random.PCG64(2)).uniform(-0.1, 0.1, m.verts.shape)
                   ).astype(np.float32)
    P = O.Problem(m.verts, m.tris, N)
    P.occ.fill_all()
    return P


def _brute_table(P, frames):
    """Sum of OBV for every 2-partition (bit t of the mask = triangle t in
    cluster 1), both clusters non-empty; -1 where one is empty."""
    T = P.F.shape[0]
    n = O.frame_normals(frames, P.h)
    cache = {}
    tbl = np.full(1 << T, -1, dtype=np.int64)
    for mask in range(1, (1 << T) - 1):
        assign = np.array([(mask >> t) & 1 for t in range(T)], dtype=np.int32)
        bnd = O.tight_bounds(P.U, P.F, assign, 2, n)
        tot = 0
        for k in range(2):
            key = (k, tuple(bnd[k]))
            if key not in cache:
                cache[key] = int(O.outer_volume(P.occ, n[k:k + 1], bnd[k:k + 1])[0][0])
            tot += cache[key]
        tbl[mask] = tot
    return tbl


@pytest.mark.parametrize("name,N", [("octa", 14), ("tetra16", 16)])
def test_lloyd_fixed_point_against_brute_force(name, N):
    """From several seeded starts, the partition rounds reach a state that
    (i) is at least the global minimum over all 2-partitions, (ii) admits no
    improving single move to an edge-adjacent cluster (local optimality),
    (iii) lost exactly the sum of the accepted gains, and (iv) stores bounds
    and OBV equal to a from-scratch recomputation."""
    P = _tiny_problem(name, N)
    T = P.F.shape[0]
    rng = np.random.Generator(np.random.PCG64(17))
    frames = np.stack([np.eye(3).reshape(9), pins.random_rotation(rng).reshape(9)])
    tbl = _brute_table(P, frames)
    gmin = tbl[tbl >= 0].min()
    improved_somewhere = False
    for s in range(6):
        a0 = rng.integers(0, 2, T).astype(np.int32)
        if a0.min() == a0.max():
            a0[0] = 1 - a0[0]
        L = O.layer_from_frames(P, a0, np.zeros(2, np.int32), frames)
        start = int(L.obv.sum())
        st = O.lloyd_moves(P, L, rounds=200)
        end = int(L.obv.sum())
        assert start - end == sum(x["gain"] for x in st)
        mask = int(sum(int(L.assign[t]) << t for t in range(T)))
        assert tbl[mask] == end
        assert end >= gmin
        improved_somewhere |= end < start
        ref = O.layer_from_frames(P, L.assign, L.parent, frames)
        assert np.array_equal(ref.bnd, L.bnd) and np.array_equal(ref.obv, L.obv)
        # local optimality over the Lloyd neighbourhood
        for t in range(T):
            src = int(L.assign[t])
            if (L.assign == src).sum() < 2:
                continue
            for nb in P.adj[t]:
                if L.assign[nb] != src:
                    m2 = mask ^ (1 << t)
                    assert tbl[m2] >= end
    assert improved_somewhere


def test_matching_gives_disjoint_clusters_and_exact_drop():
    """On a many-cluster layer each round's accepted moves touch disjoint
    clusters, and the total drops by exactly the sum of their gains."""
    m = M.torus_4096()
    P = O.Problem(m.verts, m.tris, 40)
    P.occ.fill_all()
    T = P.F.shape[0]
    # 16 clusters: wedges around the ring, 2 per parent
    ang = np.arctan2(m.verts[m.tris].mean(1)[:, 1], m.verts[m.tris].mean(1)[:, 0])
    assign = np.minimum(((ang + np.pi) / (2 * np.pi) * 16).astype(np.int32), 15)
    parent = (np.arange(16) // 2).astype(np.int32)
    L = O.layer_init(P, assign, parent)
    for _ in range(3):
        before_assign = L.assign.copy()
        before = int(L.obv.sum())
        st = O.lloyd_moves(P, L, rounds=1)
        moved = np.nonzero(before_assign != L.assign)[0]
        touched = np.concatenate([before_assign[moved], L.assign[moved]])
        assert len(np.unique(touched)) == len(touched)
        # moves stay between siblings
        assert np.all(parent[before_assign[moved]] == parent[L.assign[moved]])
        assert before - int(L.obv.sum()) == st[0]["gain"]
        ref = O.layer_from_frames(P, L.assign, L.parent, L.frames)
        assert np.array_equal(ref.obv, L.obv)


def test_refit_never_increases_and_keeps_enclosure():
    m = M.torus_4096()
    P = O.Problem(m.verts, m.tris, 40)
    P.occ.fill_all()
    ang = np.arctan2(m.verts[m.tris].mean(1)[:, 1], m.verts[m.tris].mean(1)[:, 0])
    assign = np.minimum(((ang + np.pi) / (2 * np.pi) * 8).astype(np.int32), 7)
    parent = np.zeros(8, np.int32)
    # start from deliberately poor frames so the refit has something to fix
    rng = np.random.Generator(np.random.PCG64(1))
    frames = np.stack([pins.random_rotation(rng).reshape(9) for _ in range(8)])
    L = O.layer_from_frames(P, assign, parent, frames)
    before = L.obv.copy()
    acc = O.refit(P, L)
    assert acc.sum() > 0
    assert np.all(L.obv <= before)
    assert np.all(L.obv[acc == 1] < before[acc == 1])
    # Def. 1: every vertex of a cluster lies inside its box
    for t in range(0, P.F.shape[0], 7):
        k = L.assign[t]
        d = P.U[P.F[t]].astype(np.int64) @ L.n[k].reshape(3, 3).astype(np.int64).T
        assert np.all(d >= L.bnd[k, 0::2]) and np.all(d <= L.bnd[k, 1::2])


def test_eq7_score_golden():
    g = json.load(open(os.path.join(GOLDEN, "eq7_weights.json")))
    assert O.eq7_score(g["obv_per_level"], g["depth"]) == g["score"]


def test_build_tree_invariants():
    """Top-down build (Sec. 4.2.2): nested clusters, enclosure, no empty
    cluster, and the Lloyd steps inside never raise a layer's total."""
    m = M.torus_4096()
    P = O.Problem(m.verts, m.tris, 32)
    P.occ.fill_all()
    layers = O.build_tree(P, depth=3, iters=2)
    assert [L.K for L in layers] == [1, 2, 4, 8]
    for lev in range(1, len(layers)):
        L, up = layers[lev], layers[lev - 1]
        assert np.all(np.bincount(L.assign, minlength=L.K) > 0)
        assert np.array_equal(L.parent[L.assign], up.assign)      # nesting
        ref = O.layer_from_frames(P, L.assign, L.parent, L.frames)
        assert np.array_equal(ref.bnd, L.bnd) and np.array_equal(ref.obv, L.obv)
    # a fresh median split + init has a total no lower than after its Lloyd steps
    L1 = layers[1]
    child = O.median_split(P, layers[0])
    init = O.layer_init(P, child, np.zeros(2, np.int32), np.repeat(layers[0].frames, 2, 0))
    assert int(L1.obv.sum()) <= int(init.obv.sum())


def test_median_split_order_and_sizes():
    """Median split (seeding of Sec. 4.2.2): children sizes ceil/floor of the
    parent's, every key of child 2c at most every key of child 2c+1 (key =
    major-axis projection of the fixed-point centroid), ties broken by index."""
    m = M.torus_4096()
    P = O.Problem(m.verts, m.tris, 32)
    P.occ.fill_all()
    K = 4
    c = m.verts[m.tris].mean(1)
    ang = np.arctan2(c[:, 1], c[:, 0])
    assign = np.minimum(((ang + np.pi) / (2 * np.pi) * K).astype(np.int32), K - 1)
    L = O.layer_init(P, assign, np.zeros(K, np.int32))
    child = O.median_split(P, L)
    cen3 = P.U[P.F].astype(np.int64).sum(1)
    for k in range(K):
        mem = np.nonzero(assign == k)[0]
        key = cen3[mem] @ L.n[k, 0:3].astype(np.int64)
        c0 = child[mem] == 2 * k
        assert c0.sum() == (len(mem) + 1) // 2 and (~c0).sum() == len(mem) // 2
        assert np.all(np.isin(child[mem], [2 * k, 2 * k + 1]))
        assert key[c0].max() <= key[~c0].min()
        # ties at the boundary key go to child 0 in ascending triangle order
        b = key[c0].max()
        tied = mem[key == b]
        assert np.all(np.diff(child[tied]) >= 0)


def test_probe_frames_are_exact_rotations():
    """A rotation probe turns the frame about one of its own axes by
    2 atan(t), t = 2^-(5 + level), keeping it orthonormal and right-handed."""
    rng = np.random.Generator(np.random.PCG64(31))
    R = pins.random_rotation(rng)
    for level in (0, 3):
        t = 2.0 ** -(5 + level)
        for p in range(6):
            Q = O.probe_frame(R, level, p)
            a = p // 2
            assert np.allclose(Q @ Q.T, np.eye(3), atol=1e-15)
            assert np.linalg.det(Q) > 0
            assert np.array_equal(Q[a], R[a])
            b1 = (a + 1) % 3
            ang = np.arccos(np.clip(Q[b1] @ R[b1], -1, 1))
            assert abs(ang - 2 * np.arctan(t)) < 1e-9
            sign = 1 if p % 2 == 0 else -1
            assert sign * (Q[b1] @ R[(a + 2) % 3]) > 0


def test_descent_never_increases_and_escalates():
    """Each descent step keeps a box only if its exact outer volume drops;
    clusters that find no better probe halve their angle (level += 1)."""
    m = M.torus_4096()
    P = O.Problem(m.verts, m.tris, 40)
    P.occ.fill_all()
    c = m.verts[m.tris].mean(1)
    ang = np.arctan2(c[:, 1], c[:, 0])
    assign = np.minimum(((ang + np.pi) / (2 * np.pi) * 8).astype(np.int32), 7)
    L = O.layer_init(P, assign, np.zeros(8, np.int32))
    total = [int(L.obv.sum())]
    for _ in range(6):
        before_obv, before_lev = L.obv.copy(), L.level.copy()
        kept = O.descent_step(P, L)
        assert np.all(L.obv <= before_obv)
        improved = L.obv < before_obv
        assert improved.sum() == kept
        assert np.array_equal(L.level[improved], before_lev[improved])
        stuck = ~improved & (before_lev < 8)
        assert np.array_equal(L.level[stuck], before_lev[stuck] + 1)
        total.append(int(L.obv.sum()))
        ref = O.layer_from_frames(P, L.assign, L.parent, L.frames)
        assert np.array_equal(ref.obv, L.obv)
    assert total[-1] < total[0]
