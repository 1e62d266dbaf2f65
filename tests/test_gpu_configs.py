"""GPU parity on the large workloads: the ~200k-triangle SDF union on 512^3,
the ~1M-triangle union on 768^3 and the ~2M-triangle union of spheres,
capsules and rounded boxes on 1024^3.  The oracle checks whole lattices and
the boxes of the trees built on them exactly."""
import os

import numpy as np
import pytest

import oracle as O
from synth import meshes as M
from tests import pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2203_10521_gb300 as P
    c = P.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def _small_boxes(rng, K, lo, hi, half_lo, half_hi):
    out = np.zeros((K, 12), dtype=np.float32)
    for i in range(K):
        R = pins.random_rotation(rng)
        out[i, :3] = rng.uniform(lo, hi)
        out[i, 3:6], out[i, 6:9] = R[0], R[1]
        out[i, 9:12] = rng.uniform(half_lo, half_hi, 3)
    return out


@pytest.mark.parametrize("name,N,depth", [("1m", 768, 12), ("2m", 1024, 14)])
def test_large_config_full_parity(ctx, name, N, depth):
    """The ~1M-triangle union on 768^3 and the ~2M-triangle union on 1024^3:
    every occupancy word of the whole lattice equals the oracle's per-point
    parity (padding bits zero), and the boxes of the top four levels of the
    tree built on it (depth 12 / 14), plus up to 160 boxes drawn from every
    lower level, count exactly as the oracle counts them, with their in-domain
    points, in spatial order and in the caller's order."""
    O.set_threads(os.cpu_count() or 1)
    try:
        m = M.sdf_union_1m() if name == "1m" else M.sdf_union_2m()
        assert m.n_tris > (900_000 if name == "1m" else 1_800_000)
        mesh = ctx.mesh_create(m.verts, m.tris)
        lat = ctx.build_occupancy(mesh, N)
        P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
        assert np.array_equal(lat.lo, P.lo) and np.array_equal(lat.spacing, P.h)
        assert np.array_equal(lat.fixed().cpu().numpy(), P.U)
        P.occ.fill_all()
        w = lat.words().cpu().numpy().view(np.uint8).reshape(N, N, 8 * lat.W)
        nb = N // 8
        assert np.array_equal(w[:, :, :nb], np.packbits(P.occ.occ, axis=-1, bitorder="little"))
        assert not w[:, :, nb:].any()
        tree = ctx.build_tree(lat, depth, 1)
        rng = np.random.Generator(np.random.PCG64(N))
        qs = []
        for lev in range(depth + 1):
            q = ctx.tree_read(tree, lev)["qboxes"]
            qs.append(q if lev < 4 else q[rng.choice(len(q), min(len(q), 160), replace=False)])
        q = np.concatenate(qs)
        assert len(q) >= 1024
        ref, tot, dom = O.outer_volume(P.occ, q["n"], q["b"], want_domain=True)
        try:
            for order in (1, 0):    # 1024^3 batches of 1,024 boxes or more: spatial order, then the caller's
                ctx.set_counting_order(order)
                ctx.profile_enable(True)
                cnt, pts = ctx.outer_volume_q(lat, q, want_points=True)
                pr = ctx.profile_read()
                ctx.profile_enable(False)
                assert np.array_equal(cnt, ref) and np.array_equal(pts, tot), order
                assert pr["count_points_in_domain"] == float(dom.sum()), order
        finally:
            ctx.set_counting_order(1)
        tree.free()
        lat.free()
        mesh.free()
    finally:
        O.set_threads(1)


def test_batched_meshes_one_launch(ctx):
    """Many meshes of uneven size (about 1k-100k triangles, lattices 128^3-384^3):
    every box of every mesh counted in one launch, exact against the oracle."""
    batch = M.sdf_batch(10, seed=3000)
    lats, meshes, probs = [], [], []
    for m, N in batch:
        mesh = ctx.mesh_create(m.verts, m.tris)
        meshes.append(mesh)
        lats.append(ctx.build_occupancy(mesh, N))
        probs.append(O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32)))
    rng = np.random.Generator(np.random.PCG64(33))
    qs, which = [], []
    for i, P in enumerate(probs):
        ext = P.lo + P.N * P.h
        boxes = _small_boxes(rng, 12, P.lo + 0.2 * (ext - P.lo), P.lo + 0.8 * (ext - P.lo), 0.01, 0.06)
        qs.append(ctx.quantize_boxes(lats[i], boxes))
        which.append(np.full(12, i, np.int32))
    q = np.concatenate(qs)
    li = np.concatenate(which)
    perm = rng.permutation(len(q))          # interleave the meshes' boxes
    cnt, pts = ctx.outer_volume_multi(lats, q[perm], li[perm], want_points=True)
    for i, P in enumerate(probs):
        sel = li[perm] == i
        ref, tot = O.outer_volume(P.occ, q[perm][sel]["n"], q[perm][sel]["b"])
        assert np.array_equal(cnt[sel], ref) and np.array_equal(pts[sel], tot)
        assert np.array_equal(ctx.outer_volume_q(lats[i], q[perm][sel]), ref)
    import paper_2203_10521_gb300 as PK
    with pytest.raises(PK.ObbError):
        ctx.outer_volume_multi(lats, q[:1], np.array([len(lats)], np.int32))
    for lat, mesh in zip(lats, meshes):
        lat.free()
        mesh.free()


def test_sweeps_at_scale(ctx):
    """The reciprocating sweeps (Sec. 4.2.2) on the ~200k-triangle union at 512^3
    with a depth-10 tree: Eq. 7 drops, the tree stays nested, and sampled leaf
    boxes count exactly as the oracle counts them."""
    m = M.sdf_union_200k()
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, 512)
    tree = ctx.build_tree(lat, 10, 1)
    st = ctx.tree_sweep(tree, sweeps=1, iters=1, rounds=16, refit=1)
    assert st["eq7_after"] < st["eq7_before"]
    assert st["unit_moves"] + st["triangle_moves"] > 0
    prev = None
    for lev in (7, 8, 9, 10):
        r = ctx.tree_read(tree, lev)
        par = ctx.tree_parents(tree, lev)
        if prev is not None:
            assert np.array_equal(prev, par[r["assign"]]), lev
        prev = r["assign"]
    P = O.Problem(m.verts, m.tris, 512, adj=np.zeros((m.n_tris, 3), np.int32))
    leaf = ctx.tree_read(tree, 10)
    rng = np.random.Generator(np.random.PCG64(21))
    pick = rng.choice(1024, size=3, replace=False)
    q = leaf["qboxes"][pick]
    ref, _ = O.outer_volume(P.occ, q["n"], q["b"])
    assert np.array_equal(leaf["obv"][pick], ref)
    tree.free()
    lat.free()
    mesh.free()


def test_benchmark_batch_against_oracle(ctx):
    """The benchmark's batch at full size: the 2,047 boxes of a depth-10 tree on
    the ~200k-triangle union at 512^3 (up to the whole lattice, so large boxes
    take shared rows and the doubled tile height) count exactly as the oracle
    counts them, box by box, for tile heights 8 to 64, for rows along each axis
    and for the per-box axis, in spatial order and in the caller's order, with
    and without the rank tables; the whole lattice is bit-exact."""
    O.set_threads(os.cpu_count() or 1)
    m = M.sdf_union_200k()
    mesh = ctx.mesh_create(m.verts, m.tris)
    try:
        ctx.set_counting_axis(-1)   # this lattice keeps its y- and z-row copies
        lat = ctx.build_occupancy(mesh, 512)
        ctx.set_counting_axis(0)
        P = O.Problem(m.verts, m.tris, 512, adj=np.zeros((m.n_tris, 3), np.int32))
        P.occ.fill_all()
        assert np.array_equal(lat.bits(), P.occ.occ)
        tree = ctx.build_tree(lat, 10, 2)
        q = np.concatenate([ctx.tree_read(tree, lev)["qboxes"] for lev in range(11)])
        assert len(q) == 2047
        ref, tot = O.outer_volume(P.occ, q["n"], q["b"])
        base, bpts = ctx.outer_volume_q(lat, q, want_points=True)
        assert np.array_equal(base, ref) and np.array_equal(bpts, tot)
        for tk in (8, 16, 64):
            ctx.set_counting_tile(tk)
            c, p = ctx.outer_volume_q(lat, q, want_points=True)
            assert np.array_equal(c, ref) and np.array_equal(p, tot), tk
        ctx.set_counting_tile(32)
        for axis in (1, 2, -1):
            ctx.set_counting_axis(axis)
            c, p = ctx.outer_volume_q(lat, q, want_points=True)
            assert np.array_equal(c, ref) and np.array_equal(p, tot), axis
        ctx.set_counting_axis(0)
        for order, rank in ((0, 1), (0, 0), (1, 0)):   # the caller's order; every word read
            ctx.set_counting_order(order)
            ctx.set_counting_rank(rank)
            c, p = ctx.outer_volume_q(lat, q, want_points=True)
            assert np.array_equal(c, ref) and np.array_equal(p, tot), (order, rank)
    finally:
        ctx.set_counting_axis(0)
        ctx.set_counting_tile(32)
        ctx.set_counting_order(1)
        ctx.set_counting_rank(1)
        O.set_threads(1)
    tree.free()
    lat.free()
    mesh.free()
