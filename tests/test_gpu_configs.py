"""GPU parity on the large workloads: the ~1M-triangle SDF union on a 768^3
lattice and the ~2M-triangle union of spheres, capsules and rounded boxes on
1024^3.  The oracle checks sampled occupancy rows and small boxes exactly."""
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


@pytest.mark.parametrize("name,N,ncols,nbox", [("1m", 768, 48, 4), ("2m", 1024, 32, 3)])
def test_large_config_sampled_parity(ctx, name, N, ncols, nbox):
    m = M.sdf_union_1m() if name == "1m" else M.sdf_union_2m()
    assert m.n_tris > (900_000 if name == "1m" else 1_800_000)
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    assert np.array_equal(lat.lo, P.lo) and np.array_equal(lat.spacing, P.h)
    assert np.array_equal(lat.fixed().cpu().numpy(), P.U)
    rng = np.random.Generator(np.random.PCG64(N))
    cols = rng.integers(0, N, size=(ncols, 2))
    P.occ.fill_columns(cols)
    w = lat.words().cpu().numpy().view(np.uint64).reshape(N, N, lat.W)
    for j, k in cols:
        row = np.unpackbits(w[k, j].view(np.uint8), bitorder="little")
        assert np.array_equal(row[:N], P.occ.occ[k, j])
        assert not row[N:].any()
    ext = P.lo + N * P.h
    boxes = _small_boxes(rng, nbox, P.lo + 0.3 * (ext - P.lo), P.lo + 0.7 * (ext - P.lo), 0.004, 0.012)
    cnt, pts = ctx.outer_volume(lat, boxes, want_points=True)
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    ref, tot = O.outer_volume(P.occ, n, bnd)
    assert np.array_equal(cnt, ref) and np.array_equal(pts, tot)
    assert tot.min() > 100
    lat.free()
    mesh.free()


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


def test_benchmark_batch_invariant_at_scale(ctx):
    """The benchmark's batch at full size: the 2,047 boxes of a depth-10 tree on
    the ~200k-triangle union at 512^3 (up to the whole lattice, so large boxes
    take the doubled tile height) count the same, box by box, for every tile
    height, for rows along each axis and for the per-box axis; leaf boxes of
    this tree are checked against the oracle in test_sweeps_at_scale."""
    m = M.sdf_union_200k()
    mesh = ctx.mesh_create(m.verts, m.tris)
    try:
        ctx.set_counting_axis(-1)   # this lattice keeps its y- and z-row copies
        lat = ctx.build_occupancy(mesh, 512)
        ctx.set_counting_axis(0)
        tree = ctx.build_tree(lat, 10, 1)
        q = np.concatenate([ctx.tree_read(tree, lev)["qboxes"] for lev in range(11)])
        assert len(q) == 2047
        base, bpts = ctx.outer_volume_q(lat, q, want_points=True)
        assert (bpts > 0).all() and (base <= bpts).all()
        for tk in (8, 16, 64):
            ctx.set_counting_tile(tk)
            c, p = ctx.outer_volume_q(lat, q, want_points=True)
            assert np.array_equal(c, base) and np.array_equal(p, bpts), tk
        ctx.set_counting_tile(32)
        for axis in (1, 2, -1):
            ctx.set_counting_axis(axis)
            c, p = ctx.outer_volume_q(lat, q, want_points=True)
            assert np.array_equal(c, base) and np.array_equal(p, bpts), axis
    finally:
        ctx.set_counting_axis(0)
        ctx.set_counting_tile(32)
    tree.free()
    lat.free()
    mesh.free()
