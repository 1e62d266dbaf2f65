"""Member lists of the Lloyd step (Sec. 4.2.1): every cluster's triangles in
ascending index order, i.e. the stable sort of the assignment -- a definition
that numpy's stable argsort states directly.  The library builds the lists
with its own radix sort over tiles of 4,096 triangles, digits of at most 10
bits: one pass for at most 1,024 clusters, two for up to 2^20, three beyond.
The cases cover each pass count at its boundaries, digit-count tables scanned
by the counting kernel's last block and by the two-pass scan, a ragged last
tile, assignments in long runs (whole warps of one cluster) and scattered
ones, and the lists after Lloyd moves."""
import numpy as np
import pytest

from synth import meshes as M

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


def _assignment(T, K, seed, runs):
    """Every cluster non-empty.  runs: consecutive triangles share a cluster
    (as spatial clusters of a mesh do), cut at random places; otherwise each
    triangle draws its cluster independently."""
    rng = np.random.default_rng(seed)
    if runs:
        cuts = np.sort(rng.choice(np.arange(1, T), K - 1, replace=False)) if K > 1 else np.zeros(0, np.int64)
        a = np.zeros(T, np.int64)
        a[cuts] = 1
        a = np.cumsum(a)
        a = rng.permutation(K)[a]          # run order unrelated to cluster order
    else:
        a = rng.integers(0, K, T)
        a[rng.permutation(T)[:K]] = np.arange(K)
    return a.astype(np.int32)


def _expect(assign, K):
    members = np.argsort(assign, kind="stable").astype(np.int32)
    start = np.concatenate([[0], np.cumsum(np.bincount(assign, minlength=K))]).astype(np.int32)
    return members, start


def _check(ctx, lat, assign, K):
    layer = ctx.layer_init(lat, assign, np.zeros(K, np.int32))
    try:
        members, start = ctx.layer_members(layer)
        em, es = _expect(assign, K)
        np.testing.assert_array_equal(start, es)
        np.testing.assert_array_equal(members, em)
    finally:
        layer.free()


@pytest.fixture(scope="module")
def small(ctx):
    m = M.torus(nu=50, nv=30, jitter=0.002, seed=3)   # 3,000 triangles: one ragged tile
    mesh = ctx.mesh_create(m.verts, m.tris)
    return ctx.build_occupancy(mesh, 48), len(m.tris)


@pytest.fixture(scope="module")
def large(ctx):
    m = M.sdf_union_200k()                              # 202,244 triangles: 49 tiles + a ragged one
    mesh = ctx.mesh_create(m.verts, m.tris)
    return ctx.build_occupancy(mesh, 128), len(m.tris)


@pytest.mark.parametrize("K", [1, 2, 31, 256, 257, 1024, 1025, 2999, 3000])
@pytest.mark.parametrize("runs", [True, False])
def test_members_small(ctx, small, K, runs):
    lat, T = small
    _check(ctx, lat, _assignment(T, K, 100 + K, runs), K)


@pytest.mark.parametrize("K", [64, 256, 1024, 4096, 65536, 65537, 150000])
@pytest.mark.parametrize("runs", [True, False])
def test_members_large(ctx, large, K, runs):
    lat, T = large
    _check(ctx, lat, _assignment(T, K, 200 + K, runs), K)


@pytest.mark.parametrize("runs", [True, False])
def test_members_three_passes(ctx, runs):
    """More than 2^20 clusters: three passes of 7 bits."""
    m = M.sdf_union_1m()                                # 1,059,784 triangles
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, 64)
    K = (1 << 20) + 4321
    _check(ctx, lat, _assignment(len(m.tris), K, 300, runs), K)


def test_members_after_lloyd_moves(ctx, large):
    """The lists the step rebuilds after moving rounds are the stable sort of
    the assignment it ends with."""
    lat, T = large
    tree = ctx.build_tree(lat, 8, 0)
    leaf = ctx.tree_read(tree, 8)
    K = len(leaf["frames"])
    layer = ctx.layer_init(lat, leaf["assign"], (np.arange(K) // 2).astype(np.int32), leaf["frames"])
    try:
        moved = 0
        for _ in range(3):
            moved += ctx.lloyd_step(layer, rounds=4, refit=True)["moves"]
        assert moved > 0
        assign = ctx.layer_read(layer)["assign"]
        members, start = ctx.layer_members(layer)
        em, es = _expect(assign, K)
        np.testing.assert_array_equal(start, es)
        np.testing.assert_array_equal(members, em)
    finally:
        layer.free()
        tree.free()


def test_layer_read_into_caller_arrays(ctx, small):
    """layer_read(out=...) fills the caller's arrays with what it returns
    otherwise, and refuses arrays of the wrong shape or type."""
    lat, T = small
    K = 37
    layer = ctx.layer_init(lat, _assignment(T, K, 5, True), np.zeros(K, np.int32))
    try:
        ref = ctx.layer_read(layer)
        out = {k: np.full_like(v, 0) for k, v in ref.items()}
        got = ctx.layer_read(layer, out=out)
        for k in ref:
            assert got[k] is out[k]
            assert np.array_equal(out[k].view(np.uint8), ref[k].view(np.uint8)), k
        bad = dict(out, obv=np.zeros(K + 1, np.uint64))
        with pytest.raises(ValueError):
            ctx.layer_read(layer, out=bad)
        bad = dict(out, assign=np.zeros(T, np.int64))
        with pytest.raises(ValueError):
            ctx.layer_read(layer, out=bad)
    finally:
        layer.free()


def test_outer_volume_refuses_unusable_outputs(ctx, small):
    """Caller-provided counts / points must hold K 8-byte integers on the
    boxes' side; anything else is refused before the library writes."""
    import torch
    lat, _ = small
    boxes = np.zeros(5, dtype=[("c", "<f4", (3,)), ("axis0", "<f4", (3,)), ("axis1", "<f4", (3,)),
                               ("half", "<f4", (3,))])
    boxes["axis0"] = (1, 0, 0)
    boxes["axis1"] = (0, 1, 0)
    boxes["half"] = 0.2
    ref = ctx.outer_volume(lat, boxes)
    out = np.zeros(5, np.uint64)
    got = ctx.outer_volume(lat, boxes, counts=out)
    assert got is out and np.array_equal(out, ref)
    for bad in (np.zeros(4, np.uint64), np.zeros(5, np.int32), np.zeros(10, np.uint64)[::2],
                torch.zeros(5, dtype=torch.int64, device="cuda")):
        with pytest.raises(ValueError):
            ctx.outer_volume(lat, boxes, counts=bad)
    d = torch.from_numpy(boxes.view(np.float32).reshape(5, 12)).cuda()
    with pytest.raises(ValueError):
        ctx.outer_volume(lat, d, counts=torch.zeros(4, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        ctx.outer_volume(lat, d, counts=np.zeros(5, np.uint64))


def test_members_across_lloyd_flood_lloyd(ctx, large):
    """Lists updated from Lloyd moves, then re-sorted after a flooding
    re-partition (which keeps no move records), then updated again: each
    time the stable sort of the current assignment."""
    lat, T = large
    tree = ctx.build_tree(lat, 7, 0)
    leaf = ctx.tree_read(tree, 7)
    K = len(leaf["frames"])
    layer = ctx.layer_init(lat, leaf["assign"], (np.arange(K) // 2).astype(np.int32), leaf["frames"])

    def check():
        assign = ctx.layer_read(layer)["assign"]
        members, start = ctx.layer_members(layer)
        em, es = _expect(assign, K)
        np.testing.assert_array_equal(start, es)
        np.testing.assert_array_equal(members, em)

    try:
        moved = ctx.lloyd_step(layer, rounds=3, refit=False)["moves"]
        check()
        ctx.flood_partition(layer, mode=1)
        check()
        for _ in range(2):
            moved += ctx.lloyd_step(layer, rounds=2, refit=True)["moves"]
            check()
        assert moved > 0
    finally:
        layer.free()
        tree.free()
