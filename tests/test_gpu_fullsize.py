"""GPU parity against the oracle on the paths the counting kernel takes for
large boxes: rows that span many 128-bit chunks (two-word masks, interior
words, rows counted through the rank tables), unclamped full-height tiles,
tiles twice as tall, every row axis and tile height, boxes poking out of the
lattice domain, and the in-domain point accounting (Eq. 4 per box)."""
import os

import numpy as np
import pytest

import oracle as O
from synth import meshes as M
from tests import pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def oracle_threads():
    O.set_threads(os.cpu_count() or 1)
    yield
    O.set_threads(1)


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


def rotated_boxes(rng, K, lo, ext, frac_lo, frac_hi):
    """K rotated FP32 boxes: centres uniform over the domain widened by 10% on
    each side, half extents log-uniform in [frac_lo, frac_hi] of the largest
    domain extent (from a few cells to the whole lattice)."""
    out = np.zeros((K, 12), dtype=np.float32)
    e = float(np.max(ext))
    for i in range(K):
        R = pins.random_rotation(rng)
        out[i, :3] = rng.uniform(lo - 0.1 * ext, lo + 1.1 * ext)
        out[i, 3:6], out[i, 6:9] = R[0], R[1]
        out[i, 9:12] = np.exp(rng.uniform(np.log(frac_lo * e), np.log(frac_hi * e), 3))
    return out


def test_large_boxes_every_axis_and_tile(ctx):
    """A ~5k-triangle union on a 400^3 lattice (rows of 400 points: three full
    128-bit chunks and a ragged fourth): 200 rotated boxes from a few cells to
    beyond the whole lattice, 1,000 leaf-sized ones, the domain box, a large
    interior box and the 127 boxes of a depth-6 tree count exactly as the
    oracle counts them, in spatial order and in the caller's order, with and
    without the rank tables, for rows along x, y, z and per box, at tile
    heights 8, 32 (64 for boxes of at least 16,384 rows) and 128; the
    kernel's in-domain point total equals the oracle's."""
    m = M.sdf_union_mesh(5, 24, 6, 3, 0)
    N = 400
    mesh = ctx.mesh_create(m.verts, m.tris)
    try:
        ctx.set_counting_axis(-1)   # this lattice keeps its y- and z-row copies
        lat = ctx.build_occupancy(mesh, N)
    finally:
        ctx.set_counting_axis(0)
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    P.occ.fill_all()
    assert np.array_equal(lat.bits(), P.occ.occ)
    rng = np.random.Generator(np.random.PCG64(400))
    ext = N * P.h
    boxes = np.concatenate([rotated_boxes(rng, 200, P.lo, ext, 0.004, 0.7),
                            rotated_boxes(rng, 1000, P.lo, ext, 0.004, 0.03)])   # many leaf-sized boxes
    whole = np.zeros((2, 12), np.float32)
    whole[0, :3] = P.lo + 0.5 * ext                      # the domain itself
    whole[0, 9:12] = 0.5 * ext
    whole[1, :3] = P.lo + 0.5 * ext                      # a large box inside the domain
    whole[1, 9:12] = 0.42 * ext
    whole[:, 3], whole[:, 7] = 1.0, 1.0
    q = ctx.quantize_boxes(lat, np.concatenate([boxes, whole]))
    tree = ctx.build_tree(lat, 6, 1)
    q = np.concatenate([q] + [ctx.tree_read(tree, lev)["qboxes"] for lev in range(7)])
    ref, tot, dom = O.outer_volume(P.occ, q["n"], q["b"], want_domain=True)
    assert tot.max() > N ** 3 // 2                    # up to the whole lattice
    assert (tot > dom).sum() >= 20                     # boxes poking out of the domain
    assert (ref < tot).sum() >= 100                    # boxes that meet the solid
    assert len(q) >= 1024                                # a batch counted in spatial order
    try:
        for order in (1, 0):
            ctx.set_counting_order(order)
            for rank in (1, 0):
                ctx.set_counting_rank(rank)
                for axis in (0, 1, 2, -1):
                    ctx.set_counting_axis(axis)
                    for tk in (8, 32, 128):
                        ctx.set_counting_tile(tk)
                        ctx.profile_enable(True)
                        c, p = ctx.outer_volume_q(lat, q, want_points=True)
                        pr = ctx.profile_read()
                        key = (order, rank, axis, tk)
                        assert np.array_equal(c, ref) and np.array_equal(p, tot), key
                        assert pr["count_points_in_domain"] == float(dom.sum()), key
        ctx.set_counting_order(1)
        # coverage: along x the tree's top boxes (rotated, so every slab steps
        # along the row) have rows of several 128-bit chunks; read word by
        # word they take the interior-word loop, and with the rank tables most
        # of their rows are counted from the end words
        ctx.set_counting_axis(0)
        ctx.set_counting_tile(32)
        top = slice(1202, 1202 + 7)
        assert (q["n"][top][:, [0, 3, 6]] != 0).all()
        ctx.set_counting_rank(0)
        ctx.profile_enable(True)
        ctx.outer_volume_q(lat, q[top])
        walk = ctx.profile_read()
        ctx.set_counting_rank(1)
        ctx.profile_enable(True)
        ctx.outer_volume_q(lat, q[top])
        rk = ctx.profile_read()
        print(f"top boxes: {walk['count_bytes'] / walk['count_rows']:.1f} B per row read word by word, "
              f"{rk['count_rows_rank'] / rk['count_rows']:.2f} of rows through the rank table")
        assert walk["count_rows_rank"] == 0 and walk["count_bytes"] / walk["count_rows"] >= 1.5 * 16, walk
        assert rk["count_rows_rank"] >= 0.5 * rk["count_rows"], rk
    finally:
        ctx.profile_enable(False)
        ctx.set_counting_axis(0)
        ctx.set_counting_tile(32)
        ctx.set_counting_rank(1)
        ctx.set_counting_order(1)
    tree.free()
    lat.free()
    mesh.free()


def test_rank_rows_and_walked_rows_agree(ctx):
    """Boxes counted alone and in one batch with boxes of every size give the
    oracle's counts, with and without the rank tables (the choice of a box's
    row counting depends only on the box)."""
    m = M.sdf_union_mesh(5, 24, 6, 3, 0)
    N = 256
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    rng = np.random.Generator(np.random.PCG64(256))
    q = ctx.quantize_boxes(lat, rotated_boxes(rng, 64, P.lo, N * P.h, 0.01, 0.6))
    ref, tot = O.outer_volume(P.occ, q["n"], q["b"])
    try:
        for rank in (1, 0):
            ctx.set_counting_rank(rank)
            batch = ctx.outer_volume_q(lat, q)
            alone = np.array([ctx.outer_volume_q(lat, q[i:i + 1])[0] for i in range(len(q))])
            assert np.array_equal(batch, ref) and np.array_equal(alone, ref), rank
    finally:
        ctx.set_counting_rank(1)
    lat.free()
    mesh.free()
