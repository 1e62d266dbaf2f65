"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Integer results must match bit for bit."""
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


def _rot(rng):
    return pins.random_rotation(rng)


def random_boxes(rng, K, center_lo, center_hi, half_lo, half_hi):
    out = np.zeros((K, 12), dtype=np.float32)
    for i in range(K):
        R = _rot(rng)
        out[i, :3] = rng.uniform(center_lo, center_hi)
        out[i, 3:6] = R[0]
        out[i, 6:9] = R[1]
        out[i, 9:12] = rng.uniform(half_lo, half_hi, 3)
    return out


# ---------------------------------------------------------------- occupancy

@pytest.mark.parametrize("name,N", [("torus", 64), ("torus", 37), ("ico", 100), ("ico", 129),
                                    ("sdf", 96), ("cube", 1), ("cube", 5)])
def test_occupancy_bit_exact(ctx, name, N):
    if name == "torus":
        m = M.torus_4096()
    elif name == "ico":
        m = M.icosphere(3, radius=1.0)
    elif name == "sdf":
        m = M.sdf_union_mesh(5, 24, 6, 3, 0)
    else:
        m = M.cube((0, 0, 0), (1.0, 2.0, 0.5))
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N)
    assert np.array_equal(lat.lo, P.lo) and np.array_equal(lat.spacing, P.h)
    assert np.array_equal(lat.fixed().cpu().numpy(), P.U)
    if N <= 100:
        P.occ.fill_all()
        assert np.array_equal(lat.bits(), P.occ.occ)
    else:
        rng = np.random.Generator(np.random.PCG64(N))
        cols = rng.integers(0, N, size=(400, 2))
        P.occ.fill_columns(cols)
        bits = lat.bits()
        for j, k in cols:
            assert np.array_equal(bits[k, j], P.occ.occ[k, j])
    # padding bits of every row are zero
    w = lat.words().cpu().numpy().view(np.uint64).reshape(N, N, lat.W)
    b = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    assert not b[..., N:].any()
    lat.free()
    mesh.free()


def test_occupancy_tie_rules(ctx):
    """Faces through lattice points: the half-open closed form of the oracle pin."""
    N = 12
    outer = M.cube((0, 0, 0), (N, N, N))
    inner = M.cube((2.5, 3.5, 4.5), (7.5, 9.5, 8.5))
    V = np.concatenate([outer.verts, inner.verts])
    F = np.concatenate([outer.tris, inner.tris + 8])
    mesh = ctx.mesh_create(V, F)
    lat = ctx.build_occupancy(mesh, N)
    expect = np.ones((N, N, N), dtype=np.uint8)
    expect[4:8, 3:9, 2:7] = 0
    assert np.array_equal(lat.bits(), expect)


def test_occupancy_config_200k_sampled_columns(ctx):
    """The ~200k-triangle SDF union on a 512^3 lattice: sampled rows bit-exact."""
    m = M.sdf_union_200k()
    N = 512
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    assert np.array_equal(lat.fixed().cpu().numpy(), P.U)
    rng = np.random.Generator(np.random.PCG64(2000))
    cols = rng.integers(0, N, size=(256, 2))
    P.occ.fill_columns(cols)
    w = lat.words().cpu().numpy().view(np.uint64).reshape(N, N, lat.W)
    for j, k in cols:
        row = np.unpackbits(w[k, j].view(np.uint8), bitorder="little")[:N]
        assert np.array_equal(row, P.occ.occ[k, j])


# ------------------------------------------------------------- outer volume

@pytest.fixture(scope="module")
def torus_setup(ctx):
    m = M.torus_4096()
    N = 64
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N)
    P.occ.fill_all()
    return m, mesh, lat, P


def test_quantize_bit_exact(ctx, torus_setup):
    m, mesh, lat, P = torus_setup
    rng = np.random.Generator(np.random.PCG64(5))
    boxes = random_boxes(rng, 500, [-1.5, -1.5, -0.5], [1.5, 1.5, 0.5], 0.0, 0.8)
    q = ctx.quantize_boxes(lat, boxes)
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    assert np.array_equal(q["n"], n) and np.array_equal(q["b"], bnd)


@pytest.mark.parametrize("K,scale", [(1, 0.3), (37, 0.05), (1000, 0.4), (300, 1.6)])
def test_outer_volume_bit_exact(ctx, torus_setup, K, scale):
    m, mesh, lat, P = torus_setup
    rng = np.random.Generator(np.random.PCG64(K))
    boxes = random_boxes(rng, K, [-1.6, -1.6, -0.6], [1.6, 1.6, 0.6], 0.0, scale)
    cnt, pts = ctx.outer_volume(lat, boxes, want_points=True)
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    ref, tot = O.outer_volume(P.occ, n, bnd)
    assert np.array_equal(cnt, ref)
    assert np.array_equal(pts, tot)


def test_outer_volume_device_arrays_and_qboxes(ctx, torus_setup):
    import torch
    m, mesh, lat, P = torus_setup
    rng = np.random.Generator(np.random.PCG64(77))
    boxes = random_boxes(rng, 200, [-1, -1, -0.3], [1, 1, 0.3], 0.05, 0.5)
    d = torch.from_numpy(boxes).cuda()
    cnt = ctx.outer_volume(lat, d)
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    ref, _ = O.outer_volume(P.occ, n, bnd)
    assert np.array_equal(cnt.cpu().numpy().astype(np.uint64), ref)
    q = ctx.quantize_boxes(lat, boxes)
    assert np.array_equal(ctx.outer_volume_q(lat, q), ref)


def test_outer_volume_edge_cases(ctx, torus_setup):
    m, mesh, lat, P = torus_setup
    import paper_2203_10521_gb300 as PK
    # K = 0
    assert len(ctx.outer_volume(lat, np.zeros((0, 12), np.float32))) == 0
    # zero-extent box, box far outside the lattice, axis-aligned box over the whole domain
    eye = np.eye(3, dtype=np.float32)
    boxes = np.array([
        np.concatenate([[0.5, 0.5, 0.0], eye[0], eye[1], [0, 0, 0]]),
        np.concatenate([[9.0, 9.0, 3.0], eye[0], eye[1], [0.2, 0.3, 0.1]]),
        np.concatenate([[0.0, 0.0, 0.0], eye[0], eye[1], [1.4, 1.4, 0.33]]),
    ], dtype=np.float32)
    cnt, pts = ctx.outer_volume(lat, boxes, want_points=True)
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    ref, tot = O.outer_volume(P.occ, n, bnd)
    assert np.array_equal(cnt, ref) and np.array_equal(pts, tot)
    assert cnt[1] == pts[1] > 0
    # invalid boxes are rejected
    bad = boxes.copy()
    bad[0, 9] = -1.0
    with pytest.raises(PK.ObbError) as e:
        ctx.outer_volume(lat, bad)
    assert e.value.code == -1
    bad = boxes.copy()
    bad[1, 0] = np.nan
    with pytest.raises(PK.ObbError):
        ctx.outer_volume(lat, bad)
    # the context stays usable
    assert np.array_equal(ctx.outer_volume(lat, boxes), ref)


@pytest.mark.parametrize("name,N", [("torus", 64), ("sdf", 37), ("ico", 100)])
def test_outer_volume_every_row_axis(ctx, name, N):
    """The lattice's copies with rows along x, y and z (bit transposes of one
    occupancy) give the oracle's exact counts on rotated boxes, for every
    forced row axis and for the per-box choice."""
    if name == "torus":
        m = M.torus_4096()
    elif name == "ico":
        m = M.icosphere(3, radius=1.0)
    else:
        m = M.sdf_union_mesh(5, 24, 6, 3, 0)
    mesh = ctx.mesh_create(m.verts, m.tris)
    ctx.set_counting_axis(-1)   # lattices built from now on keep their y- and z-row copies
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N)
    P.occ.fill_all()
    rng = np.random.Generator(np.random.PCG64(300 + N))
    lo, hi = m.verts.min(0), m.verts.max(0)
    ext = hi - lo
    boxes = random_boxes(rng, 200, lo - 0.1 * ext, hi + 0.1 * ext, 0.0, 0.45 * float(ext.max()))
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    ref, tot = O.outer_volume(P.occ, n, bnd)
    try:
        for axis in (0, 1, 2, -1):
            ctx.set_counting_axis(axis)
            cnt, pts = ctx.outer_volume(lat, boxes, want_points=True)
            assert np.array_equal(cnt, ref), axis
            assert np.array_equal(pts, tot), axis
        # a rebuild refreshes the copies
        ctx.set_counting_axis(2)
        ctx.occupancy_rebuild(lat)
        assert np.array_equal(ctx.outer_volume(lat, boxes), ref)
    finally:
        ctx.set_counting_axis(0)
    lat.free()
    mesh.free()


def _steep_qboxes():
    """Boxes thousands of rows tall whose third slab is almost parallel to x
    (|n_20| of a few dozen against n_22 = +-2^24): its quotient bounds start far
    beyond +-2^30 and move by ~2^24 per row of a one-lane-wide tile."""
    import paper_2203_10521_gb300 as PK
    big = 1 << 24
    kl, kh = -3000, 5000
    rows = []
    # |n_20| >= 32 steps by DDA; 0 < |n_20| < 32 is clipped exactly per row
    for s0, s2, jrow in [(40, 1, 30), (-40, 1, 12), (33, -1, 47), (-127, -1, 5), (5, 1, 20), (-7, -1, 40)]:
        q = np.zeros((), PK.QBOX_DTYPE)
        q["n"] = [big, 0, 0, 50, big, 0, s0, 0, s2 * big]
        z = sorted([s2 * big * kl, s2 * big * kh])
        lq = [10 * big, jrow * big, z[0] - 5000]
        hq = [20 * big, jrow * big + 2000, z[1] + 5000]
        q["b"] = [v for a in range(3) for v in (256 * lq[a], 256 * hq[a])]
        rows.append(q)
    return np.array(rows, dtype=PK.QBOX_DTYPE)


def test_outer_volume_steep_slabs_tall_tiles(ctx, torus_setup):
    """Exact at every tile height, up to 128 rows per lane: a saturated quotient
    must not drift back into the box's x-range within a tile."""
    m, mesh, lat, P = torus_setup
    q = _steep_qboxes()
    ref, tot = O.outer_volume(P.occ, q["n"], q["b"])
    assert (tot > 50000).all()
    try:
        for tk in (32, 64, 128, 7):
            ctx.set_counting_tile(tk)
            cnt, pts = ctx.outer_volume_q(lat, q, want_points=True)
            assert np.array_equal(cnt, ref), tk
            assert np.array_equal(pts, tot), tk
    finally:
        ctx.set_counting_tile(32)


def test_outer_volume_config_200k_sampled(ctx):
    """512^3 lattice of the 200k-triangle mesh: leaf-sized boxes, exact."""
    m = M.sdf_union_200k()
    N = 512
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    rng = np.random.Generator(np.random.PCG64(2001))
    boxes = random_boxes(rng, 24, [0.0, 0.1, 0.1], [1.0, 0.9, 0.9], 0.01, 0.06)
    cnt = ctx.outer_volume(lat, boxes)
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    ref, _ = O.outer_volume(P.occ, n, bnd)
    assert np.array_equal(cnt, ref)


def test_mesh_validation(ctx):
    import paper_2203_10521_gb300 as PK
    m = M.cube()
    with pytest.raises(PK.ObbError) as e:
        ctx.mesh_create(m.verts, m.tris[:-1])
    assert e.value.code == -2
    mesh = ctx.mesh_create(m.verts, m.tris)
    with pytest.raises(PK.ObbError) as e:
        ctx.build_occupancy(mesh, 4096)
    assert e.value.code == -3
    # checks made on the device while the mesh is uploaded
    bad = m.tris.copy()
    bad[3, 1] = 99
    with pytest.raises(PK.ObbError) as e:
        ctx.mesh_create(m.verts, bad)
    assert e.value.code == -1 and "out of range" in str(e.value)
    V = m.verts.copy()
    V[2, 1] = np.nan
    with pytest.raises(PK.ObbError) as e:
        ctx.mesh_create(V, m.tris)
    assert e.value.code == -1 and "non-finite" in str(e.value)
    bad = m.tris.copy()
    bad[5, 2] = bad[5, 0]
    with pytest.raises(PK.ObbError) as e:
        ctx.mesh_create(m.verts, bad)
    assert e.value.code == -2 and "repeated" in str(e.value)
    three = np.concatenate([m.tris, m.tris[:1]])          # one edge set shared by three triangles
    with pytest.raises(PK.ObbError) as e:
        ctx.mesh_create(m.verts, three)
    assert e.value.code == -2 and "shared by 3" in str(e.value)
    # the reported edge is the smallest of the repeated triangle's edges
    t = three[-1]
    edges = sorted((min(t[q], t[(q + 1) % 3]), max(t[q], t[(q + 1) % 3])) for q in range(3))
    assert f"edge ({edges[0][0]}, {edges[0][1]})" in str(e.value)


# -------------------------------------------------------------------- Lloyd

def _wedges(m, K):
    c = m.verts[m.tris].mean(1)
    ang = np.arctan2(c[:, 1], c[:, 0])
    return np.minimum(((ang + np.pi) / (2 * np.pi) * K).astype(np.int32), K - 1)


@pytest.mark.parametrize("K,rounds", [(2, 2), (8, 1), (16, 3), (16, 16), (48, 3)])
def test_lloyd_moves_bit_exact(ctx, torus_setup, K, rounds):
    """The partition rounds' moves, boxes and statistics equal the oracle's
    (Eq. 11-13) on the 4,096-triangle torus; the cluster extents run with a
    block per cluster at K = 2 (2,048 triangles a cluster) and a warp per
    cluster at K = 8, 16 and 48 (512 to 85)."""
    m, mesh, lat, P = torus_setup
    assign = _wedges(m, K)
    parent = (np.arange(K) // 2).astype(np.int32)
    frames = O.cluster_frames(P.V, P.F, assign, K, P.center)
    layer = ctx.layer_init(lat, assign, parent, frames)
    g0 = ctx.layer_read(layer)
    L = O.layer_from_frames(P, assign, parent, frames)
    assert np.array_equal(g0["qboxes"]["n"], L.n) and np.array_equal(g0["qboxes"]["b"], L.bnd)
    assert np.array_equal(g0["obv"], L.obv)
    st = ctx.lloyd_step(layer, rounds=rounds, refit=False)
    so = O.lloyd_moves(P, L, rounds)
    g = ctx.layer_read(layer)
    assert np.array_equal(g["assign"], L.assign)
    assert np.array_equal(g["qboxes"]["b"], L.bnd)
    assert np.array_equal(g["obv"], L.obv)
    assert st["moves"] == sum(s["accepted"] for s in so)
    assert st["gain"] == sum(s["gain"] for s in so)
    assert st["proposals"] == sum(s["proposals"] for s in so)
    assert st["box_evals"] == sum(s["evals"] for s in so)
    assert st["total_obv"] == int(L.obv.sum())
    layer.free()


def test_refit_matches_oracle(ctx, torus_setup):
    """Refit frames within 1e-5 of the FP64 oracle (compensated FP32 sums);
    counts of the refit boxes cross-checked by the oracle on the GPU's boxes."""
    m, mesh, lat, P = torus_setup
    K = 8
    assign = _wedges(m, K)
    parent = np.zeros(K, np.int32)
    rng = np.random.Generator(np.random.PCG64(1))
    frames = np.stack([_rot(rng).reshape(9) for _ in range(K)])
    layer = ctx.layer_init(lat, assign, parent, frames)
    st = ctx.lloyd_step(layer, rounds=1, refit=True)
    g = ctx.layer_read(layer)
    # frames: every cluster's covariance frame vs the oracle's
    ref = O.cluster_frames(P.V, P.F, g["assign"], K, P.center)
    kept = np.any(g["frames"] != frames, axis=1)
    assert kept.sum() == st["refits_accepted"] > 0
    for k in np.nonzero(kept)[0]:
        Rg = g["frames"][k].reshape(3, 3)
        Ro = ref[k].reshape(3, 3)
        assert np.max(np.abs(Rg - Ro)) <= 1e-5
    # exact counts on the GPU's quantised boxes
    cnt, _ = O.outer_volume(P.occ, g["qboxes"]["n"], g["qboxes"]["b"])
    assert np.array_equal(cnt, g["obv"])
    tb = O.tight_bounds(P.U, P.F, g["assign"], K, g["qboxes"]["n"])
    assert np.array_equal(tb, g["qboxes"]["b"])
    layer.free()


def test_descent_bit_exact(ctx, torus_setup):
    """Rotation-probe descent from identical state: FP64 frames, quantised
    boxes and exact outer volumes match the oracle bit for bit."""
    m, mesh, lat, P = torus_setup
    K = 8
    assign = _wedges(m, K)
    parent = (np.arange(K) // 2).astype(np.int32)
    frames = O.cluster_frames(P.V, P.F, assign, K, P.center)
    layer = ctx.layer_init(lat, assign, parent, frames)
    L = O.layer_from_frames(P, assign, parent, frames)
    for it in range(2):
        st = ctx.lloyd_step(layer, rounds=4, refit=2, descent_steps=3)
        O.lloyd_step(P, L, rounds=4, do_refit=2, descent_steps=3)
        g = ctx.layer_read(layer)
        assert np.array_equal(g["assign"], L.assign)
        assert np.array_equal(g["frames"], L.frames)
        assert np.array_equal(g["qboxes"]["n"], L.n) and np.array_equal(g["qboxes"]["b"], L.bnd)
        assert np.array_equal(g["obv"], L.obv)
    assert st["refits_accepted"] >= 0
    layer.free()


def test_layer_init_covariance_frames(ctx, torus_setup):
    m, mesh, lat, P = torus_setup
    K = 16
    assign = _wedges(m, K)
    parent = np.zeros(K, np.int32)
    layer = ctx.layer_init(lat, assign, parent)
    g = ctx.layer_read(layer)
    ref = O.cluster_frames(P.V, P.F, assign, K, P.center)
    assert np.max(np.abs(g["frames"] - ref)) <= 1e-5
    cnt, _ = O.outer_volume(P.occ, g["qboxes"]["n"], g["qboxes"]["b"])
    assert np.array_equal(cnt, g["obv"])
    layer.free()


def test_split_bit_exact(ctx, torus_setup):
    m, mesh, lat, P = torus_setup
    K = 4
    assign = _wedges(m, K)
    layer = ctx.layer_init(lat, assign, np.zeros(K, np.int32))
    g = ctx.layer_read(layer)
    L = O.Layer(g["assign"], np.zeros(K, np.int32), g["frames"], g["qboxes"]["n"].copy(),
                g["qboxes"]["b"].copy(), g["obv"])
    assert np.array_equal(ctx.layer_split(layer), O.median_split(P, L))
    layer.free()


def test_build_tree_against_oracle(ctx, torus_setup):
    """Top-down tree: nesting and enclosure hold; the per-level total outer
    volume is within 0.5% of the oracle's tree on the same mesh (the two
    differ only through FP32 vs FP64 covariance frames)."""
    m, mesh, lat, P = torus_setup
    depth, iters = 3, 4
    tree = ctx.build_tree(lat, depth, iters)
    ref = O.build_tree(P, depth, iters)
    prev = None
    for lev in range(depth + 1):
        g = ctx.tree_read(tree, lev)
        K = 1 << lev
        assert np.all(np.bincount(g["assign"], minlength=K) > 0)
        if prev is not None:
            assert np.array_equal(g["assign"] // 2, prev)
        prev = g["assign"]
        cnt, _ = O.outer_volume(P.occ, g["qboxes"]["n"], g["qboxes"]["b"])
        assert np.array_equal(cnt, g["obv"])
        tot_g, tot_o = int(g["obv"].sum()), int(ref[lev].obv.sum())
        assert abs(tot_g - tot_o) <= 0.005 * tot_o, (lev, tot_g, tot_o)
    pts, vol = ctx.tree_score(tree)
    assert pts == O.eq7_score([ctx.tree_read(tree, l)["obv"] for l in range(depth + 1)], depth)
    tree.free()


def test_determinism(ctx, torus_setup):
    m, mesh, lat, P = torus_setup
    outs = []
    for _ in range(2):
        tree = ctx.build_tree(lat, 2, 3)
        outs.append([ctx.tree_read(tree, l) for l in range(3)])
        tree.free()
    for a, b in zip(*outs):
        for key in ("assign", "frames", "obv"):
            assert np.array_equal(a[key], b[key])
