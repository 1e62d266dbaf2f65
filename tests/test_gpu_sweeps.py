"""GPU parity of the moves between levels (Sec. 4.2.2, bottom-up merging with
boxes as units) and of the reciprocating sweeps, against the oracle."""
import numpy as np
import pytest

import oracle as O
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


@pytest.fixture(scope="module")
def blobs(ctx):
    """6 spheres and 3 capsules, about 2k triangles, on a 32^3 lattice."""
    m = M.sdf_union_mesh(7, 14, n_spheres=6, n_capsules=3)
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, 32)
    P = O.Problem(m.verts, m.tris, 32)
    yield m, mesh, lat, P
    lat.free()
    mesh.free()


def _gpu_layer(ctx, lat, L):
    return ctx.layer_init(lat, L.assign, L.parent, L.frames)


@pytest.mark.parametrize("level", [2, 3, 4])
def test_unit_step_bit_exact(ctx, blobs, level):
    m, mesh, lat, P = blobs
    layers = O.build_tree(P, 5, iters=0)
    up, low = layers[level].copy(), layers[level + 1].copy()
    gu, gl = _gpu_layer(ctx, lat, up), _gpu_layer(ctx, lat, low)
    st = ctx.unit_step(gu, gl, rounds=64, refit=False)
    so = O.unit_moves(P, up, low, 64)
    g = ctx.layer_read(gu)
    assert np.array_equal(ctx.layer_parents(gl), low.parent)
    assert np.array_equal(g["assign"], up.assign)
    assert np.array_equal(g["qboxes"]["b"], up.bnd) and np.array_equal(g["obv"], up.obv)
    assert st["moves"] == sum(s["accepted"] for s in so)
    assert st["gain"] == sum(s["gain"] for s in so)
    assert st["proposals"] == sum(s["proposals"] for s in so)
    assert st["box_evals"] == sum(s["evals"] for s in so)
    assert st["rounds_run"] == len(so)
    gu.free()
    gl.free()


def test_unit_step_with_single_triangle_units_is_the_triangle_step(ctx, blobs):
    m, mesh, lat, P = blobs
    layers = O.build_tree(P, 4, iters=0)
    L = layers[4]
    T = P.F.shape[0]
    a, b = _gpu_layer(ctx, lat, L), _gpu_layer(ctx, lat, L)
    frames = np.tile(np.eye(3).reshape(1, 9), (T, 1))
    units = ctx.layer_init(lat, np.arange(T, dtype=np.int32), L.assign, frames)
    st_t = ctx.lloyd_step(a, rounds=32, refit=False)
    st_u = ctx.unit_step(b, units, rounds=32, refit=False)
    ga, gb = ctx.layer_read(a), ctx.layer_read(b)
    assert st_t["moves"] > 0
    for k in ("moves", "gain", "proposals", "box_evals", "rounds_run", "total_obv"):
        assert st_t[k] == st_u[k], k
    assert np.array_equal(ga["assign"], gb["assign"]) and np.array_equal(ga["obv"], gb["obv"])
    assert np.array_equal(ctx.layer_parents(units), gb["assign"])
    for h in (a, b, units):
        h.free()


def test_unit_step_rejects_layers_that_do_not_nest(ctx, blobs):
    import paper_2203_10521_gb300 as PK
    m, mesh, lat, P = blobs
    layers = O.build_tree(P, 3, iters=0)
    up, low = layers[2], layers[3]
    bad_parent = low.parent.copy()
    bad_parent[0] = (bad_parent[0] + 1) % up.K
    gu = _gpu_layer(ctx, lat, up)
    gl = ctx.layer_init(lat, low.assign, bad_parent, low.frames)
    with pytest.raises(PK.ObbError):
        ctx.unit_step(gu, gl, refit=False)
    gu.free()
    gl.free()


def _tree_snapshot(ctx, tree, P):
    """The oracle's layers rebuilt from a GPU tree (assignments, parent maps, frames)."""
    out = []
    for lev in range(tree.depth + 1):
        r = ctx.tree_read(tree, lev)
        out.append(O.layer_from_frames(P, r["assign"], ctx.tree_parents(tree, lev), r["frames"]))
    return out


def test_tree_sweep_integer_path_bit_exact(ctx, blobs):
    """Without the floating-point refit every step is exact integers: the GPU
    sweeps must reproduce the oracle's sweeps from the same tree bit for bit."""
    m, mesh, lat, P = blobs
    tree = ctx.build_tree(lat, 5, 1)
    layers = _tree_snapshot(ctx, tree, P)
    assert len(layers) == 6
    hist = O.tree_sweeps(P, layers, sweeps=2, iters=2, rounds=16, do_refit=0)
    st = ctx.tree_sweep(tree, sweeps=2, iters=2, rounds=16, refit=0)
    assert st["eq7_before"] == hist[0] and st["eq7_after"] == hist[-1]
    assert st["unit_moves"] + st["triangle_moves"] > 0
    for lev, L in enumerate(layers):
        r = ctx.tree_read(tree, lev)
        assert np.array_equal(r["assign"], L.assign), lev
        assert np.array_equal(ctx.tree_parents(tree, lev), L.parent), lev
        assert np.array_equal(r["qboxes"]["b"], L.bnd) and np.array_equal(r["obv"], L.obv), lev
    tree.free()


def test_tree_sweep_with_refit(ctx, blobs):
    """With the covariance refit (compensated FP32 on the GPU, FP64 in the
    oracle) the sweeps lower Eq. 7, keep the tree nested, and end within 0.5%
    of the oracle's sweeps from the same tree."""
    m, mesh, lat, P = blobs
    tree = ctx.build_tree(lat, 5, 1)
    layers = _tree_snapshot(ctx, tree, P)
    hist = O.tree_sweeps(P, layers, sweeps=2, iters=2, rounds=16, do_refit=1)
    st = ctx.tree_sweep(tree, sweeps=2, iters=2, rounds=16, refit=1)
    assert st["eq7_after"] < st["eq7_before"]
    assert abs(st["eq7_after"] - hist[-1]) <= 0.005 * hist[-1]
    prev = None
    for lev in range(6):
        r = ctx.tree_read(tree, lev)
        par = ctx.tree_parents(tree, lev)
        if prev is not None:
            assert np.array_equal(prev, par[r["assign"]]), lev
        assert np.all(np.bincount(r["assign"], minlength=1 << lev) > 0)
        ref, _ = O.outer_volume(P.occ, r["qboxes"]["n"], r["qboxes"]["b"])
        assert np.array_equal(r["obv"], ref), lev
        prev = r["assign"]
    pts, _ = ctx.tree_score(tree)
    assert pts == st["eq7_after"]
    tree.free()
