"""Batched Lloyd iterations over many meshes of uneven size (Sec. 4.2.1 per
layer, batched): every layer's exact counts of a round go into one counting
launch over all the lattices.  The batch must reproduce the per-layer
iteration exactly, and its moves are the oracle's."""
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


def batch_depths(meshes, seed):
    """Tree depth per mesh, log-uniform in 6..9 and at most log2(T / 16)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m, _ in meshes:
        d = int(np.floor(np.exp(rng.uniform(np.log(6), np.log(10)))))
        out.append(max(2, min(d, int(np.log2(m.n_tris / 16)))))
    return out


def fresh_leaf_split(ctx, lat, depth):
    """The leaf level of a tree freshly split from its parent level."""
    tree = ctx.build_tree(lat, depth - 1, 1)
    up = ctx.tree_read(tree, depth - 1)
    Kp = 1 << (depth - 1)
    up_layer = ctx.layer_init(lat, up["assign"], (np.arange(Kp) // 2).astype(np.int32), up["frames"])
    child = ctx.layer_split(up_layer)
    up_layer.free()
    tree.free()
    return child, (np.arange(2 * Kp) // 2).astype(np.int32)


def test_batched_lloyd_equals_per_layer_steps(ctx):
    """32 seeded SDF unions (about 1k to 185k triangles, lattices 128^3 to
    384^3, depths 6 to 9): two Lloyd iterations of the whole batch (covariance
    refit, then covariance refit and rotation descent) leave every layer
    exactly as the per-layer iterations do, with the same statistics."""
    meshes = M.sdf_batch(32, seed=3000)
    depths = batch_depths(meshes, 31)
    objs, As, Bs = [], [], []
    for (m, N), d in zip(meshes, depths):
        mesh = ctx.mesh_create(m.verts, m.tris)
        lat = ctx.build_occupancy(mesh, N)
        child, parent = fresh_leaf_split(ctx, lat, d)
        As.append(ctx.layer_init(lat, child, parent))
        Bs.append(ctx.layer_init(lat, child, parent))
        objs.append((mesh, lat))
    assert len(set(depths)) >= 3 and len({N for _, N in meshes}) >= 4
    batch = ctx.batch_create(As)
    for refit, dsteps in ((1, 0), (3, 2)):
        sa = ctx.batch_lloyd_step(batch, rounds=16, refit=refit, descent_steps=dsteps)
        sb = [ctx.lloyd_step(B, rounds=16, refit=refit, descent_steps=dsteps) for B in Bs]
        assert sa == sb, refit
        assert sum(s["moves"] for s in sa) > 0
    for A, B in zip(As, Bs):
        ga, gb = ctx.layer_read(A), ctx.layer_read(B)
        for key in ("assign", "frames", "obv"):
            assert np.array_equal(ga[key], gb[key]), key
        assert np.array_equal(ga["qboxes"], gb["qboxes"])
    batch.free()
    for A, B in zip(As, Bs):
        A.free()
        B.free()
    for mesh, lat in objs:
        lat.free()
        mesh.free()


def test_batched_moves_match_oracle(ctx):
    """Three small meshes of the batch in one batch, from the oracle's frames
    (identical quantised boxes on both sides): the partition rounds' moves,
    boxes, outer volumes and statistics equal the oracle's (Eq. 11-13)."""
    meshes = [mn for mn in M.sdf_batch(32, seed=3000) if mn[0].n_tris <= 4000][:3]
    assert len(meshes) == 3
    layers, probs, states = [], [], []
    for m, N in meshes:
        mesh = ctx.mesh_create(m.verts, m.tris)
        lat = ctx.build_occupancy(mesh, N)
        P = O.Problem(m.verts, m.tris, N)
        child, parent = fresh_leaf_split(ctx, lat, 4)
        K = len(parent)
        frames = O.cluster_frames(P.V, P.F, child, K, P.center)
        layers.append(ctx.layer_init(lat, child, parent, frames))
        probs.append((P, mesh, lat))
        states.append(O.layer_from_frames(P, child, parent, frames))
    batch = ctx.batch_create(layers)
    st = ctx.batch_lloyd_step(batch, rounds=4, refit=0)
    for layer, (P, _, _), L, s in zip(layers, probs, states, st):
        so = O.lloyd_moves(P, L, 4)
        g = ctx.layer_read(layer)
        assert np.array_equal(g["assign"], L.assign)
        assert np.array_equal(g["qboxes"]["b"], L.bnd)
        assert np.array_equal(g["obv"], L.obv)
        assert s["moves"] == sum(x["accepted"] for x in so)
        assert s["box_evals"] == sum(x["evals"] for x in so)
    assert sum(s["moves"] for s in st) > 0
    batch.free()
    for layer in layers:
        layer.free()
    for _, mesh, lat in probs:
        lat.free()
        mesh.free()


def test_batch_with_a_screened_layer_equals_per_layer_steps(ctx):
    """A batch holding a surrogate-screened layer (which the batch steps
    without its per-layer graphs) still leaves every layer as the per-layer
    iterations do, screened layer included."""
    meshes = [mn for mn in M.sdf_batch(32, seed=3000) if mn[0].n_tris <= 8000][:3]
    assert len(meshes) == 3
    mlp = ctx.mlp_create(7)
    objs, As, Bs = [], [], []
    for i, (m, N) in enumerate(meshes):
        mesh = ctx.mesh_create(m.verts, m.tris)
        lat = ctx.build_occupancy(mesh, N)
        child, parent = fresh_leaf_split(ctx, lat, 5)
        A, B = ctx.layer_init(lat, child, parent), ctx.layer_init(lat, child, parent)
        if i == 1:
            ctx.layer_set_surrogate(A, mlp, 2)
            ctx.layer_set_surrogate(B, mlp, 2)
        As.append(A)
        Bs.append(B)
        objs.append((mesh, lat))
    batch = ctx.batch_create(As)
    sa = ctx.batch_lloyd_step(batch, rounds=16, refit=1)
    sb = [ctx.lloyd_step(B, rounds=16, refit=1) for B in Bs]
    assert sa == sb
    for A, B in zip(As, Bs):
        ga, gb = ctx.layer_read(A), ctx.layer_read(B)
        for key in ("assign", "frames", "obv"):
            assert np.array_equal(ga[key], gb[key]), key
    batch.free()
    for A, B in zip(As, Bs):
        A.free()
        B.free()
    for mesh, lat in objs:
        lat.free()
        mesh.free()
    mlp.free()
