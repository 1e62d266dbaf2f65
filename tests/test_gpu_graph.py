"""The Lloyd iteration captured as one CUDA graph (device-side round loop)
must reproduce the host-driven iteration exactly; the counting tile height
and its autotuner change speed only, never a count."""
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


@pytest.fixture(scope="module")
def blobs(ctx):
    m = M.sdf_union_mesh(7, 18, n_spheres=6, n_capsules=3)
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, 64)
    P = O.Problem(m.verts, m.tris, 64)
    seed = O.build_tree(P, 4, iters=0)[4]
    yield mesh, lat, seed
    lat.free()
    mesh.free()


@pytest.mark.parametrize("refit", [0, 1, 2, 3])
def test_graph_iteration_equals_host_loop(ctx, blobs, refit):
    mesh, lat, seed = blobs
    a = ctx.layer_init(lat, seed.assign, seed.parent, seed.frames)
    b = ctx.layer_init(lat, seed.assign, seed.parent, seed.frames)
    moved = 0
    for it in range(4):
        sa = ctx.lloyd_step(a, rounds=16, refit=refit, descent_steps=2)
        sb = ctx.lloyd_step(b, rounds=16, refit=refit, descent_steps=2, graph=True)
        assert sa == sb, it
        moved += sa["moves"]
        ga, gb = ctx.layer_read(a), ctx.layer_read(b)
        for key in ("assign", "frames", "obv"):
            assert np.array_equal(ga[key], gb[key]), (it, key)
        assert np.array_equal(ga["qboxes"], gb["qboxes"])
    assert moved > 0
    a.free()
    b.free()


def test_graph_is_recaptured_for_new_options_and_counts_launches(ctx, blobs):
    mesh, lat, seed = blobs
    a = ctx.layer_init(lat, seed.assign, seed.parent, seed.frames)
    b = ctx.layer_init(lat, seed.assign, seed.parent, seed.frames)
    for rounds in (1, 3, 1):
        sa = ctx.lloyd_step(a, rounds=rounds, refit=1)
        n0 = ctx.profile_read()["launches"]
        sb = ctx.lloyd_step(b, rounds=rounds, refit=1, graph=True)
        n1 = ctx.profile_read()["launches"]
        assert sa == sb and sb["rounds_run"] <= rounds
        assert n1 - n0 >= 8 * sb["rounds_run"]
    assert np.array_equal(ctx.layer_read(a)["obv"], ctx.layer_read(b)["obv"])
    a.free()
    b.free()


def test_counts_do_not_depend_on_tile_height_and_autotuner(ctx, blobs):
    """Rows per tile only change the work split: counts are identical for every
    setting, and the autotuner keeps one of its candidates."""
    mesh, lat, seed = blobs
    rng = np.random.Generator(np.random.PCG64(12))
    boxes = np.zeros((300, 12), np.float32)
    lo, hi = lat.lo, lat.lo + lat.N * lat.spacing
    for i in range(len(boxes)):
        R = pins.random_rotation(rng)
        boxes[i, :3] = rng.uniform(lo, hi)
        boxes[i, 3:6], boxes[i, 6:9] = R[0], R[1]
        boxes[i, 9:12] = rng.uniform(0.01, 0.5, 3) * (hi - lo)
    q = ctx.quantize_boxes(lat, boxes)
    ref = None
    for tk in (1, 3, 8, 16, 32, 64, 128):
        ctx.set_counting_tile(tk)
        c, p = ctx.outer_volume_q(lat, q, want_points=True)
        if ref is None:
            ref = (c, p)
        assert np.array_equal(c, ref[0]) and np.array_equal(p, ref[1]), tk
    best, ms = ctx.tune_counting(lat, q)
    assert best in (8, 16, 32, 64) and all(v > 0 for v in ms.values())
    assert np.array_equal(ctx.outer_volume_q(lat, q), ref[0])
    ctx.set_counting_tile(32)
