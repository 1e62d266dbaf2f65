"""Every handle (mesh, lattice, layer, tree, network) belongs to the context
that made it: device pointers, scratch and stream of one context must not be
mixed with another's (two contexts may sit on different devices).  Each entry
point that takes a handle refuses one from another context with
OBB_ERR_STATE before any device work, and the owner's objects stay usable.
Both contexts here are on device 0, so nothing is ever launched with a
foreign pointer: the refusals happen on the host."""
import numpy as np
import pytest

from synth import meshes as M

pytestmark = pytest.mark.gpu

OBB_ERR_STATE = -8


@pytest.fixture(scope="module")
def two():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2203_10521_gb300 as P
    a, b = P.Context(0), P.Context(0)
    m = M.torus_4096()
    mesh = a.mesh_create(m.verts, m.tris)
    lat = a.build_occupancy(mesh, 64)
    tree = a.build_tree(lat, 2, 1)
    r = a.tree_read(tree, 2)
    parents = a.tree_parents(tree, 2)
    layer = a.layer_init(lat, r["assign"], parents, r["frames"])
    mlp_a, mlp_b = a.mlp_create(1), b.mlp_create(2)
    yield dict(P=P, a=a, b=b, mesh=mesh, lat=lat, tree=tree, r=r, parents=parents, layer=layer, mlp_a=mlp_a,
               mlp_b=mlp_b)
    torch.cuda.synchronize()
    for h in (layer, mlp_a, tree, lat, mesh):
        h.free()
    mlp_b.free()
    b.close()
    a.close()


def _refused(P, what, fn):
    with pytest.raises(P.ObbError) as e:
        fn()
    assert e.value.code == OBB_ERR_STATE and f"{what} belongs to another context" in str(e.value)


def test_foreign_handles_are_refused(two):
    P, b = two["P"], two["b"]
    lat, mesh, tree, layer, r = two["lat"], two["mesh"], two["tree"], two["layer"], two["r"]
    feats = np.zeros((2, b.SURROGATE_INPUTS), np.float32)
    cases = [
        ("lattice", lambda: b.quantize_boxes(lat, r["boxes"])),
        ("lattice", lambda: b.outer_volume(lat, r["boxes"])),
        ("lattice", lambda: b.outer_volume_q(lat, r["qboxes"])),
        ("lattice", lambda: b.outer_volume_multi([lat], r["qboxes"], np.zeros(len(r["qboxes"]), np.int32))),
        ("lattice", lambda: b.tune_counting(lat, r["qboxes"])),
        ("lattice", lambda: b.occupancy_rebuild(lat)),
        ("lattice", lambda: b.layer_init(lat, r["assign"], two["parents"])),
        ("lattice", lambda: b.build_tree(lat, 2, 1)),
        ("lattice", lambda: b.surrogate_features(lat, r["qboxes"])),
        ("mesh", lambda: b.build_occupancy(mesh, 64)),
        ("mesh", lambda: b.directional_outer_volume(mesh, r["boxes"], 4)),
        ("layer", lambda: b.lloyd_step(layer)),
        ("layer", lambda: b.layer_read(layer)),
        ("layer", lambda: b.layer_parents(layer)),
        ("layer", lambda: b.layer_split(layer)),
        ("layer", lambda: b.layer_members(layer)),
        ("layer", lambda: b.layer_moments(layer)),
        ("layer", lambda: b.layer_set_surrogate(layer, two["mlp_b"], 5)),
        ("layer", lambda: b.layer_last_candidates(layer, cap=16)),
        ("layer", lambda: b.batch_create([layer])),
        ("tree", lambda: b.tree_read(tree, 1)),
        ("tree", lambda: b.tree_parents(tree, 1)),
        ("tree", lambda: b.tree_score(tree)),
        ("tree", lambda: b.tree_sweep(tree)),
        ("network", lambda: two["a"].layer_set_surrogate(layer, two["mlp_b"], 5)),
        ("network", lambda: b.mlp_params(two["mlp_a"])),
        ("network", lambda: b.mlp_forward(two["mlp_a"], feats)),
    ]
    for what, fn in cases:
        _refused(P, what, fn)


def test_owner_still_works_after_refusals(two):
    a, lat, tree, layer, r = two["a"], two["lat"], two["tree"], two["layer"], two["r"]
    counts = a.outer_volume_q(lat, r["qboxes"])
    np.testing.assert_array_equal(np.asarray(counts, np.uint64), r["obv"])
    st = a.lloyd_step(layer, rounds=2)
    assert st["total_obv"] == int(a.layer_read(layer)["obv"].sum())
    pts, _ = a.tree_score(tree)
    assert pts > 0


def test_device_inputs_are_checked_before_any_call(two):
    """CUDA-tensor inputs: element type, length, whole rows, contiguity and
    one placement for all of a call's arrays are checked in the binding
    (ValueError, nothing called); well-formed device inputs give the same
    layer as host inputs."""
    import torch
    a, lat, r, parents = two["a"], two["lat"], two["r"], two["parents"]
    dev = f"cuda:{a.device}"
    d_assign = torch.from_numpy(r["assign"]).to(dev)
    d_parent = torch.from_numpy(parents).to(dev)
    d_frames = torch.from_numpy(np.ascontiguousarray(r["frames"])).to(dev)
    bad = [
        lambda: a.layer_init(lat, d_assign, parents),                                  # mixed placement
        lambda: a.layer_init(lat, d_assign.long(), d_parent),                          # element type
        lambda: a.layer_init(lat, d_assign[:-1].contiguous(), d_parent),               # length
        lambda: a.layer_init(lat, d_assign, d_parent, d_frames[:-1].contiguous()),     # frames length
        lambda: a.mlp_forward(two["mlp_a"], torch.zeros((2, 100), dtype=torch.float32, device=dev)),
        lambda: a.mlp_train_step(two["mlp_a"], torch.zeros((2, 524), dtype=torch.float32, device=dev),
                                 torch.zeros(3, dtype=torch.float32, device=dev), 1e-3),
        lambda: a.surrogate_targets(torch.from_numpy(r["qboxes"].view(np.uint8).copy()).to(dev),
                                    r["obv"].astype(np.uint64)),
        lambda: a.outer_volume(lat, torch.from_numpy(np.ascontiguousarray(
            r["boxes"]).view(np.float32).reshape(-1, 12)).to(dev).t()),               # not contiguous
        lambda: a.quantize_boxes(lat, torch.from_numpy(np.ascontiguousarray(r["boxes"]).view(np.float32)).to(dev),
                                 out=torch.zeros(len(r["boxes"]) * 88 - 1, dtype=torch.uint8, device=dev)),
    ]
    for fn in bad:
        with pytest.raises(ValueError):
            fn()
    host = a.layer_init(lat, r["assign"], parents, r["frames"])
    on_dev = a.layer_init(lat, d_assign, d_parent, d_frames)
    try:
        x, y = a.layer_read(host), a.layer_read(on_dev)
        for k in ("assign", "frames", "obv"):
            np.testing.assert_array_equal(x[k], y[k])
        np.testing.assert_array_equal(x["qboxes"].view(np.uint8), y["qboxes"].view(np.uint8))
    finally:
        host.free()
        on_dev.free()
