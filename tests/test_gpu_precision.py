"""Measured precision of the floating-point steps against FP64 (the oracle):
the cluster moments summed with compensation (as the refit sums them) and in
plain FP32, the covariances and the frames of the FP64 Jacobi, on the leaf
level and a coarse level of the trees of the 202,244-triangle union (512^3)
and the 2,029,088-triangle union (1024^3); and the FP16 tensor-core network
against the FP64 network on real box features.  Each test asserts a bound
and prints the measured worst case (pytest -s shows the lines)."""
import os

import numpy as np
import pytest

import oracle as O
from synth import meshes as M
from synth import params as SP

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


def _group_error(got, ref, cols):
    """Largest over clusters of max_c |got - ref| / max_c |ref| over the columns cols."""
    d = np.abs(got[:, cols] - ref[:, cols]).max(axis=1)
    s = np.abs(ref[:, cols]).max(axis=1)
    ok = s > 0
    return float((d[ok] / s[ok]).max())


def _shift(mom, d):
    """FP64 moments about the origin c moved to the origin c + d (per cluster):
    sum A m - A d, and the second moments by the parallel-axis rule."""
    out = mom.copy()
    A = mom[:, 0]
    out[:, 1:4] = mom[:, 1:4] - A[:, None] * d
    ia, ib = [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]
    for q in range(6):
        a, b = ia[q], ib[q]
        out[:, 4 + q] = (mom[:, 4 + q] - d[:, b] * out[:, 1 + a] - d[:, a] * out[:, 1 + b]
                         - A * d[:, a] * d[:, b])
    return out


def _covariances(mom):
    A = mom[:, :1]
    mu = mom[:, 1:4] / A
    ia, ib = [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]
    return mom[:, 4:10] / A - mu[:, ia] * mu[:, ib]


def _full(c6):
    C = np.zeros((len(c6), 3, 3))
    for q, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        C[:, a, b] = C[:, b, a] = c6[:, q]
    return C


@pytest.mark.parametrize("name,N,depth", [("200k", 512, 10), ("2m", 1024, 14)])
def test_moments_covariance_frames_against_fp64(ctx, name, N, depth):
    m = M.sdf_union_200k() if name == "200k" else M.sdf_union_2m()
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    tree = ctx.build_tree(lat, depth, 1)
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    for lev in (3, depth):
        r = ctx.tree_read(tree, lev)
        K = 1 << lev
        layer = ctx.layer_init(lat, r["assign"], (np.arange(K) // 2).astype(np.int32))
        comp = ctx.layer_moments(layer, compensated=True)
        plain = ctx.layer_moments(layer, compensated=False)
        # the oracle's FP64 moments (about the lattice centre) moved to the
        # GPU's per-cluster origins: the first vertex of the lowest-numbered
        # triangle of each cluster
        first = np.full(K, m.n_tris, np.int64)
        np.minimum.at(first, r["assign"], np.arange(m.n_tris))
        origin = P.V[P.F[first, 0]].astype(np.float64)
        ref = _shift(O.moments(P.V, P.F, r["assign"], K, P.center), origin - P.center)
        err = {}
        for label, got in (("compensated", comp), ("plain", plain)):
            err[label] = {g: _group_error(got, ref, cols) for g, cols in
                          (("area", [0]), ("first", [1, 2, 3]), ("second", [4, 5, 6, 7, 8, 9]))}
            cg, cr = _covariances(got), _covariances(ref)
            d = np.abs(cg - cr).max(axis=1) / np.abs(cr).max(axis=1)
            err[label]["covariance"] = float(d.max())
        # frames: the GPU's (FP64 Jacobi of its compensated moments) against the
        # oracle's (FP64 moments and Jacobi), on clusters whose spectrum is not
        # degenerate (relative eigengaps of at least 1e-3)
        frames = ctx.layer_read(layer)["frames"].reshape(K, 3, 3)
        ref_frames = O.cluster_frames(P.V, P.F, r["assign"], K, P.center).reshape(K, 3, 3)
        ev = np.linalg.eigvalsh(_full(_covariances(ref)))
        gap = np.minimum(ev[:, 2] - ev[:, 1], ev[:, 1] - ev[:, 0]) / np.maximum(ev[:, 2], 1e-300)
        ok = gap >= 1e-3
        ferr = float(np.abs(frames[ok] - ref_frames[ok]).max())
        print(f"{name} level {lev} ({K} clusters, {m.n_tris // K} triangles each): "
              f"moments rel. error compensated {err['compensated']}, plain FP32 {err['plain']}; "
              f"frames max |dR| {ferr:.2e} on {int(ok.sum())} clusters")
        assert max(err["compensated"].values()) <= 1e-6, err
        assert ferr <= 1e-5
        layer.free()
    tree.free()
    lat.free()
    mesh.free()


def test_fp16_network_against_fp64(ctx):
    """The tensor-core network (FP16 weights and activations, FP32 accumulate)
    against the FP64 network on the features of real boxes."""
    m = M.torus_4096()
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, 64)
    tree = ctx.build_tree(lat, 6, 1)
    q = np.concatenate([ctx.tree_read(tree, lev)["qboxes"] for lev in range(7)])
    X = ctx.surrogate_features(lat, q)
    mlp = ctx.mlp_create(0)
    p = SP.mlp_params(11)
    ctx.mlp_set_params(mlp, p)
    y16 = ctx.mlp_forward(mlp, X, half=True)
    y32 = ctx.mlp_forward(mlp, X, half=False)
    y_ref, _ = O.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    e16 = np.abs(y16 - y_ref)
    e32 = np.abs(y32 - y_ref)
    rel16 = float((e16 / np.maximum(np.abs(y_ref), 1e-3)).max())
    print(f"network on {len(q)} real boxes: FP16 tensor cores max abs {e16.max():.2e} rel {rel16:.2e}; "
          f"FP32 CUDA cores max abs {e32.max():.2e}")
    assert rel16 <= 2e-2 and e32.max() <= 1e-4
    mlp.free()
    tree.free()
    lat.free()
    mesh.free()
