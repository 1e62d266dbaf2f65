"""The cube-map directional estimator (Sec. 4.1, Eq. 9-10) on the GPU against
the oracle's FP64 restatement, and both against the exact lattice count."""
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


@pytest.mark.parametrize("shape", ["icosphere", "torus"])
def test_directional_matches_oracle_and_lattice(ctx, shape):
    m = M.icosphere(3, radius=1.0) if shape == "icosphere" else M.torus(1.0, 0.4, 48, 24)
    rng = np.random.Generator(np.random.PCG64(71))
    K, res = 8, 24
    V = m.verts.astype(np.float64)
    lo, hi = V.min(0), V.max(0)
    boxes = np.zeros((K, 12), np.float32)
    for i in range(K):
        R = pins.random_rotation(rng)
        boxes[i, :3] = rng.uniform(lo + 0.1 * (hi - lo), hi - 0.1 * (hi - lo))
        boxes[i, 3:6], boxes[i, 6:9] = R[0], R[1]
        boxes[i, 9:12] = rng.uniform(0.1, 0.45, 3)
    mesh = ctx.mesh_create(m.verts, m.tris)
    got = ctx.directional_outer_volume(mesh, boxes, m=res)
    vol = 8.0 * boxes[:, 9:12].astype(np.float64).prod(1)
    ref = np.array([O.directional_outer_volume(m.verts, m.tris, b, m=res) for b in boxes])
    # FP32 ray casting vs FP64: a ray grazing an edge may flip one texel
    assert np.all(np.abs(got - ref) <= 2e-3 * vol + 1e-6), np.abs(got - ref) / vol
    N = 256
    lat = ctx.build_occupancy(mesh, N)
    cnt = ctx.outer_volume(lat, boxes).astype(np.float64)
    exact = cnt * float(np.prod(lat.spacing))
    # angular sampling of a 24 x 24 cube map: well under 1% of the box volume here
    assert np.all(np.abs(got - exact) <= 0.01 * vol), np.abs(got - exact) / vol
    lat.free()
    mesh.free()


def test_directional_degenerate(ctx):
    m = M.icosphere(2, radius=1.0)
    mesh = ctx.mesh_create(m.verts, m.tris)
    assert len(ctx.directional_outer_volume(mesh, np.zeros((0, 12), np.float32))) == 0
    inside = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0, 0.2, 0.2, 0.2]], np.float32)
    far = np.array([[5, 5, 5, 1, 0, 0, 0, 1, 0, 0.5, 0.3, 0.2]], np.float32)
    assert abs(ctx.directional_outer_volume(mesh, inside)[0]) < 1e-6
    v = ctx.directional_outer_volume(mesh, far)[0]
    assert abs(v - 8 * 0.5 * 0.3 * 0.2) < 2e-3 * 8 * 0.5 * 0.3 * 0.2
    mesh.free()
