"""Pins of the oracle's surrogate pieces: backpropagation against finite
differences, and the box features against a closed-form box and solid."""
import numpy as np

import oracle as O
from synth import meshes as M
from synth import params as SP


def test_mlp_gradient_matches_finite_differences():
    """Backpropagation of the mean squared error equals central differences
    (FP64) on a sample of parameters from every layer."""
    rng = np.random.Generator(np.random.PCG64(3))
    p = SP.mlp_params(7).astype(np.float64)
    X = SP.features(8, 6).astype(np.float64)
    T = SP.targets(9, 6).astype(np.float64)
    loss, g = O.mlp_loss_grad(p, X, T)
    sizes = [524 * 128, 128, 128 * 128, 128, 128 * 128, 128, 128, 1]
    offs = np.cumsum([0] + sizes)
    idx = np.concatenate([rng.integers(offs[i], offs[i + 1], min(12, sizes[i])) for i in range(8)])
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (O.mlp_loss_grad(pp, X, T)[0] - O.mlp_loss_grad(pm, X, T)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])
    # the forward pass of zero parameters predicts 1/2 everywhere
    y, _ = O.mlp_forward(np.zeros_like(p), X)
    assert np.allclose(y, 0.5)


def test_features_of_axis_aligned_box_on_known_solid():
    """Isotropic lattice (h = 1) with an inner cube on lattice planes: an
    axis-aligned box's parameters are its index centre / N, the coordinate axes
    and half widths / N; its patch bits follow the half-open closed form."""
    N = 16
    outer = M.cube((0, 0, 0), (N, N, N))
    inner = M.cube((3.5, 4.5, 5.5), (9.5, 11.5, 12.5))     # removes [3,9) x [4,11) x [5,12)
    V = np.concatenate([outer.verts, inner.verts])
    F = np.concatenate([outer.tris, inner.tris + 8])
    P = O.Problem(V, F, N)
    n = O.frame_normals(np.eye(3).reshape(1, 9), P.h)[0]
    assert np.array_equal(n, np.diag([1 << 24] * 3).ravel())
    i0, i1 = np.array([1, 2, 3]), np.array([14, 13, 15])
    bnd = np.stack([i0 * (1 << 32), i1 * (1 << 32)], -1).reshape(1, 6)   # U = 256 i, n = 2^24
    f = O.surrogate_features(P.occ, n[None], bnd)[0]
    assert np.allclose(f[:3], (i0 + i1) / 2 / N)
    assert np.array_equal(f[3:9], [1, 0, 0, 0, 1, 0])
    assert np.allclose(f[9:12], (i1 - i0) / 2 / N)
    bits = f[12:].reshape(8, 8, 8)          # [sz][sy][sx]
    s = np.arange(8)
    px = np.floor(i0[0] + (i1[0] - i0[0]) * (2 * s + 1) / 16 + 0.5)
    py = np.floor(i0[1] + (i1[1] - i0[1]) * (2 * s + 1) / 16 + 0.5)
    pz = np.floor(i0[2] + (i1[2] - i0[2]) * (2 * s + 1) / 16 + 0.5)
    hole = ((pz[:, None, None] >= 5) & (pz[:, None, None] < 12) & (py[None, :, None] >= 4)
            & (py[None, :, None] < 11) & (px[None, None, :] >= 3) & (px[None, None, :] < 9))
    assert np.array_equal(bits, (~hole).astype(np.float32))
    assert 0 < bits.sum() < 512
