"""Pins of the oracle's surrogate pieces: backpropagation against finite
differences, and the box features against a closed-form box and solid."""
import numpy as np

import oracle as O
from synth import meshes as M
from synth import params as SP
from tests import pins


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


def test_features_of_rotated_boxes_match_exact_rationals():
    """Rotated boxes on the torus: every patch bit equals the occupancy at the
    exact sample point M^-1 v (Python rationals) rounded to the nearest
    lattice point, ties included, and the tie flag marks exactly the points
    within 1e-3 of a half-integer; the box parameters agree with their exact
    values to FP32 rounding."""
    from fractions import Fraction as Fr
    m = M.torus_4096()
    N = 64
    P = O.Problem(m.verts, m.tris, N)
    P.occ.fill_all()
    rng = np.random.Generator(np.random.PCG64(41))
    boxes = np.zeros((12, 12), np.float32)
    for i in range(12):
        R = pins.random_rotation(rng)
        boxes[i, :3] = rng.uniform([-1.2, -1.2, -0.3], [1.2, 1.2, 0.3])
        boxes[i, 3:6], boxes[i, 6:9] = R[0], R[1]
        boxes[i, 9:12] = rng.uniform(0.05, 0.6, 3)
    n, bnd = O.quantize_boxes(boxes, P.lo, P.h)
    f, tie = O.surrogate_features(P.occ, n, bnd, return_ties=True)
    checked = ties = 0
    for b in range(len(n)):
        Mi = [[int(v) for v in n[b, 3 * a:3 * a + 3]] for a in range(3)]
        L = [-((-int(bnd[b, 2 * a])) // 256) for a in range(3)]
        H = [int(bnd[b, 2 * a + 1]) // 256 for a in range(3)]
        det = (Mi[0][0] * (Mi[1][1] * Mi[2][2] - Mi[1][2] * Mi[2][1]) - Mi[0][1] * (Mi[1][0] * Mi[2][2] - Mi[1][2] * Mi[2][0])
               + Mi[0][2] * (Mi[1][0] * Mi[2][1] - Mi[1][1] * Mi[2][0]))
        inv = [[Fr((Mi[(c + 1) % 3][(r + 1) % 3] * Mi[(c + 2) % 3][(r + 2) % 3]
                    - Mi[(c + 1) % 3][(r + 2) % 3] * Mi[(c + 2) % 3][(r + 1) % 3]), det) for c in range(3)] for r in range(3)]
        mid = [Fr(L[a] + H[a], 2) for a in range(3)]
        cen = [sum(inv[r][a] * mid[a] for a in range(3)) for r in range(3)]
        assert np.array_equal(f[b, :3], np.array([float(x / N) for x in cen], np.float32))
        for a in range(2):
            nn = np.sqrt(sum(float(x) ** 2 for x in Mi[a]))
            assert np.allclose(f[b, 3 + 3 * a:6 + 3 * a], np.array(Mi[a]) / nn, rtol=1e-7, atol=1e-8)
        bits = f[b, 12:]
        for s in range(512):
            sv = (s & 7, (s >> 3) & 7, s >> 6)
            v = [L[a] + Fr((H[a] - L[a]) * (2 * sv[a] + 1), 16) for a in range(3)]
            p = [sum(inv[r][a] * v[a] for a in range(3)) for r in range(3)]
            near = any(abs(x - (x.numerator // x.denominator) - Fr(1, 2)) < Fr(1, 1000) for x in p)
            assert bool(tie[b, s]) == near, (b, s)
            ties += near
            idx = [int((x + Fr(1, 2)) // 1) for x in p]
            inside = all(0 <= i < N for i in idx)
            want = float(P.occ.occ[idx[2], idx[1], idx[0]]) if inside else 0.0
            assert bits[s] == want, (b, s)
            checked += 1
    assert checked == 12 * 512
