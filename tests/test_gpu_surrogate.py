"""GPU parity and behaviour of the learned surrogate: features against their
definition, forward and gradients against the FP64 oracle network, training
on real candidate boxes, and screened Lloyd iterations against plain ones."""
import time

import numpy as np
import pytest

import oracle as O
from synth import meshes as M
from synth import params as SP
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
def torus(ctx):
    m = M.torus_4096()
    N = 64
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    P = O.Problem(m.verts, m.tris, N)
    P.occ.fill_all()
    return m, mesh, lat, P


def _rand_qboxes(ctx, lat, rng, K):
    out = np.zeros((K, 12), dtype=np.float32)
    for i in range(K):
        R = pins.random_rotation(rng)
        out[i, :3] = rng.uniform([-1.4, -1.4, -0.4], [1.4, 1.4, 0.4])
        out[i, 3:6], out[i, 6:9] = R[0], R[1]
        out[i, 9:12] = rng.uniform(0.05, 0.6, 3)
    return ctx.quantize_boxes(lat, out)


def test_features_match_definition(ctx, torus):
    """The kernel's features (FP32 arithmetic) against their definition (the
    oracle: FP64 parameters from exact integers, patch bits at the exact
    rational sample points): every patch bit whose sample point lies more than
    1e-3 cells from a rounding tie is equal, and the 12 box parameters agree
    to FP32 accuracy.  The share of tie-adjacent bits and the disagreements
    among them are reported."""
    m, mesh, lat, P = torus
    q = _rand_qboxes(ctx, lat, np.random.Generator(np.random.PCG64(1)), 300)
    f = ctx.surrogate_features(lat, q)
    ref, tie = O.surrogate_features(P.occ, q["n"], q["b"], return_ties=True)
    assert np.allclose(f[:, :12], ref[:, :12], rtol=1e-5, atol=1e-5)
    far = tie == 0
    assert np.array_equal(f[:, 12:][far], ref[:, 12:][far])
    near = int((~far).sum())
    differ = int((f[:, 12:] != ref[:, 12:]).sum())
    print(f"patch bits near a rounding tie: {near} of {far.size} ({near / far.size:.2e}); "
          f"of these {differ} differ; max parameter error {np.abs(f[:, :12] - ref[:, :12]).max():.2e}")
    assert far.mean() > 0.99


def test_targets_are_exact_counts_over_cell_volume(ctx, torus):
    """The library's training targets are the exact outer volume divided by
    the box's cell volume prod(H_a - L_a + 1) / |det n| (the scale the screen
    multiplies its prediction by), clipped to [0, 1]: checked against exact
    rational arithmetic on the oracle's counts."""
    from fractions import Fraction as Fr
    m, mesh, lat, P = torus
    q = _rand_qboxes(ctx, lat, np.random.Generator(np.random.PCG64(5)), 200)
    ref, _ = O.outer_volume(P.occ, q["n"], q["b"])
    t = ctx.surrogate_targets(q, ref)
    for i in range(len(q)):
        n = [[int(v) for v in q["n"][i, 3 * a:3 * a + 3]] for a in range(3)]
        det = (n[0][0] * (n[1][1] * n[2][2] - n[1][2] * n[2][1]) - n[0][1] * (n[1][0] * n[2][2] - n[1][2] * n[2][0])
               + n[0][2] * (n[1][0] * n[2][1] - n[1][1] * n[2][0]))
        w = 1
        for a in range(3):
            L = -((-int(q["b"][i, 2 * a])) // 256)
            H = int(q["b"][i, 2 * a + 1]) // 256
            w *= max(H - L + 1, 0)
        want = 0.0 if w == 0 else float(min(max(Fr(int(ref[i]) * abs(det), w), Fr(0)), Fr(1)))
        assert abs(float(t[i]) - want) <= 1e-6 * max(want, 1e-6), (i, float(t[i]), want)


def test_forward_and_gradients_match_fp64_oracle(ctx):
    mlp = ctx.mlp_create(0)
    p = SP.mlp_params(11)
    ctx.mlp_set_params(mlp, p)
    X = SP.features(12, 257)            # a ragged batch (not a multiple of the 64-row tile)
    T = SP.targets(13, 257)
    y_ref, _ = O.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    y32 = ctx.mlp_forward(mlp, X, half=False)
    y16 = ctx.mlp_forward(mlp, X, half=True)
    assert np.max(np.abs(y32 - y_ref)) <= 1e-4
    assert np.max(np.abs(y16 - y_ref) / np.maximum(np.abs(y_ref), 1e-3)) <= 2e-2
    g, loss = ctx.mlp_gradients(mlp, X, T)
    loss_ref, g_ref = O.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    assert np.linalg.norm(g - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    assert np.array_equal(ctx.mlp_params(mlp), p)     # gradients do not update
    mlp.free()


def _fresh_leaf_layer(ctx, lat, tree, depth):
    """The leaf level seeded by a median split of the parent level, no Lloyd yet."""
    up = ctx.tree_read(tree, depth - 1)
    Kp = 1 << (depth - 1)
    parent_layer = ctx.layer_init(lat, up["assign"], (np.arange(Kp) // 2).astype(np.int32), up["frames"])
    child = ctx.layer_split(parent_layer)
    parent_layer.free()
    K = 1 << depth
    return ctx.layer_init(lat, child, (np.arange(K) // 2).astype(np.int32)), child


def test_train_and_screen(ctx, torus):
    """Training on real candidate boxes lowers the held-out error; screened
    Lloyd iterations reach the plain final outer volume within 0.5% with fewer
    exact box counts: the box update is the rotation-probe descent, and the
    surrogate keeps the 2 most promising of each cluster's 6 probes."""
    import torch
    from paper_2203_10521_gb300 import surrogate as S
    m, mesh, lat, P = torus
    depth = 4
    tree = ctx.build_tree(lat, depth, 2)
    q, c = S.collect_pairs(ctx, lat, tree, depth, iters=3, perturb=24, seed=1)
    assert len(q) > 300
    mlp = ctx.mlp_create(5)
    losses, before, after = S.train(ctx, mlp, lat, q, c, steps=300, batch=256, lr=2e-3, seed=2)
    assert after < 0.5 * before, (before, after)
    results = {}
    for mode in ("plain", "screened"):
        layer, child = _fresh_leaf_layer(ctx, lat, tree, depth)
        if mode == "screened":
            ctx.layer_set_surrogate(layer, mlp, 2)
        evals = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(8):
            st = ctx.lloyd_step(layer, rounds=16, refit=2, descent_steps=2)
            evals += st["box_evals"]
        torch.cuda.synchronize()
        results[mode] = (st["total_obv"], evals, time.perf_counter() - t0)
        # the exact count decides every move: stored outer volumes are exact
        g = ctx.layer_read(layer)
        cnt, _ = O.outer_volume(P.occ, g["qboxes"]["n"], g["qboxes"]["b"])
        assert np.array_equal(cnt, g["obv"])
        layer.free()
    (tp, ep, sp), (ts, es, ss) = results["plain"], results["screened"]
    print(f"plain: total {tp} evals {ep} {sp*1e3:.1f} ms; screened: total {ts} evals {es} {ss*1e3:.1f} ms")
    assert abs(int(ts) - int(tp)) <= 0.005 * int(tp)
    assert es < ep
    tree.free()
    mlp.free()


def test_tensor_core_wait_timeout_is_reported(ctx):
    """A tensor-core wait that can never complete (the test hook skips the first
    MMA commit, so nothing is in flight) gives up after its time limit: the call
    reports OBB_ERR_TIMEOUT and the context stays usable."""
    import paper_2203_10521_gb300 as PK
    mlp = ctx.mlp_create(0)
    p = SP.mlp_params(11)
    ctx.mlp_set_params(mlp, p)
    X = SP.features(12, 257)
    ctx.test_inject(1)
    with pytest.raises(PK.ObbError) as e:
        ctx.mlp_forward(mlp, X, half=True)
    assert e.value.code == -6
    y_ref, _ = O.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    y16 = ctx.mlp_forward(mlp, X, half=True)
    assert np.max(np.abs(y16 - y_ref) / np.maximum(np.abs(y_ref), 1e-3)) <= 2e-2
    mlp.free()
