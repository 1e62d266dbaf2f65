"""Training data and training loop for the learned outer-volume surrogate.

Orchestration only: every feature, count, forward and backward pass runs in
libobbvar's kernels; torch holds the device arrays and shuffles indices.
Training pairs are (quantised box, exact outer volume) from real runs of the
method: the candidate boxes the Lloyd partition rounds count on every level of
a tree, plus the cluster boxes with their slab bounds moved in or out.
"""
from __future__ import annotations

import numpy as np

from . import QBOX_DTYPE


def box_cells(q):
    """Box volume in lattice cells, prod(H_a - L_a + 1) / |det n| (the scale of the prediction)."""
    n = q["n"].reshape(-1, 3, 3).astype(np.float64)
    b = q["b"].astype(np.int64)
    L = -((-b[:, 0::2]) >> 8)
    H = b[:, 1::2] >> 8
    w = np.maximum(H - L + 1, 0).astype(np.float64)
    det = np.abs(np.linalg.det(n))
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.where(det > 0, w.prod(axis=1) / det, 0.0)
    return c


def collect_pairs(ctx, lat, tree, depth, iters=3, perturb=2, seed=0, levels=None):
    """(qboxes, counts) from Lloyd candidate boxes on tree levels and perturbed cluster boxes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes, counts = [], []
    levels = range(1, depth + 1) if levels is None else levels
    for lev in levels:
        r = ctx.tree_read(tree, lev)
        K = 1 << lev
        parent = (np.arange(K) // 2).astype(np.int32)
        layer = ctx.layer_init(lat, r["assign"], parent, r["frames"])
        for _ in range(iters):
            ctx.lloyd_step(layer, rounds=1, refit=False)
            q, c = ctx.layer_last_candidates(layer)
            if len(q):
                boxes.append(q)
                counts.append(c)
        q0 = ctx.layer_read(layer)["qboxes"]
        layer.free()
        for _ in range(perturb):
            q = q0.copy()
            b = q["b"].astype(np.int64)
            w = (b[:, 1::2] - b[:, 0::2]).astype(np.float64)
            d_lo = (rng.uniform(-0.25, 0.25, w.shape) * w).astype(np.int64)
            d_hi = (rng.uniform(-0.25, 0.25, w.shape) * w).astype(np.int64)
            b[:, 0::2] += d_lo
            b[:, 1::2] -= d_hi
            bad = b[:, 0::2] > b[:, 1::2]
            b[:, 1::2] = np.where(bad, b[:, 0::2], b[:, 1::2])
            q["b"] = b
            c = ctx.outer_volume_q(lat, q)
            boxes.append(q)
            counts.append(c)
    q = np.concatenate(boxes) if boxes else np.zeros(0, QBOX_DTYPE)
    c = np.concatenate(counts) if counts else np.zeros(0, np.uint64)
    return q, c


def targets(q, counts):
    """Empty fraction of each box, clipped to [0, 1]."""
    cells = box_cells(q)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(cells > 0, counts.astype(np.float64) / cells, 0.0)
    return np.clip(t, 0.0, 1.0).astype(np.float32)


def train(ctx, mlp, lat, q, counts, steps=400, batch=1024, lr=1e-3, seed=0, holdout=0.1):
    """Adam on the empty fraction; returns (train losses, held-out MSE before, after)."""
    import torch
    dev = f"cuda:{ctx.device}"
    X = ctx.surrogate_features(lat, torch.from_numpy(q.view(np.uint8).copy()).to(dev))
    T = torch.from_numpy(targets(q, counts)).to(dev)
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(n, generator=g).to(dev)
    n_hold = max(1, int(holdout * n))
    hold, tr = perm[:n_hold], perm[n_hold:]
    Xh, Th = X[hold].contiguous(), T[hold].contiguous()

    def held_mse():
        y = ctx.mlp_forward(mlp, Xh, half=True)
        return float(((y - Th) ** 2).mean().item())

    before = held_mse()
    losses = []
    for s in range(steps):
        idx = tr[torch.randint(0, tr.numel(), (min(batch, tr.numel()),), generator=g).to(dev)]
        xb, tb = X[idx].contiguous(), T[idx].contiguous()
        ctx.mlp_train_step(mlp, xb, tb, lr)
        if s % 50 == 0 or s == steps - 1:
            losses.append(float(((ctx.mlp_forward(mlp, xb, half=False) - tb) ** 2).mean().item()))
    return losses, before, held_mse()
