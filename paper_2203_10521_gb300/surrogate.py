"""Training data and training loop for the learned outer-volume surrogate.

Orchestration only: every feature, count, target, forward and backward pass
runs in libobbvar's kernels; torch holds the device arrays and shuffles
indices.  Training pairs are (quantised box, exact outer volume) from real
runs of the method: the candidate boxes the Lloyd partition rounds count on
every level of a tree, plus the tree's cluster boxes with their slab bounds
moved in or out.
"""
from __future__ import annotations

import numpy as np

from . import QBOX_DTYPE


def _perturbed(q0, rng, reps):
    """reps copies of the boxes q0 with every slab bound moved by up to a
    quarter of the slab's width, inwards or outwards (an empty slab is
    closed at its lower bound)."""
    q = np.tile(q0, reps)
    b = q["b"].astype(np.int64)
    w = (b[:, 1::2] - b[:, 0::2]).astype(np.float64)
    d_lo = (rng.uniform(-0.25, 0.25, w.shape) * w).astype(np.int64)
    d_hi = (rng.uniform(-0.25, 0.25, w.shape) * w).astype(np.int64)
    b[:, 0::2] += d_lo
    b[:, 1::2] -= d_hi
    bad = b[:, 0::2] > b[:, 1::2]
    b[:, 1::2] = np.where(bad, b[:, 0::2], b[:, 1::2])
    q["b"] = b
    return q


def collect_pairs(ctx, lat, tree, depth, iters=3, perturb=2, seed=0, levels=None, target_pairs=None):
    """(qboxes, exact counts) from Lloyd candidate boxes on tree levels and
    perturbed cluster boxes; with target_pairs, perturbed copies of all the
    tree's boxes are added until there are at least that many pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    boxes, counts = [], []
    levels = range(1, depth + 1) if levels is None else levels
    tree_q = []
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
        tree_q.append(q0)
        if perturb:
            q = _perturbed(q0, rng, perturb)
            boxes.append(q)
            counts.append(ctx.outer_volume_q(lat, q))
    n = sum(len(x) for x in boxes)
    if target_pairs and n < target_pairs:
        allq = np.concatenate(tree_q)
        reps = max(1, min(64, (target_pairs - n) // max(len(allq), 1) + 1))
        while n < target_pairs:
            q = _perturbed(allq, rng, reps)
            boxes.append(q)
            counts.append(ctx.outer_volume_q(lat, q))
            n += len(q)
    q = np.concatenate(boxes) if boxes else np.zeros(0, QBOX_DTYPE)
    c = np.concatenate(counts) if counts else np.zeros(0, np.uint64)
    return q, c


def train(ctx, mlp, lat, q, counts, steps=400, batch=1024, lr=1e-3, seed=0, holdout=0.1):
    """Adam on the empty fraction (the library's targets); returns (train
    losses, held-out MSE before, after)."""
    import torch
    dev = f"cuda:{ctx.device}"
    dq = torch.from_numpy(q.view(np.uint8).copy()).to(dev)
    X = ctx.surrogate_features(lat, dq)
    T = ctx.surrogate_targets(dq, torch.from_numpy(counts.astype(np.int64)).to(dev))
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(n, generator=g).to(dev)
    n_hold = max(1, min(int(holdout * n), 65536))
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
