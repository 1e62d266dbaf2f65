"""Seeded parameter vectors for the surrogate network (random numbers only)."""
import numpy as np

N_IN, N_H = 524, 128
N_PARAMS = N_IN * N_H + N_H + 2 * (N_H * N_H + N_H) + N_H + 1


def mlp_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """He-uniform weights, small random biases, flat float32 in the layer order W1 b1 W2 b2 W3 b3 W4 b4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fi, fo in ((N_IN, N_H), (N_H, N_H), (N_H, N_H), (N_H, 1)):
        lim = scale * np.sqrt(6.0 / fi)
        parts.append(rng.uniform(-lim, lim, fi * fo))
        parts.append(rng.uniform(-0.05, 0.05, fo))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == N_PARAMS
    return p


def features(seed: int, B: int) -> np.ndarray:
    """Random feature rows shaped like the surrogate's inputs: 12 box numbers, 512 bits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.concatenate([rng.uniform(-1.0, 1.0, (B, 12)), (rng.uniform(0, 1, (B, 512)) < 0.4)], axis=1)
    return X.astype(np.float32)


def targets(seed: int, B: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, B).astype(np.float32)
