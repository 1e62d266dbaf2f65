"""Independent references the oracle is pinned to (test helpers, FP64 numpy).

None of these share arithmetic with the oracle: they come from textbook
geometry (solid angles, the divergence theorem, quadrature rules)."""
import numpy as np


def fixed_to_world(U, lo, h):
    """World position of a fixed-point vertex: x = lo + h (U / 2^8 + 1/2)."""
    return np.asarray(lo) + np.asarray(h) * (np.asarray(U, dtype=np.float64) / 256.0 + 0.5)


def winding_numbers(P, V, F, chunk=256):
    """Generalised winding number of the closed triangle mesh (V, F) at points P,
    from the Van Oosterom-Strackee triangle solid angle: sum(Omega) / (4 pi)."""
    P = np.asarray(P, dtype=np.float64)
    A = V[F[:, 0]]
    B = V[F[:, 1]]
    Cc = V[F[:, 2]]
    out = np.empty(P.shape[0])
    for s in range(0, P.shape[0], chunk):
        p = P[s:s + chunk, None, :]
        a = A[None] - p
        b = B[None] - p
        c = Cc[None] - p
        la = np.linalg.norm(a, axis=-1)
        lb = np.linalg.norm(b, axis=-1)
        lc = np.linalg.norm(c, axis=-1)
        det = np.einsum("ptk,ptk->pt", a, np.cross(b, c))
        den = (la * lb * lc + np.einsum("ptk,ptk->pt", a, b) * lc
               + np.einsum("ptk,ptk->pt", a, c) * lb + np.einsum("ptk,ptk->pt", b, c) * la)
        out[s:s + chunk] = (2.0 * np.arctan2(det, den)).sum(axis=1) / (4.0 * np.pi)
    return out


def polyhedron_volume(V, F):
    """Signed volume of a closed, consistently oriented mesh (divergence theorem)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return float(np.einsum("tk,tk->t", a, np.cross(b, c)).sum() / 6.0)


def surface_area(V, F):
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return float(0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum())


def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
