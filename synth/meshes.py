"""Seeded synthetic closed triangle meshes.

These generators only build input geometry (vertex positions and triangle
indices); they hold none of the outer-volume / Lloyd arithmetic, so both the
CPU oracle and the CUDA path may consume them.

All meshes are watertight: every undirected edge is shared by exactly two
triangles, with vertices welded by index.  Triangles are oriented with the
outward normal where the construction makes that easy (the occupancy test
itself is orientation-free: it uses crossing parity).

Shapes:
  * ``cube``        axis-aligned closed cube, 12 triangles
  * ``octahedron``  8 triangles
  * ``icosphere``   subdivided icosahedron projected to a sphere
  * ``torus``       (u, v) quad grid split into triangles, optional jitter
  * ``sdf_union``   union of spheres / capsules / rounded boxes, surface
                    extracted by marching tetrahedra on the six-tetrahedron
                    (Kuhn) split of every grid cube; vertices are welded by
                    grid-edge id, which makes the surface closed by
                    construction (every output edge lies in one tetrahedron
                    face, and every interior face is shared by two tetrahedra).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    verts: np.ndarray  # float32 [nv, 3]
    tris: np.ndarray   # int32 [nt, 3]

    @property
    def n_verts(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


def _mesh(v, f) -> Mesh:
    return Mesh(np.ascontiguousarray(np.asarray(v, dtype=np.float32)),
                np.ascontiguousarray(np.asarray(f, dtype=np.int32)))


def cube(lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
         (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)]
    f = [(0, 2, 1), (0, 3, 2),      # z0 (normal -z)
         (4, 5, 6), (4, 6, 7),      # z1
         (0, 1, 5), (0, 5, 4),      # y0
         (3, 7, 6), (3, 6, 2),      # y1
         (0, 4, 7), (0, 7, 3),      # x0
         (1, 2, 6), (1, 6, 5)]      # x1
    return _mesh(v, f)


def octahedron(center=(0.0, 0.0, 0.0), radius=1.0) -> Mesh:
    cx, cy, cz = center
    r = radius
    v = [(cx + r, cy, cz), (cx - r, cy, cz), (cx, cy + r, cz),
         (cx, cy - r, cz), (cx, cy, cz + r), (cx, cy, cz - r)]
    f = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4),
         (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    return _mesh(v, f)


def icosphere(subdiv=2, center=(0.0, 0.0, 0.0), radius=1.0) -> Mesh:
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    V = np.array(v) * radius + np.asarray(center, dtype=np.float64)
    return _mesh(V, f)


def torus(R=1.0, r=0.3, nu=64, nv=32, jitter=0.0, seed=0) -> Mesh:
    """Closed torus: nu x nv quads, each split into two triangles."""
    u = 2.0 * np.pi * np.arange(nu) / nu
    w = 2.0 * np.pi * np.arange(nv) / nv
    U, W = np.meshgrid(u, w, indexing="ij")
    x = (R + r * np.cos(W)) * np.cos(U)
    y = (R + r * np.cos(W)) * np.sin(U)
    z = r * np.sin(W)
    V = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        V = V + rng.uniform(-jitter, jitter, size=V.shape)
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a = ii * nv + jj
    b = ((ii + 1) % nu) * nv + jj
    c = ((ii + 1) % nu) * nv + (jj + 1) % nv
    d = ii * nv + (jj + 1) % nv
    f = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3),
                        np.stack([a, c, d], -1).reshape(-1, 3)])
    return _mesh(V, f)


# ---------------------------------------------------------------------------
# SDF unions
# ---------------------------------------------------------------------------

@dataclass
class SdfScene:
    spheres: np.ndarray   # [n, 4]: cx cy cz r
    capsules: np.ndarray  # [n, 8]: ax ay az bx by bz r pad
    rboxes: np.ndarray    # [n, 16]: c[3], half[3], rounding, R row-major[9]

    def bounds(self):
        lo = np.full(3, np.inf)
        hi = np.full(3, -np.inf)
        for s in self.spheres:
            lo = np.minimum(lo, s[:3] - s[3])
            hi = np.maximum(hi, s[:3] + s[3])
        for c in self.capsules:
            lo = np.minimum(lo, np.minimum(c[:3], c[3:6]) - c[6])
            hi = np.maximum(hi, np.maximum(c[:3], c[3:6]) + c[6])
        for b in self.rboxes:
            rad = np.linalg.norm(b[3:6]) + b[6]
            lo = np.minimum(lo, b[:3] - rad)
            hi = np.maximum(hi, b[:3] + rad)
        return lo, hi

    def sdf(self, P: np.ndarray) -> np.ndarray:
        """Signed distance (negative inside) of the union at points P [..., 3] (float64)."""
        d = np.full(P.shape[:-1], np.inf)
        for s in self.spheres:
            d = np.minimum(d, np.linalg.norm(P - s[:3], axis=-1) - s[3])
        for c in self.capsules:
            a, b, r = c[:3], c[3:6], c[6]
            ab = b - a
            t = np.clip(((P - a) @ ab) / max(float(ab @ ab), 1e-300), 0.0, 1.0)
            q = a + t[..., None] * ab
            d = np.minimum(d, np.linalg.norm(P - q, axis=-1) - r)
        for bx in self.rboxes:
            c, h, rr = bx[:3], bx[3:6], bx[6]
            R = bx[7:16].reshape(3, 3)
            L = (P - c) @ R.T
            q = np.abs(L) - (h - rr)
            outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
            inside = np.minimum(np.max(q, axis=-1), 0.0)
            d = np.minimum(d, outside + inside - rr)
        return d


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def sdf_scene(seed: int, n_spheres=40, n_capsules=20, n_rboxes=0) -> SdfScene:
    """Random primitives: sphere radii U[0.05,0.2], centres U[0,1]^3; capsules with
    centre U[0,1]^3, uniform direction, half-length U[0.05,0.25], radius U[0.03,0.1];
    rounded boxes with half-extents U[0.03,0.12], rounding U[0.005,0.03], uniform rotation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sph = np.concatenate([rng.uniform(0.0, 1.0, (n_spheres, 3)),
                          rng.uniform(0.05, 0.2, (n_spheres, 1))], axis=1)
    caps = np.zeros((n_capsules, 8))
    for i in range(n_capsules):
        c = rng.uniform(0.0, 1.0, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        hl = rng.uniform(0.05, 0.25)
        caps[i, :3] = c - hl * d
        caps[i, 3:6] = c + hl * d
        caps[i, 6] = rng.uniform(0.03, 0.1)
    rbx = np.zeros((n_rboxes, 16))
    for i in range(n_rboxes):
        rbx[i, :3] = rng.uniform(0.0, 1.0, 3)
        rbx[i, 3:6] = rng.uniform(0.03, 0.12, 3)
        rbx[i, 6] = min(rng.uniform(0.005, 0.03), 0.9 * rbx[i, 3:6].min())
        rbx[i, 7:16] = _random_rotation(rng).reshape(-1)
    return SdfScene(sph, caps, rbx)


# Six tetrahedra of the Kuhn split of a unit cube: for each permutation of the
# axes, the path 000 -> e_p0 -> e_p0+e_p1 -> 111.  Corner index = dx + 2 dy + 4 dz.
def _kuhn_tets():
    tets = []
    for p in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        c = [0]
        cur = 0
        for a in p:
            cur |= 1 << a
            c.append(cur)
        tets.append(c)
    return np.array(tets, dtype=np.int64)


_KUHN = _kuhn_tets()


def marching_tetrahedra(f: np.ndarray, origin, spacing) -> Mesh:
    """Closed iso-surface {f = 0} of a sampled field f[G0, G1, G2] (negative = inside).

    Field values exactly 0 are treated as outside.  The field must be positive on
    the whole grid boundary so that the surface is closed."""
    G = np.array(f.shape, dtype=np.int64)
    inside = f < 0.0
    strides = np.array([1, G[0], G[0] * G[1]], dtype=np.int64)
    # cubes that contain a sign change (any corner differs from corner 0)
    cs = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0],
                   [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]], dtype=np.int64)
    base = inside[:-1, :-1, :-1]
    mixed = np.zeros(base.shape, dtype=bool)
    for d in cs[1:]:
        mixed |= inside[d[0]:G[0] - 1 + d[0], d[1]:G[1] - 1 + d[1], d[2]:G[2] - 1 + d[2]] != base
    cube_ijk = np.argwhere(mixed).astype(np.int64)          # [nc, 3]
    corner_ijk = cube_ijk[:, None, :] + cs[None, :, :]      # [nc, 8, 3]
    corner_id = corner_ijk @ strides                        # [nc, 8]
    flat_f = f.reshape(-1, order="F")
    corner_f = flat_f[corner_id]                            # [nc, 8]

    tri_edges_a = []   # per output triangle: 3 edges, each (gid_in, gid_out)
    # per tetrahedron of the split
    for tet in _KUHN:
        vid = corner_id[:, tet]          # [nc, 4]
        vf = corner_f[:, tet]
        ins = vf < 0.0
        n_in = ins.sum(axis=1)
        # --- one inside or three inside: one triangle ---
        for lone_inside in (True, False):
            sel = n_in == (1 if lone_inside else 3)
            if not np.any(sel):
                continue
            ins_s = ins[sel]
            vid_s = vid[sel]
            lone = np.argmax(ins_s if lone_inside else ~ins_s, axis=1)   # index of the lone vertex
            others = np.array([[o for o in range(4) if o != l] for l in range(4)])[lone]  # [n, 3]
            lone_id = vid_s[np.arange(len(lone)), lone]
            oth_id = np.take_along_axis(vid_s, others, axis=1)
            if lone_inside:
                e = np.stack([np.stack([lone_id, oth_id[:, k]], -1) for k in range(3)], axis=1)
            else:
                e = np.stack([np.stack([oth_id[:, k], lone_id], -1) for k in range(3)], axis=1)
            tri_edges_a.append(e)       # [n, 3, 2] (inside id, outside id)
        # --- two inside: quad, two triangles ---
        sel = n_in == 2
        if np.any(sel):
            ins_s = ins[sel]
            vid_s = vid[sel]
            order = np.argsort(~ins_s, axis=1, kind="stable")   # inside first
            a0 = np.take_along_axis(vid_s, order[:, 0:1], 1)[:, 0]
            a1 = np.take_along_axis(vid_s, order[:, 1:2], 1)[:, 0]
            b0 = np.take_along_axis(vid_s, order[:, 2:3], 1)[:, 0]
            b1 = np.take_along_axis(vid_s, order[:, 3:4], 1)[:, 0]
            # quad cycle: (a0,b0) (a0,b1) (a1,b1) (a1,b0)
            e00 = np.stack([a0, b0], -1)
            e01 = np.stack([a0, b1], -1)
            e11 = np.stack([a1, b1], -1)
            e10 = np.stack([a1, b0], -1)
            tri_edges_a.append(np.stack([e00, e01, e11], axis=1))
            tri_edges_a.append(np.stack([e00, e11, e10], axis=1))
    E = np.concatenate(tri_edges_a, axis=0)       # [nt, 3, 2]
    nt = E.shape[0]
    key = E[..., 0] * int(flat_f.size) + E[..., 1]
    uniq, inv = np.unique(key.reshape(-1), return_inverse=True)
    tris = inv.reshape(nt, 3)
    gin = uniq // int(flat_f.size)
    gout = uniq % int(flat_f.size)

    def pos(gid):
        k = gid // strides[2]
        r = gid % strides[2]
        j = r // strides[1]
        i = r % strides[1]
        return np.asarray(origin) + np.stack([i, j, k], -1) * np.asarray(spacing)

    fi = flat_f[gin]
    fo = flat_f[gout]
    t = fi / (fi - fo)
    P = pos(gin) + t[:, None] * (pos(gout) - pos(gin))
    # orient each triangle so its normal points from inside to outside
    V = P[tris]
    n = np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
    e0 = E[:, 0, :]
    outward = pos(e0[:, 1]) - pos(e0[:, 0])
    flip = (n * outward).sum(-1) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return _mesh(P, tris)


def _primitive_boxes(scene):
    """(kind, index, lo, hi) bounding boxes of every primitive."""
    out = []
    for i, s in enumerate(scene.spheres):
        out.append(("s", i, s[:3] - s[3], s[:3] + s[3]))
    for i, c in enumerate(scene.capsules):
        out.append(("c", i, np.minimum(c[:3], c[3:6]) - c[6], np.maximum(c[:3], c[3:6]) + c[6]))
    for i, b in enumerate(scene.rboxes):
        rad = np.linalg.norm(b[3:6]) + b[6]
        out.append(("b", i, b[:3] - rad, b[:3] + rad))
    return out


def _primitive_sdf(scene, kind, i, P):
    if kind == "s":
        s = scene.spheres[i]
        return np.linalg.norm(P - s[:3], axis=-1) - s[3]
    if kind == "c":
        c = scene.capsules[i]
        a, b, r = c[:3], c[3:6], c[6]
        ab = b - a
        t = np.clip(((P - a) @ ab) / max(float(ab @ ab), 1e-300), 0.0, 1.0)
        return np.linalg.norm(P - (a + t[..., None] * ab), axis=-1) - r
    bx = scene.rboxes[i]
    c, h, rr = bx[:3], bx[3:6], bx[6]
    R = bx[7:16].reshape(3, 3)
    L = (P - c) @ R.T
    q = np.abs(L) - (h - rr)
    return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(np.max(q, axis=-1), 0.0) - rr


def sdf_union_mesh(seed: int, grid: int, n_spheres=40, n_capsules=20, n_rboxes=0) -> Mesh:
    """Watertight surface of a seeded SDF union on a grid^3 sampling of its padded AABB.

    Each primitive updates the field only inside its bounding box widened by
    three cells; elsewhere the field keeps a positive placeholder.  Every grid
    edge that changes sign lies within one cell of the surface, hence inside
    the widened box of each primitive that can be the minimum there, so the
    sign everywhere and the values used for interpolation are those of the
    full union."""
    scene = sdf_scene(seed, n_spheres, n_capsules, n_rboxes)
    lo, hi = scene.bounds()
    ext = hi - lo
    pad = 0.02 * ext.max()
    lo = lo - pad
    hi = hi + pad
    spacing = (hi - lo) / (grid - 1)
    fld = np.full((grid, grid, grid), 1.0, dtype=np.float64)
    for kind, i, plo, phi in _primitive_boxes(scene):
        a = np.maximum(np.floor((plo - lo) / spacing).astype(np.int64) - 3, 1)
        b = np.minimum(np.ceil((phi - lo) / spacing).astype(np.int64) + 3, grid - 2)
        if np.any(a > b):
            continue
        xs = lo[0] + spacing[0] * np.arange(a[0], b[0] + 1)
        ys = lo[1] + spacing[1] * np.arange(a[1], b[1] + 1)
        zs = lo[2] + spacing[2] * np.arange(a[2], b[2] + 1)
        X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
        d = _primitive_sdf(scene, kind, i, np.stack([X, Y, Z], -1))
        sub = fld[a[0]:b[0] + 1, a[1]:b[1] + 1, a[2]:b[2] + 1]
        np.minimum(sub, d, out=sub)
    return marching_tetrahedra(fld, lo, spacing)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def torus_4096(seed=1000) -> Mesh:
    """Closed torus R=1.0, r=0.3, 64x32 quads -> 4,096 triangles, coordinates jittered U[-0.002, 0.002]."""
    return torus(1.0, 0.3, 64, 32, jitter=0.002, seed=seed)


# grid resolutions giving roughly the target triangle counts for the seeded scenes
SDF_GRID_200K = 74


def sdf_union_200k(seed=2000, grid=SDF_GRID_200K) -> Mesh:
    """SDF union of 40 spheres and 20 capsules, ~200k watertight triangles."""
    return sdf_union_mesh(seed, grid, 40, 20, 0)


SDF_GRID_1M = 165
SDF_GRID_2M = 206


def sdf_union_1m(seed=4000, grid=SDF_GRID_1M) -> Mesh:
    """SDF union of 40 spheres and 20 capsules at a finer sampling, ~1M triangles."""
    return sdf_union_mesh(seed, grid, 40, 20, 0)


def sdf_union_2m(seed=5000, grid=SDF_GRID_2M) -> Mesh:
    """SDF union of 200 spheres, 100 capsules and 50 rounded boxes, ~2M triangles."""
    return sdf_union_mesh(seed, grid, 200, 100, 50)


def watertight_edges(tris: np.ndarray) -> bool:
    """True when every undirected edge is used by exactly two triangles."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.sort(e, axis=1)
    _, cnt = np.unique(e[:, 0].astype(np.int64) * (int(tris.max()) + 1) + e[:, 1], return_counts=True)
    return bool(np.all(cnt == 2))


def subdivided_tetrahedron(jitter=0.0, seed=0) -> Mesh:
    """Regular tetrahedron with every face split into four (16 triangles), welded."""
    v = [np.array(p, dtype=np.float64) for p in ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1))]
    f = [(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)]
    cache = {}

    def mid(a, b):
        key = (min(a, b), max(a, b))
        if key not in cache:
            v.append(0.5 * (v[a] + v[b]))
            cache[key] = len(v) - 1
        return cache[key]

    nf = []
    for a, b, c in f:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    V = np.array(v)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        V = V + rng.uniform(-jitter, jitter, size=V.shape)
    return _mesh(V, nf)


def sdf_batch(count: int, seed: int = 3000):
    """Meshes of uneven size for batched runs: SDF unions of 10 spheres and 5
    capsules sampled on a log-uniform grid (about 1k to 100k triangles), each
    with a lattice size drawn from {128, 192, 256, 320, 384}.  Returns a list of
    (mesh, N)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        grid = int(round(np.exp(rng.uniform(np.log(12), np.log(110)))))
        N = int(rng.choice([128, 192, 256, 320, 384]))
        out.append((sdf_union_mesh(seed + 1 + i, grid, 10, 5, 0), N))
    return out
