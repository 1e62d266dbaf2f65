"""CPU oracle for the outer-volume / Lloyd path (arXiv 2203.10521).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product library
never does.  The arithmetic lives in ``obb_oracle.c`` (plain C, one lattice
point at a time); this module is ctypes marshalling plus the orchestration
of the Lloyd step and the top-down tree build written as plain loops.

Every function states the passage of the paper it follows.  Pins (tests that
tie the oracle to something other than itself) live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "obb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

S_BITS = 8    # fixed-point fraction bits of the snapped vertices
Q_BITS = 24   # fraction bits of the quantised box normals


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction; OpenMP where the
    compiler has it, for the loops over independent columns and slices)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
        _lib.orc_set_threads(1)
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's loops over independent columns, slices and
    boxes (1 by default); returns the count in effect (1 without OpenMP)."""
    L = lib()
    L.orc_set_threads(int(n))
    return int(L.orc_threads())


def threads() -> int:
    return int(lib().orc_threads())


class RoundStats(C.Structure):
    _fields_ = [("proposals", C.c_int64), ("accepted", C.c_int64),
                ("gain", C.c_int64), ("evals", C.c_int64)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _declare(L):
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    L.orc_set_threads.argtypes = [i32]
    L.orc_threads.restype = C.c_int32
    L.orc_lattice_frame.argtypes = [vp, i64, i32, vp, vp]
    L.orc_snap.argtypes = [vp, i64, vp, vp, vp]
    L.orc_occupancy_columns.argtypes = [vp, vp, i64, i32, vp, i64, vp, vp]
    L.orc_column_crossing_counts.argtypes = [vp, vp, i64, vp, i64, vp]
    L.orc_frame_normals.argtypes = [vp, i64, vp, vp]
    L.orc_quantize_boxes.argtypes = [vp, i64, vp, vp, vp, vp]
    L.orc_quantize_boxes.restype = C.c_int
    L.orc_box_aabb.argtypes = [vp, vp, vp]
    L.orc_box_aabb.restype = C.c_int
    L.orc_outer_volume.argtypes = [vp, vp, i32, vp, vp, i64, vp, vp, vp]
    L.orc_outer_volume.restype = C.c_int
    L.orc_tight_bounds.argtypes = [vp, vp, i64, vp, i32, vp, vp]
    L.orc_lloyd_moves.argtypes = [vp, vp, vp, i64, vp, vp, i32, vp, vp, vp, vp, vp, i32, i32, vp]
    L.orc_lloyd_moves.restype = C.c_int
    L.orc_unit_moves.argtypes = [vp, vp, vp, i64, vp, i32, vp, vp, i32, vp, vp, vp, vp, vp, i32, i32, vp]
    L.orc_unit_moves.restype = C.c_int
    L.orc_flood_partition.argtypes = [vp, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp]
    L.orc_flood_partition.restype = C.c_int
    L.orc_moments.argtypes = [vp, vp, i64, vp, i32, vp, vp]
    L.orc_covariance_from_moments.argtypes = [vp, vp]
    L.orc_covariance_from_moments.restype = C.c_int
    L.orc_jacobi3.argtypes = [vp, vp, vp]
    L.orc_refit.argtypes = [vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    L.orc_refit.restype = C.c_int
    L.orc_cluster_frames.argtypes = [vp, vp, i64, vp, i32, vp, vp, vp]
    L.orc_median_split.argtypes = [vp, vp, i64, vp, i32, vp, vp]
    L.orc_median_split.restype = C.c_int


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# ---------------------------------------------------------------------------
# Lattice (Sec. 3: the solid Omega(X); lattice discretisation of Eq. 3-4)
# ---------------------------------------------------------------------------

def lattice_frame(verts, N):
    """lo, h of the N^3 cell-centred lattice over the vertex AABB."""
    V = _c(verts, np.float32)
    lo = np.zeros(3)
    h = np.zeros(3)
    lib().orc_lattice_frame(_p(V), V.shape[0], int(N), _p(lo), _p(h))
    return lo, h


def snap(verts, lo, h):
    """Fixed-point vertices U = rint(((x - lo)/h - 1/2) * 2^S)."""
    V = _c(verts, np.float32)
    U = np.zeros(V.shape, dtype=np.int32)
    lib().orc_snap(_p(V), V.shape[0], _p(_c(lo, np.float64)), _p(_c(h, np.float64)), _p(U))
    return U


@dataclass
class Occupancy:
    """Per-point solid occupancy, filled column by column.

    occ[k, j, i] in {0, 1}; known[k, j] marks the columns computed so far."""
    N: int
    U: np.ndarray
    F: np.ndarray
    occ: np.ndarray = None
    known: np.ndarray = None

    def __post_init__(self):
        if self.occ is None:
            self.occ = np.zeros((self.N, self.N, self.N), dtype=np.uint8)
            self.known = np.zeros((self.N, self.N), dtype=np.uint8)

    def fill_columns(self, cols):
        """Compute the columns cols[:, (j, k)] not yet known."""
        cols = np.asarray(cols, dtype=np.int64).reshape(-1, 2)
        if cols.size == 0:
            return
        need = cols[self.known[cols[:, 1], cols[:, 0]] == 0]
        if need.size == 0:
            return
        need = _c(np.unique(need, axis=0), np.int32)
        lib().orc_occupancy_columns(_p(self.U), _p(self.F), self.F.shape[0], self.N,
                                    _p(need), need.shape[0], _p(self.occ), _p(self.known))

    def fill_all(self):
        j, k = np.meshgrid(np.arange(self.N), np.arange(self.N), indexing="ij")
        self.fill_columns(np.stack([j.ravel(), k.ravel()], -1))

    def fill_boxes(self, n, bnd):
        """Compute every in-domain column that the given boxes' AABBs cover."""
        cols = []
        for b in range(n.shape[0]):
            ab = box_aabb(n[b], bnd[b])
            j0, j1 = max(ab[2], 0), min(ab[3], self.N - 1)
            k0, k1 = max(ab[4], 0), min(ab[5], self.N - 1)
            if j0 > j1 or k0 > k1:
                continue
            jj, kk = np.meshgrid(np.arange(j0, j1 + 1), np.arange(k0, k1 + 1), indexing="ij")
            m = self.known[kk, jj] == 0
            if m.any():
                cols.append(np.stack([jj[m], kk[m]], -1))
        if cols:
            self.fill_columns(np.concatenate(cols))


def occupancy(U, F, N, cols=None):
    """Occupancy object; all columns when cols is None."""
    o = Occupancy(int(N), _c(U, np.int32), _c(F, np.int32))
    if cols is None:
        o.fill_all()
    else:
        o.fill_columns(cols)
    return o


def column_crossings(U, F, cols):
    U = _c(U, np.int32)
    F = _c(F, np.int32)
    cols = _c(cols, np.int32).reshape(-1, 2)
    out = np.zeros(cols.shape[0], dtype=np.int64)
    lib().orc_column_crossing_counts(_p(U), _p(F), F.shape[0], _p(cols), cols.shape[0], _p(out))
    return out


# ---------------------------------------------------------------------------
# Boxes (Eq. 4 per box) and their quantisation
# ---------------------------------------------------------------------------

def frame_normals(R, h):
    R = _c(R, np.float64).reshape(-1, 9)
    n = np.zeros((R.shape[0], 9), dtype=np.int32)
    lib().orc_frame_normals(_p(R), R.shape[0], _p(_c(h, np.float64)), _p(n))
    return n


def quantize_boxes(boxes, lo, h):
    """FP32 boxes [K, 12] (c, axis0, axis1, half) -> (n [K, 9] int32, bounds [K, 6] int64)."""
    B = _c(boxes, np.float32).reshape(-1, 12)
    n = np.zeros((B.shape[0], 9), dtype=np.int32)
    bnd = np.zeros((B.shape[0], 6), dtype=np.int64)
    rc = lib().orc_quantize_boxes(_p(B), B.shape[0], _p(_c(lo, np.float64)), _p(_c(h, np.float64)),
                                  _p(n), _p(bnd))
    if rc:
        raise ValueError("invalid box")
    return n, bnd


def box_aabb(n, bnd):
    out = np.zeros(6, dtype=np.int64)
    rc = lib().orc_box_aabb(_p(_c(n, np.int32)), _p(_c(bnd, np.int64)), _p(out))
    if rc:
        raise ValueError(f"box_aabb failed ({rc})")
    return out


def outer_volume(occ: Occupancy, n, bnd, want_domain=False):
    """Eq. 4: exact count of unoccupied lattice points in each box, and the box's
    point count (and, with want_domain, its points inside [0, N)^3)."""
    n = _c(n, np.int32).reshape(-1, 9)
    bnd = _c(bnd, np.int64).reshape(-1, 6)
    occ.fill_boxes(n, bnd)
    cnt = np.zeros(n.shape[0], dtype=np.uint64)
    tot = np.zeros(n.shape[0], dtype=np.uint64)
    dom = np.zeros(n.shape[0], dtype=np.uint64)
    rc = lib().orc_outer_volume(_p(occ.occ), _p(occ.known), occ.N, _p(n), _p(bnd), n.shape[0],
                                _p(cnt), _p(tot), _p(dom))
    if rc:
        raise RuntimeError(f"orc_outer_volume failed ({rc})")
    return (cnt, tot, dom) if want_domain else (cnt, tot)


def tight_bounds(U, F, assign, K, n):
    bnd = np.zeros((K, 6), dtype=np.int64)
    lib().orc_tight_bounds(_p(_c(U, np.int32)), _p(_c(F, np.int32)), F.shape[0],
                           _p(_c(assign, np.int32)), int(K), _p(_c(n, np.int32)), _p(bnd))
    return bnd


# ---------------------------------------------------------------------------
# Refit pieces (covariance frame, FP64 Jacobi)
# ---------------------------------------------------------------------------

def moments(V, F, assign, K, center):
    mom = np.zeros((K, 10))
    lib().orc_moments(_p(_c(V, np.float32)), _p(_c(F, np.int32)), F.shape[0], _p(_c(assign, np.int32)),
                      int(K), _p(_c(center, np.float64)), _p(mom))
    return mom


def covariance(mom):
    cov = np.zeros(6)
    rc = lib().orc_covariance_from_moments(_p(_c(mom, np.float64)), _p(cov))
    return None if rc else cov


def jacobi3(cov6):
    R = np.zeros(9)
    ev = np.zeros(3)
    lib().orc_jacobi3(_p(_c(cov6, np.float64)), _p(R), _p(ev))
    return R.reshape(3, 3), ev


def cluster_frames(V, F, assign, K, center, fallback=None):
    if fallback is None:
        fallback = np.tile(np.eye(3).reshape(1, 9), (K, 1))
    fr = np.zeros((K, 9))
    lib().orc_cluster_frames(_p(_c(V, np.float32)), _p(_c(F, np.int32)), F.shape[0],
                             _p(_c(assign, np.int32)), int(K), _p(_c(center, np.float64)),
                             _p(_c(fallback, np.float64)), _p(fr))
    return fr


# ---------------------------------------------------------------------------
# Mesh topology (edge adjacency) -- plain dictionary walk
# ---------------------------------------------------------------------------

def edge_adjacency(F):
    """adj[t, e] = the other triangle on edge e = (v_e, v_{e+1}) of t.

    Raises ValueError unless every undirected edge has exactly two triangles."""
    F = np.asarray(F, dtype=np.int64)
    edges = {}
    for t in range(F.shape[0]):
        for e in range(3):
            a, b = int(F[t, e]), int(F[t, (e + 1) % 3])
            edges.setdefault((min(a, b), max(a, b)), []).append((t, e))
    adj = np.full((F.shape[0], 3), -1, dtype=np.int32)
    for key, lst in edges.items():
        if len(lst) != 2:
            raise ValueError(f"edge {key} has {len(lst)} triangles")
        (t0, e0), (t1, e1) = lst
        adj[t0, e0] = t1
        adj[t1, e1] = t0
    return adj


# ---------------------------------------------------------------------------
# Layer state and the Lloyd step (Sec. 4.2.1, Eq. 11-13)
# ---------------------------------------------------------------------------

@dataclass
class Layer:
    assign: np.ndarray      # int32 [T]
    parent: np.ndarray      # int32 [K]
    frames: np.ndarray      # float64 [K, 9], rows = box axes
    n: np.ndarray           # int32 [K, 9]
    bnd: np.ndarray         # int64 [K, 6]
    obv: np.ndarray         # uint64 [K]
    level: np.ndarray = None  # int32 [K], descent level (theta = 2^-(5 + level))

    def __post_init__(self):
        if self.level is None:
            self.level = np.zeros(self.parent.shape[0], dtype=np.int32)

    @property
    def K(self):
        return int(self.parent.shape[0])

    def copy(self):
        return Layer(self.assign.copy(), self.parent.copy(), self.frames.copy(), self.n.copy(),
                     self.bnd.copy(), self.obv.copy(), self.level.copy())


@dataclass
class Problem:
    """A mesh on its lattice, with the oracle's per-point occupancy."""
    V: np.ndarray
    F: np.ndarray
    N: int
    lo: np.ndarray = None
    h: np.ndarray = None
    U: np.ndarray = None
    adj: np.ndarray = None
    occ: Occupancy = None
    center: np.ndarray = field(default=None)

    def __post_init__(self):
        self.V = _c(self.V, np.float32)
        self.F = _c(self.F, np.int32)
        self.lo, self.h = lattice_frame(self.V, self.N)
        self.U = snap(self.V, self.lo, self.h)
        if self.adj is None:
            self.adj = edge_adjacency(self.F)
        self.occ = Occupancy(self.N, self.U, self.F)
        # moments are taken about the lattice AABB centre lo + N h / 2
        self.center = self.lo + 0.5 * self.N * self.h


def layer_from_frames(P: Problem, assign, parent, frames) -> Layer:
    """Layer state from an assignment and given frames: quantised normals, tight bounds, exact OBV."""
    assign = _c(assign, np.int32)
    parent = _c(parent, np.int32)
    K = parent.shape[0]
    frames = _c(frames, np.float64).reshape(K, 9)
    n = frame_normals(frames, P.h)
    bnd = tight_bounds(P.U, P.F, assign, K, n)
    obv, _ = outer_volume(P.occ, n, bnd)
    return Layer(assign, parent, frames.copy(), n, bnd, obv)


def layer_init(P: Problem, assign, parent, fallback=None) -> Layer:
    """New layer seeded from covariance frames of the given assignment."""
    assign = _c(assign, np.int32)
    K = int(np.asarray(parent).shape[0])
    fr = cluster_frames(P.V, P.F, assign, K, P.center, fallback)
    return layer_from_frames(P, assign, parent, fr)


def lloyd_moves(P: Problem, L: Layer, rounds: int):
    """Partition rounds of one Lloyd step (in place). Returns per-round stats."""
    # every column any candidate box may touch is inside the AABB of the union
    # of grown boxes; the C side reports -3 if one is missing, in which case
    # the needed columns are computed and the step is retried from a copy.
    st = (RoundStats * max(rounds, 1))()
    while True:
        work = L.copy()
        rc = lib().orc_lloyd_moves(_p(P.U), _p(P.F), _p(P.adj), P.F.shape[0], _p(work.assign),
                                   _p(work.parent), work.K, _p(work.n), _p(work.bnd), _p(work.obv),
                                   _p(P.occ.occ), _p(P.occ.known), P.N, int(rounds), st)
        if rc == -3:
            P.occ.fill_all()
            continue
        if rc < 0:
            raise RuntimeError(f"orc_lloyd_moves failed ({rc})")
        moved = np.nonzero(L.assign != work.assign)[0]
        L.level[L.assign[moved]] = 0       # a new member set restarts the descent
        L.level[work.assign[moved]] = 0
        L.assign[:], L.bnd[:], L.obv[:] = work.assign, work.bnd, work.obv
        return [dict(proposals=s.proposals, accepted=s.accepted, gain=s.gain, evals=s.evals)
                for s in st[:rc]]


def refit(P: Problem, L: Layer):
    """Box parameter update (Sec. 4.2.1 step 2, restated as a covariance frame kept only if the exact OBV drops)."""
    acc = np.zeros(L.K, dtype=np.uint8)
    while True:
        fr, n, bnd, obv = L.frames.copy(), L.n.copy(), L.bnd.copy(), L.obv.copy()
        rc = lib().orc_refit(_p(P.V), _p(P.U), _p(P.F), P.F.shape[0], _p(L.assign), L.K, _p(P.center),
                             _p(P.h), _p(fr), _p(n), _p(bnd), _p(obv), _p(P.occ.occ), _p(P.occ.known),
                             P.N, _p(acc))
        if rc == -3:
            P.occ.fill_all()
            continue
        if rc < 0:
            raise RuntimeError(f"orc_refit failed ({rc})")
        L.frames[:], L.n[:], L.bnd[:], L.obv[:] = fr, n, bnd, obv
        return acc


def probe_frame(R, level, p):
    out = np.zeros(9)
    L = lib()
    if not hasattr(L, "_pf_declared"):
        L.orc_probe_frame.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
        L.orc_descent_step.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int32]
        L.orc_descent_step.restype = C.c_int
        L._pf_declared = True
    L.orc_probe_frame(_p(_c(R, np.float64)), int(level), int(p), _p(out))
    return out.reshape(3, 3)


def descent_step(P: Problem, L: Layer):
    """One rotation-probe step of the box update (Sec. 4.2.1 step 2, restated)."""
    probe_frame(np.eye(3), 0, 0)     # declares the C signatures
    while True:
        fr, n, bnd, obv, lev = L.frames.copy(), L.n.copy(), L.bnd.copy(), L.obv.copy(), L.level.copy()
        rc = lib().orc_descent_step(_p(P.U), _p(P.F), P.F.shape[0], _p(L.assign), L.K, _p(P.h), _p(fr), _p(n),
                                    _p(bnd), _p(obv), _p(lev), _p(P.occ.occ), _p(P.occ.known), P.N)
        if rc == -3:
            P.occ.fill_all()
            continue
        if rc < 0:
            raise RuntimeError(f"orc_descent_step failed ({rc})")
        L.frames[:], L.n[:], L.bnd[:], L.obv[:], L.level[:] = fr, n, bnd, obv, lev
        return rc


def lloyd_step(P: Problem, L: Layer, rounds: int = 16, do_refit=1, descent_steps: int = 2):
    """One Lloyd iteration: partition rounds, then the box update
    (do_refit: 0 none, 1 covariance frame, 2 rotation descent, 3 both)."""
    st = lloyd_moves(P, L, rounds)
    mode = int(do_refit)
    acc = refit(P, L) if mode & 1 else np.zeros(L.K, dtype=np.uint8)
    if mode & 2:
        for _ in range(descent_steps):
            descent_step(P, L)
    return st, acc


def unit_moves(P: Problem, up: Layer, low: Layer, rounds: int):
    """Partition rounds between levels (Sec. 4.2.2, bottom-up merging): the
    clusters of `low` move as whole units between sibling clusters of `up`.
    Updates low.parent (the unit -> cluster map), up.assign, up.bnd, up.obv in
    place.  Returns per-round stats."""
    st = (RoundStats * max(rounds, 1))()
    T = P.F.shape[0]
    while True:
        cl = low.parent.copy()
        bnd, obv = up.bnd.copy(), up.obv.copy()
        rc = lib().orc_unit_moves(_p(P.U), _p(P.F), _p(P.adj), T, _p(low.assign), low.K, _p(cl), _p(up.parent),
                                  up.K, _p(up.n), _p(bnd), _p(obv), _p(P.occ.occ), _p(P.occ.known), P.N,
                                  int(rounds), st)
        if rc == -3:
            P.occ.fill_all()
            continue
        if rc < 0:
            raise RuntimeError(f"orc_unit_moves failed ({rc})")
        moved = np.nonzero(cl != low.parent)[0]
        up.level[low.parent[moved]] = 0     # a new member set restarts the descent
        up.level[cl[moved]] = 0
        low.parent[:] = cl
        up.assign[:] = cl[low.assign]
        up.bnd[:], up.obv[:] = bnd, obv
        return [dict(proposals=s.proposals, accepted=s.accepted, gain=s.gain, evals=s.evals)
                for s in st[:rc]]


def unit_lloyd_step(P: Problem, up: Layer, low: Layer, rounds: int = 16, do_refit=1, descent_steps: int = 2):
    """One Lloyd iteration of level `up` with the clusters of `low` as units,
    then the box update of `up` (same modes as lloyd_step)."""
    st = unit_moves(P, up, low, rounds)
    mode = int(do_refit)
    acc = refit(P, up) if mode & 1 else np.zeros(up.K, dtype=np.uint8)
    if mode & 2:
        for _ in range(descent_steps):
            descent_step(P, up)
    return st, acc


def tree_eq7(layers):
    """Eq. 7 of a list of layers (root first) in lattice points."""
    return eq7_score([L.obv for L in layers], len(layers) - 1)


def tree_sweeps(P: Problem, layers, sweeps: int = 1, iters: int = 2, rounds: int = 16, do_refit=1):
    """Reciprocating optimisation between levels (Sec. 4.2.2).  Each sweep
    first merges bottom-up: for levels D-1 .. 1 the clusters of the level
    below are the units; the pass stops at the first level whose Eq. 7 does
    not strictly drop.  Then it decomposes top-down: levels 1 .. D again, with
    units at the inner levels and triangles at the leaves.  Every level runs
    up to `iters` Lloyd iterations and stops early on one that changes nothing.
    Returns Eq. 7 before and after each sweep."""
    D = len(layers) - 1
    hist = [tree_eq7(layers)]

    def level(lev):
        for _ in range(iters):
            if lev < D:
                st, acc = unit_lloyd_step(P, layers[lev], layers[lev + 1], rounds, do_refit)
            else:
                st, acc = lloyd_step(P, layers[lev], rounds, do_refit)
            if sum(s["accepted"] for s in st) == 0 and not acc.any():
                break

    for _ in range(sweeps):
        for lev in range(D - 1, 0, -1):
            e0 = tree_eq7(layers)
            level(lev)
            if not tree_eq7(layers) < e0:
                break
        for lev in range(1, D + 1):
            level(lev)
        hist.append(tree_eq7(layers))
    return hist


def box_centres(P: Problem, L: Layer):
    """World-space centres (FP64) of a layer's quantised boxes: the midpoint of
    each slab, mapped back through the frame."""
    s = 4294967296.0 / float(np.max(P.h))
    base = L.frames.reshape(-1, 3, 3) @ (P.lo + 0.5 * P.h)
    mid = 0.5 * (L.bnd[:, 0::2].astype(np.float64) + L.bnd[:, 1::2].astype(np.float64)) / s + base
    return np.einsum("kab,ka->kb", L.frames.reshape(-1, 3, 3), mid)


def flood_partition(P: Problem, group, box_group, n, centre):
    """Patch division by flooding (Sec. 4.2.1 step 1), sequential in the
    paper's priority order; see orc_flood_partition.  Returns (assign, bnd,
    obv) with exact tight slabs and outer volumes."""
    T = P.F.shape[0]
    group = _c(group, np.int32)
    box_group = _c(box_group, np.int32)
    n = _c(n, np.int32).reshape(-1, 9)
    centre = _c(centre, np.float64).reshape(-1, 3)
    K = box_group.shape[0]
    while True:
        assign = np.zeros(T, np.int32)
        bnd = np.zeros((K, 6), np.int64)
        obv = np.zeros(K, np.uint64)
        rc = lib().orc_flood_partition(_p(P.V), _p(P.U), _p(P.F), _p(P.adj), T, _p(group), K, _p(box_group),
                                       _p(n), _p(centre), _p(P.occ.occ), _p(P.occ.known), P.N, _p(assign),
                                       _p(bnd), _p(obv))
        if rc == -3:
            P.occ.fill_all()
            continue
        if rc < 0:
            raise ValueError("a box has no triangle of its group to seed from")
        return assign, bnd, obv


def adjust_step(P: Problem, L: Layer, iters: int = 2, rounds: int = 16, do_refit=1):
    """Box adjustment for local minima (Sec. 4.2.1 step 3), in place.  The
    least important box k (fewest triangles, ties -> smaller index; only boxes
    with a sibling) gives its triangles to the sibling sharing most triangle
    edges with it (ties -> smaller index; none -> the smallest sibling index),
    whose box is recomputed.  Then the sibling j with the largest outer volume
    (ties -> smaller index) is split at the median of its triangles along its
    major axis (key n_0 . (U_p + U_q + U_r), ties by triangle index): the
    first ceil(n / 2) stay in j, the rest form box k, which takes j's frame.
    `iters` Lloyd iterations follow.  The adjustment is kept only if the
    layer's total outer volume is then smaller; otherwise the layer is
    restored.  Returns (kept, k, j)."""
    saved = L.copy()
    total0 = int(L.obv.astype(np.int64).sum())
    K = L.K
    size = np.bincount(L.assign, minlength=K)
    nsib = np.bincount(L.parent, minlength=K)[L.parent]
    elig = np.nonzero(nsib >= 2)[0]
    if elig.size == 0:
        return False, -1, -1
    k = int(elig[np.lexsort((elig, size[elig]))[0]])
    g = L.parent[k]
    sibs = [c for c in range(K) if L.parent[c] == g and c != k]
    edges = np.zeros(K, np.int64)
    for t in np.nonzero(L.assign == k)[0]:
        for u in P.adj[t]:
            c = L.assign[u]
            if c != k and L.parent[c] == g:
                edges[c] += 1
    m = max(sibs, key=lambda c: (edges[c], -c))
    L.assign[L.assign == k] = m

    def rebox(cs):
        cs = list(cs)
        b = tight_bounds(P.U, P.F, L.assign, K, L.n)
        for c in cs:
            L.bnd[c] = b[c]
        L.obv[cs] = outer_volume(P.occ, L.n[cs], L.bnd[cs])[0]

    rebox([m])
    j = max(sibs, key=lambda c: (int(L.obv[c]), -c))
    tj = np.nonzero(L.assign == j)[0]
    if tj.size < 2:
        L.assign[:], L.frames[:], L.n[:], L.bnd[:], L.obv[:], L.level[:] = (
            saved.assign, saved.frames, saved.n, saved.bnd, saved.obv, saved.level)
        return False, k, j
    S = P.U[P.F[tj]].astype(np.int64).sum(1)
    key = S @ L.n[j, 0:3].astype(np.int64)
    order = tj[np.lexsort((tj, key))]
    L.assign[order[(tj.size + 1) // 2:]] = k
    L.frames[k] = L.frames[j]
    L.n[k] = L.n[j]
    rebox([j, k])
    L.level[[k, m, j]] = 0
    for _ in range(iters):
        lloyd_step(P, L, rounds, do_refit)
    if int(L.obv.astype(np.int64).sum()) < total0:
        return True, k, j
    L.assign[:], L.frames[:], L.n[:], L.bnd[:], L.obv[:], L.level[:] = (
        saved.assign, saved.frames, saved.n, saved.bnd, saved.obv, saved.level)
    return False, k, j


def median_split(P: Problem, L: Layer):
    child = np.zeros(P.F.shape[0], dtype=np.int32)
    rc = lib().orc_median_split(_p(P.U), _p(P.F), P.F.shape[0], _p(L.assign), L.K, _p(L.n), _p(child))
    if rc:
        raise ValueError("a cluster has fewer than two triangles")
    return child


def eq7_score(obv_per_level, depth):
    """Eq. 7 with the weights of Sec. 5: level L (root 0, leaves `depth`)
    weighs (depth - L) + 1, i.e. leaves 1, their parents 2, ...  Returns the
    weighted sum of per-level outer volumes (in lattice points)."""
    return sum(float(depth - L + 1) * float(np.sum(np.asarray(o, dtype=np.float64)))
               for L, o in enumerate(obv_per_level))


def build_tree(P: Problem, depth: int, iters: int, rounds: int = 16):
    """Top-down construction (Sec. 4.2.2): root box, then per level a median
    split of every node into two children followed by `iters` Lloyd steps
    restricted to siblings.  Returns the list of layers (root first)."""
    T = P.F.shape[0]
    root = layer_init(P, np.zeros(T, dtype=np.int32), np.zeros(1, dtype=np.int32))
    layers = [root]
    for lev in range(1, depth + 1):
        prev = layers[-1]
        child = median_split(P, prev)
        K = 2 * prev.K
        parent = (np.arange(K) // 2).astype(np.int32)
        fallback = np.repeat(prev.frames, 2, axis=0)
        L = layer_init(P, child, parent, fallback)
        for _ in range(iters):
            st, acc = lloyd_step(P, L, rounds)
            if sum(s["accepted"] for s in st) == 0 and not acc.any():
                break
        layers.append(L)
    return layers


# ---------------------------------------------------------------------------
# Learned surrogate: its input features and a plain FP64 network
# ---------------------------------------------------------------------------

SURROGATE_INPUTS = 524
MLP_HIDDEN = 128


def surrogate_features(occ: Occupancy, n, bnd, return_ties=False):
    """Features of quantised boxes: 12 box parameters (FP64 from exact
    integers, rounded once to FP32) + an 8^3 occupancy patch at the exact
    rational sample points of the box's own frame.  With return_ties, also a
    [K, 512] uint8 mask of the patch points lying within 1e-3 of a rounding
    tie on some axis."""
    n = _c(n, np.int32).reshape(-1, 9)
    bnd = _c(bnd, np.int64).reshape(-1, 6)
    L = lib()
    if not hasattr(L, "_sf_declared"):
        L.orc_surrogate_features.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                             C.c_int64, C.c_void_p, C.c_void_p]
        L.orc_surrogate_features.restype = C.c_int
        L._sf_declared = True
    occ.fill_boxes(n, bnd)
    out = np.zeros((n.shape[0], SURROGATE_INPUTS), np.float32)
    ties = np.zeros((n.shape[0], 512), np.uint8)
    rc = L.orc_surrogate_features(_p(occ.occ), _p(occ.known), occ.N, _p(n), _p(bnd), n.shape[0], _p(out),
                                  _p(ties))
    if rc == -3:
        occ.fill_all()
        rc = L.orc_surrogate_features(_p(occ.occ), _p(occ.known), occ.N, _p(n), _p(bnd), n.shape[0], _p(out),
                                      _p(ties))
    if rc:
        raise RuntimeError(f"orc_surrogate_features failed ({rc})")
    return (out, ties) if return_ties else out


def mlp_unpack(params):
    """Flat parameter vector -> [(W, b)] for 524 -> 128 -> 128 -> 128 -> 1 (W [in][out])."""
    p = np.asarray(params, dtype=np.float64)
    sizes = [(SURROGATE_INPUTS, MLP_HIDDEN), (MLP_HIDDEN, MLP_HIDDEN), (MLP_HIDDEN, MLP_HIDDEN), (MLP_HIDDEN, 1)]
    out, o = [], 0
    for fi, fo in sizes:
        W = p[o:o + fi * fo].reshape(fi, fo)
        o += fi * fo
        b = p[o:o + fo]
        o += fo
        out.append((W, b))
    assert o == p.size
    return out


def mlp_forward(params, X):
    """ReLU hidden layers, sigmoid output (the predicted empty fraction); FP64."""
    layers = mlp_unpack(params)
    h = np.asarray(X, dtype=np.float64)
    acts = [h]
    for i, (W, b) in enumerate(layers):
        z = h @ W + b
        h = np.maximum(z, 0.0) if i < 3 else 1.0 / (1.0 + np.exp(-z))
        acts.append(h)
    return h[:, 0], acts


def mlp_loss_grad(params, X, T):
    """Mean squared error of the fraction and its gradient (backpropagation), FP64."""
    layers = mlp_unpack(params)
    y, acts = mlp_forward(params, X)
    B = y.shape[0]
    T = np.asarray(T, dtype=np.float64)
    loss = float(np.mean((y - T) ** 2))
    dz = (2.0 * (y - T) / B * y * (1.0 - y))[:, None]
    grads = [None] * 4
    for i in range(3, -1, -1):
        W, b = layers[i]
        h_in = acts[i]
        grads[i] = (h_in.T @ dz, dz.sum(axis=0))
        if i > 0:
            dz = (dz @ W.T) * (acts[i] > 0.0)
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1].ravel()]) for g in grads])
    return loss, flat


# ---------------------------------------------------------------------------
# The paper's directional estimator (Sec. 4.1, Eq. 9-10), FP64
# ---------------------------------------------------------------------------

def l_out(r_e, r, s, chi_o):
    """Outside length of the segment [o, p_e] along one ray (Eq. 9 generalised to
    a segment that may end inside the solid): crossings at r with signs s (+1
    leaving the solid)."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    chi_e = chi_o - s.sum()
    return r_e - (s * r).sum() - chi_e * r_e


def directional_outer_volume(V, F, box, m=32):
    """Cube-map estimate of the outer volume of one box (c, axis0, axis1, half):
    per texel dOmega / 3 (r_e^3 - sum s_i r_i^3 - chi_e r_e^3), FP64."""
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    b = np.asarray(box, dtype=np.float64).reshape(12)
    o = b[:3]
    R = np.stack([b[3:6], b[6:9], np.cross(b[3:6], b[6:9])])
    half = b[9:12]
    A, B, Cc = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1, e2 = B - A, Cc - A
    nrm = np.cross(e1, e2)

    def hits(d):
        p = np.cross(d, e2)
        det = (e1 * p).sum(-1)
        ok = np.abs(det) > 1e-300
        inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
        s_ = o - A
        u = (s_ * p).sum(-1) * inv
        q = np.cross(s_, e1)
        v = (q @ d) * inv
        t = (e2 * q).sum(-1) * inv
        hit = ok & (u >= 0) & (u <= 1) & (v >= 0) & (u + v <= 1) & (t > 0)
        sign = np.where((nrm @ d) > 0, 1.0, -1.0)
        return t[hit], sign[hit]

    _, s0 = hits(np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0))
    chi_o = float(np.rint(s0.sum()))
    edges = -1.0 + 2.0 * np.arange(m + 1) / m

    def F_(u, v):
        return np.arctan2(u * v, np.sqrt(u * u + v * v + 1.0))

    total = 0.0
    for face in range(6):
        axis, sg = face // 2, (-1.0 if face % 2 else 1.0)
        for iv in range(m):
            for iu in range(m):
                u0, u1, v0, v1 = edges[iu], edges[iu + 1], edges[iv], edges[iv + 1]
                w = np.zeros(3)
                w[axis] = sg
                w[(axis + 1) % 3] = 0.5 * (u0 + u1)
                w[(axis + 2) % 3] = 0.5 * (v0 + v1)
                d = w / np.linalg.norm(w)
                c = np.abs(R @ d)
                re = np.min(np.where(c > 0, half / np.where(c > 0, c, 1.0), np.inf))
                t, s = hits(d)
                sel = t < re
                dom = F_(u1, v1) - F_(u0, v1) - F_(u1, v0) + F_(u0, v0)
                chi_e = chi_o - s[sel].sum()
                total += dom / 3.0 * (re ** 3 - (s[sel] * t[sel] ** 3).sum() - chi_e * re ** 3)
    return total
