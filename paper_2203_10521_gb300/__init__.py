"""Python binding of libobbvar (include/obbvar.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module converts
numpy arrays / torch CUDA tensors to pointers, calls the C ABI and raises on
error.  There is no CPU fallback: importing works without a GPU, but creating
a Context needs the built library and a CUDA device.

Host arrays (numpy) are passed with on_device=0; torch CUDA tensors with
on_device=1 (they must be contiguous and on the context's device).  The
context enqueues on torch's current CUDA stream unless told otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

OBB_OK = 0
_ERRORS = {-1: "OBB_ERR_ARG", -2: "OBB_ERR_NOT_WATERTIGHT", -3: "OBB_ERR_RANGE", -4: "OBB_ERR_EMPTY_CLUSTER",
           -5: "OBB_ERR_CUDA", -6: "OBB_ERR_TIMEOUT", -7: "OBB_ERR_OOM", -8: "OBB_ERR_STATE"}

BOX_DTYPE = np.dtype([("c", "<f4", (3,)), ("axis0", "<f4", (3,)), ("axis1", "<f4", (3,)), ("half", "<f4", (3,))])
QBOX_DTYPE = np.dtype([("n", "<i4", (9,)), ("reserved", "<i4"), ("b", "<i8", (6,))])
assert BOX_DTYPE.itemsize == 48 and QBOX_DTYPE.itemsize == 88


class ObbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class StepOpts(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("refit", C.c_int32), ("descent_steps", C.c_int32),
                ("graph", C.c_int32)]


class StepStats(C.Structure):
    _fields_ = [("rounds_run", C.c_int32), ("refits_accepted", C.c_int32), ("proposals", C.c_int64),
                ("moves", C.c_int64), ("gain", C.c_int64), ("box_evals", C.c_int64),
                ("points_counted", C.c_uint64), ("total_obv", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ProfileStats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("count_launches", C.c_int64), ("count_ms", C.c_double),
                ("count_bytes", C.c_double), ("count_rows", C.c_double),
                ("count_points_in_domain", C.c_double), ("count_rows_rank", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TreeOpts(C.Structure):
    _fields_ = [("depth", C.c_int32), ("iters", C.c_int32), ("rounds", C.c_int32), ("refit", C.c_int32)]


class FloodStats(C.Structure):
    _fields_ = [("waves", C.c_int32), ("reserved", C.c_int32), ("box_evals", C.c_int64)]


class AdjustStats(C.Structure):
    _fields_ = [("kept", C.c_int32), ("k", C.c_int32), ("m", C.c_int32), ("j", C.c_int32),
                ("total_before", C.c_uint64), ("total_after", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SweepOpts(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("iters", C.c_int32), ("rounds", C.c_int32), ("refit", C.c_int32)]


class SweepStats(C.Structure):
    _fields_ = [("eq7_before", C.c_double), ("eq7_after", C.c_double), ("unit_moves", C.c_int64),
                ("triangle_moves", C.c_int64), ("level_iters", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None


def load(build_if_missing: bool = True):
    """Load libobbvar.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libobbvar.so is not built ({LIB_PATH}); run paper_2203_10521_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "obb_create": [C.POINTER(vp), i32, vp],
        "obb_set_stream": [vp, vp],
        "obb_synchronize": [vp],
        "obb_mesh_create": [vp, vp, i64, vp, i64, C.POINTER(vp)],
        "obb_build_occupancy": [vp, vp, i32, C.POINTER(vp)],
        "obb_occupancy_rebuild": [vp, vp],
        "obb_profile_enable": [vp, i32],
        "obb_profile_read": [vp, C.POINTER(ProfileStats)],
        "obb_lattice_desc": [vp, vp, vp, vp, vp, vp, vp],
        "obb_quantize_boxes": [vp, vp, vp, i64, vp, i32],
        "obb_outer_volume_q": [vp, vp, vp, i64, vp, vp, i32],
        "obb_outer_volume": [vp, vp, vp, i64, vp, vp, i32],
        "obb_outer_volume_q_noalloc": [vp, vp, vp, i64, vp, vp],
        "obb_outer_volume_multi": [vp, vp, i32, vp, vp, i64, vp, vp, i32],
        "obb_directional_outer_volume": [vp, vp, vp, i64, i32, vp, i32],
        "obb_layer_init": [vp, vp, vp, vp, i32, vp, i32, C.POINTER(vp)],
        "obb_lloyd_step": [vp, vp, C.POINTER(StepOpts), C.POINTER(StepStats)],
        "obb_layer_read": [vp, vp, vp, vp, vp, vp, vp, i32],
        "obb_layer_split": [vp, vp, vp, i32],
        "obb_build_tree": [vp, vp, C.POINTER(TreeOpts), C.POINTER(vp)],
        "obb_tree_read": [vp, vp, i32, vp, vp, vp, vp, vp],
        "obb_tree_score": [vp, vp, vp, vp],
        "obb_tree_parents": [vp, vp, i32, vp],
        "obb_tree_sweep": [vp, vp, C.POINTER(SweepOpts), C.POINTER(SweepStats)],
        "obb_layer_parents": [vp, vp, vp],
        "obb_flood_partition": [vp, vp, vp, i32, C.POINTER(FloodStats)],
        "obb_layer_adjust": [vp, vp, C.POINTER(StepOpts), i32, C.POINTER(AdjustStats)],
        "obb_set_counting_tile": [vp, i32],
        "obb_set_counting_axis": [vp, i32],
        "obb_set_counting_rank": [vp, i32],
        "obb_set_counting_order": [vp, i32],
        "obb_test_inject": [vp, i32],
        "obb_tune_counting": [vp, vp, vp, i64, i32, vp, vp],
        "obb_unit_step": [vp, vp, vp, C.POINTER(StepOpts), C.POINTER(StepStats)],
        "obb_mlp_create": [vp, C.c_uint64, C.POINTER(vp)],
        "obb_mlp_params": [vp, vp, vp, i32],
        "obb_mlp_set_params": [vp, vp, vp, i32],
        "obb_surrogate_features": [vp, vp, vp, i64, vp, i32],
        "obb_surrogate_targets": [vp, vp, vp, i64, vp, i32],
        "obb_mlp_forward": [vp, vp, vp, i64, vp, i32, i32],
        "obb_mlp_gradients": [vp, vp, vp, vp, i64, vp, vp, i32],
        "obb_mlp_train_step": [vp, vp, vp, vp, i64, C.c_float, vp, i32],
        "obb_layer_set_surrogate": [vp, vp, vp, i32],
        "obb_layer_last_candidates": [vp, vp, vp, vp, i64, C.POINTER(i64)],
        "obb_layer_moments": [vp, vp, i32, vp],
        "obb_layer_members": [vp, vp, vp, vp],
        "obb_batch_create": [vp, vp, i32, C.POINTER(vp)],
        "obb_batch_lloyd_step": [vp, vp, C.POINTER(StepOpts), vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int32
    L.obb_mlp_num_params.argtypes = []
    L.obb_mlp_num_params.restype = C.c_int64
    for name in ("obb_destroy", "obb_mesh_free", "obb_lattice_free", "obb_layer_free", "obb_tree_free",
                 "obb_mlp_free", "obb_batch_free"):
        getattr(L, name).argtypes = [vp]
        getattr(L, name).restype = None
    L.obb_last_error.argtypes = [vp]
    L.obb_last_error.restype = C.c_char_p
    L.obb_layer_clusters.argtypes = [vp]
    L.obb_layer_clusters.restype = C.c_int32
    L.obb_tree_depth.argtypes = [vp]
    L.obb_tree_depth.restype = C.c_int32
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points declared in include/obbvar.h."""
    return ["obb_create", "obb_set_stream", "obb_synchronize", "obb_destroy", "obb_last_error",
            "obb_profile_enable", "obb_profile_read", "obb_occupancy_rebuild",
            "obb_mesh_create", "obb_mesh_free", "obb_build_occupancy", "obb_lattice_desc", "obb_lattice_free",
            "obb_quantize_boxes", "obb_outer_volume_q", "obb_outer_volume", "obb_outer_volume_q_noalloc",
            "obb_outer_volume_multi", "obb_directional_outer_volume", "obb_layer_init", "obb_lloyd_step",
            "obb_layer_read", "obb_layer_clusters", "obb_layer_split", "obb_layer_free", "obb_build_tree",
            "obb_tree_read", "obb_tree_depth", "obb_tree_score", "obb_tree_free", "obb_tree_parents",
            "obb_tree_sweep", "obb_layer_parents", "obb_unit_step", "obb_flood_partition",
            "obb_layer_adjust", "obb_set_counting_tile", "obb_set_counting_axis", "obb_set_counting_rank",
            "obb_set_counting_order", "obb_test_inject",
            "obb_tune_counting",
            "obb_mlp_create", "obb_mlp_free", "obb_mlp_num_params", "obb_mlp_params", "obb_mlp_set_params",
            "obb_surrogate_features", "obb_surrogate_targets", "obb_mlp_forward", "obb_mlp_gradients",
            "obb_mlp_train_step",
            "obb_layer_set_surrogate", "obb_layer_last_candidates", "obb_layer_moments", "obb_layer_members",
            "obb_batch_create", "obb_batch_lloyd_step", "obb_batch_free"]


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _host(x, dtype):
    """Contiguous numpy copy/view of x with the given dtype.  Boxes may come
    as [K, 12] numbers (converted to float32); records of any other form are
    taken as their raw bytes (e.g. quantised boxes as uint8), never converted
    field by field."""
    a = np.asarray(x)
    dtype = np.dtype(dtype)
    if dtype.fields is not None and a.dtype != dtype:
        if dtype == BOX_DTYPE and a.dtype != np.uint8:
            a = np.ascontiguousarray(a, dtype=np.float32)
            if a.size % 12:
                raise ValueError("boxes must be records or rows of 12 numbers")
            return a.reshape(-1, 12).view(BOX_DTYPE).reshape(-1)
        b = np.ascontiguousarray(a).reshape(-1).view(np.uint8)
        if b.size % dtype.itemsize:
            raise ValueError(f"{b.size} bytes do not make whole {dtype.itemsize}-byte records")
        return b.view(dtype)
    if a.dtype != dtype:
        a = a.astype(dtype)
    return np.ascontiguousarray(a)


# the torch element types a plain input of each numpy type may have on the device
_TORCH_TYPES = {np.dtype(np.int32): ("int32",), np.dtype(np.float32): ("float32",),
                np.dtype(np.float64): ("float64",), np.dtype(np.uint64): ("int64", "uint64"),
                np.dtype(np.int64): ("int64", "uint64")}


def _input(name, x, dtype, device, n=None, dev=None, row=1):
    """(pointer, on_device, keepalive, count) of an input array.  A torch CUDA
    tensor must be contiguous and on `device`; for a record type (boxes) any
    element type whose bytes make whole records, else the element type the
    C call reads.  Anything else goes through numpy as a contiguous copy of
    `dtype`.  count = elements of `dtype`; n: the count the call reads; dev:
    the placement of the call's other arrays (0 host, 1 device); row: count
    must be a multiple of it (rows of a matrix)."""
    dtype = np.dtype(dtype)
    if _is_torch(x) and x.is_cuda:
        if x.device.index != device:
            raise ValueError(f"{name} is on {x.device}; this context is on cuda:{device}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if dtype.fields is None and str(x.dtype).replace("torch.", "") not in _TORCH_TYPES.get(dtype, ()):
            raise ValueError(f"{name} must be a {' or '.join(_TORCH_TYPES.get(dtype, ('?',)))} tensor")
        nbytes = x.numel() * x.element_size()
        if nbytes % dtype.itemsize:
            raise ValueError(f"{name} must hold whole {dtype.itemsize}-byte elements")
        p, on, keep, count = C.c_void_p(x.data_ptr()), 1, x, nbytes // dtype.itemsize
    else:
        if _is_torch(x):
            x = x.numpy()
        a = _host(x, dtype)
        p, on, keep, count = a.ctypes.data_as(C.c_void_p), 0, a, a.nbytes // dtype.itemsize
    if dev is not None and on != dev:
        raise ValueError(f"{name} must be {'a CUDA tensor' if dev else 'a host array'}, like the call's other arrays")
    if n is not None and count != n:
        raise ValueError(f"{name} holds {count} elements; the call reads {n}")
    if count % row:
        raise ValueError(f"{name} must hold whole rows of {row} elements")
    return p, on, keep, count


def _output(name, a, n, dtype, dev, device):
    """Pointer to a caller-supplied output of n elements of dtype on the
    inputs' side: a contiguous CUDA tensor of `device` with room for them
    (records: any element type; plain types: elements of the same size), or
    a writeable contiguous numpy array with room for them."""
    dtype = np.dtype(dtype)
    need = n * dtype.itemsize
    if dev:
        ok = (_is_torch(a) and a.is_cuda and a.device.index == device and a.is_contiguous()
              and a.numel() * a.element_size() >= need
              and (dtype.fields is not None or a.element_size() == dtype.itemsize))
        where = f"a contiguous CUDA tensor on cuda:{device}"
    else:
        ok = (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.flags.writeable and a.nbytes >= need
              and (dtype.fields is not None or a.itemsize == dtype.itemsize))
        where = "a writeable contiguous numpy array"
    if not ok:
        raise ValueError(f"{name} must be {where} with room for {n} elements of {dtype.itemsize} bytes")
    return C.c_void_p(a.data_ptr()) if dev else a.ctypes.data_as(C.c_void_p)


class _DevArray:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Context:
    """A library context bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        h = C.c_void_p()
        rc = self.lib.obb_create(C.byref(h), int(device), C.c_void_p(stream))
        if rc != OBB_OK:
            raise ObbError(rc, "cannot create a context (no CUDA device?)")
        self.h = h
        self.device = device

    def check(self, rc):
        if rc != OBB_OK:
            raise ObbError(rc, self.lib.obb_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.obb_destroy(self.h)
            self.h = None

    def set_stream(self, stream):
        self.check(self.lib.obb_set_stream(self.h, C.c_void_p(stream)))

    def synchronize(self):
        self.check(self.lib.obb_synchronize(self.h))

    # ------------------------------------------------------------------ mesh
    def mesh_create(self, verts, tris):
        V = np.ascontiguousarray(verts, dtype=np.float32)
        F = np.ascontiguousarray(tris, dtype=np.int32)
        h = C.c_void_p()
        self.check(self.lib.obb_mesh_create(self.h, V.ctypes.data_as(C.c_void_p), V.shape[0],
                                            F.ctypes.data_as(C.c_void_p), F.shape[0], C.byref(h)))
        return Mesh(self, h, V.shape[0], F.shape[0])

    # ------------------------------------------------------------- occupancy
    def build_occupancy(self, mesh, N: int):
        h = C.c_void_p()
        self.check(self.lib.obb_build_occupancy(self.h, mesh.h, int(N), C.byref(h)))
        return Lattice(self, h, mesh)

    def occupancy_rebuild(self, lat):
        self.check(self.lib.obb_occupancy_rebuild(self.h, lat.h))

    # ------------------------------------------------------- instrumentation
    def profile_enable(self, on=True):
        """True/1: time every counting launch and add up its algorithmic bytes
        and rows; 2: time only (the kernel without its counters); False/0: off."""
        self.check(self.lib.obb_profile_enable(self.h, int(on)))

    def profile_read(self):
        st = ProfileStats()
        self.check(self.lib.obb_profile_read(self.h, C.byref(st)))
        return st.as_dict()

    # ---------------------------------------------------------- outer volume
    def quantize_boxes(self, lat, boxes, out=None):
        p, dev, keep, K = _input("boxes", boxes, BOX_DTYPE, self.device)
        if out is None:
            out = self._out_like(dev, K, QBOX_DTYPE, 88)
        po = _output("out", out, K, QBOX_DTYPE, dev, self.device)
        self.check(self.lib.obb_quantize_boxes(self.h, lat.h, p, K, po, dev))
        return out

    def outer_volume(self, lat, boxes, counts=None, points=None, want_points=False):
        p, dev, keep, K = _input("boxes", boxes, BOX_DTYPE, self.device)
        return self._ov(self.lib.obb_outer_volume, lat, p, dev, K, counts, points, want_points)

    def outer_volume_q(self, lat, qboxes, counts=None, points=None, want_points=False):
        p, dev, keep, K = _input("qboxes", qboxes, QBOX_DTYPE, self.device)
        return self._ov(self.lib.obb_outer_volume_q, lat, p, dev, K, counts, points, want_points)

    def set_counting_tile(self, tile_k):
        self.check(self.lib.obb_set_counting_tile(self.h, int(tile_k)))

    def test_inject(self, flags):
        """Arm a one-shot test hook (OBB_INJECT_TC_STALL = 1: the next tensor-core
        network launch times out on purpose, bounded, and reports it)."""
        self.check(self.lib.obb_test_inject(self.h, int(flags)))

    def set_counting_axis(self, axis):
        """Row axis of the counting kernel: 0 (default) x rows; -1 picks per box
        the axis with the smallest shadow; 1, 2 force y, z rows (lattices built
        or rebuilt afterwards keep the y- and z-row copies these need)."""
        self.check(self.lib.obb_set_counting_axis(self.h, int(axis)))

    def set_counting_rank(self, on):
        """1 (default): long rows counted from their end words and the rank
        table; 0: every word of every row interval read."""
        self.check(self.lib.obb_set_counting_rank(self.h, int(on)))

    def set_counting_order(self, on):
        """1 (default): batches of at least 1,024 boxes on lattices of at least
        64 MiB counted in spatial order; 0: in the caller's order."""
        self.check(self.lib.obb_set_counting_order(self.h, int(on)))

    def tune_counting(self, lat, qboxes):
        """Time the count of these quantised boxes with 8/16/32/64 rows per tile and
        keep the fastest; returns (tile_k, {tile_k: ms})."""
        q = _host(qboxes, QBOX_DTYPE)
        tk = C.c_int32()
        ms = (C.c_float * 4)()
        self.check(self.lib.obb_tune_counting(self.h, lat.h, q.ctypes.data_as(C.c_void_p), len(q), 0,
                                              C.byref(tk), ms))
        return tk.value, dict(zip((8, 16, 32, 64), list(ms)))

    def directional_outer_volume(self, mesh, boxes, m=32):
        """The paper's cube-map ray estimator of the outer volume (world units^3), host arrays."""
        b = _host(boxes, BOX_DTYPE)
        out = np.zeros(len(b), np.float64)
        self.check(self.lib.obb_directional_outer_volume(self.h, mesh.h, b.ctypes.data_as(C.c_void_p), len(b), int(m),
                                                         out.ctypes.data_as(C.c_void_p), 0))
        return out

    def outer_volume_multi(self, lats, qboxes, lattice_of_box, want_points=False):
        """Counts of quantised boxes on several lattices in one launch (host arrays)."""
        q = _host(qboxes, QBOX_DTYPE)
        K = len(q)
        _, _, li, _ = _input("lattice_of_box", lattice_of_box, np.int32, self.device, n=K, dev=0)
        table = (C.c_void_p * len(lats))(*[l.h.value for l in lats])
        cnt = np.zeros(K, np.uint64)
        pts = np.zeros(K, np.uint64) if want_points else None
        self.check(self.lib.obb_outer_volume_multi(self.h, table, len(lats), q.ctypes.data_as(C.c_void_p),
                                                   li.ctypes.data_as(C.c_void_p), K, cnt.ctypes.data_as(C.c_void_p),
                                                   pts.ctypes.data_as(C.c_void_p) if want_points else None, 0))
        return (cnt, pts) if want_points else cnt

    def outer_volume_q_noalloc(self, lat, qboxes, counts, points=None):
        """Device-only variant that allocates nothing (see obbvar.h); qboxes
        (88-byte records), counts and points (8-byte elements) are contiguous
        torch CUDA tensors on this context's device that the caller owns."""
        import torch
        dev = torch.device(f"cuda:{self.device}")

        def check(t, name, itemsize):
            if not (_is_torch(t) and t.is_cuda and t.device == dev):
                raise ValueError(f"{name} must be a CUDA tensor on {dev}")
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
            if itemsize and t.element_size() != itemsize:
                raise ValueError(f"{name} must have {itemsize}-byte elements")

        check(qboxes, "qboxes", 0)
        nbytes = qboxes.numel() * qboxes.element_size()
        if nbytes % 88:
            raise ValueError("qboxes must hold whole 88-byte box records")
        K = nbytes // 88
        check(counts, "counts", 8)
        if counts.numel() < K:
            raise ValueError(f"counts holds {counts.numel()} values for {K} boxes")
        pp = None
        if points is not None:
            check(points, "points", 8)
            if points.numel() < K:
                raise ValueError(f"points holds {points.numel()} values for {K} boxes")
            pp = C.c_void_p(points.data_ptr())
        self.check(self.lib.obb_outer_volume_q_noalloc(self.h, lat.h, C.c_void_p(qboxes.data_ptr()), K,
                                                         C.c_void_p(counts.data_ptr()), pp))
        return counts

    def _out_like(self, dev, K, dtype, itemsize, torch_dtype=None):
        if dev:
            import torch
            if torch_dtype is not None:
                return torch.empty(K, dtype=torch_dtype, device=f"cuda:{self.device}")
            return torch.empty(K * itemsize, dtype=torch.uint8, device=f"cuda:{self.device}")
        return np.zeros(K, dtype=dtype)

    def _check_out(self, name, a, K, dev):
        """An output of K 8-byte integers on the inputs' side: a contiguous
        CUDA tensor of this context's device, or a writeable contiguous numpy
        array on the host."""
        if dev:
            ok = (_is_torch(a) and a.is_cuda and a.device.index == self.device and a.is_contiguous()
                  and a.element_size() == 8 and a.numel() >= K)
            want = f"a contiguous 8-byte CUDA tensor on cuda:{self.device} with at least {K} elements"
        else:
            ok = (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.flags.writeable and a.itemsize == 8
                  and a.size >= K)
            want = f"a writeable contiguous numpy array of 8-byte integers with at least {K} elements"
        if not ok:
            raise ValueError(f"{name} must be {want}")

    def _ov(self, fn, lat, p, dev, K, counts, points, want_points):
        import_torch = dev
        if counts is None:
            if import_torch:
                import torch
                counts = torch.empty(K, dtype=torch.int64, device=f"cuda:{self.device}")
            else:
                counts = np.zeros(K, dtype=np.uint64)
        if points is None and want_points:
            if import_torch:
                import torch
                points = torch.empty(K, dtype=torch.int64, device=f"cuda:{self.device}")
            else:
                points = np.zeros(K, dtype=np.uint64)
        for name, a in (("counts", counts), ("points", points)):
            if a is not None:
                self._check_out(name, a, K, dev)
        pc = C.c_void_p(counts.data_ptr()) if dev else counts.ctypes.data_as(C.c_void_p)
        pp = None
        if points is not None:
            pp = C.c_void_p(points.data_ptr()) if dev else points.ctypes.data_as(C.c_void_p)
        self.check(fn(self.h, lat.h, p, K, pc, pp, dev))
        return (counts, points) if want_points or points is not None else counts

    # ----------------------------------------------------------------- layer
    def layer_init(self, lat, assign, parent, frames=None):
        """assign int32 [n_tris] cluster of each triangle, parent int32 [K],
        frames float64 [K, 9] or None: all host arrays or all CUDA tensors."""
        pa, dev, ka, _ = _input("assign", assign, np.int32, self.device, n=lat.mesh.nt)
        pp, _, kp, K = _input("parent", parent, np.int32, self.device, dev=dev)
        pf, kf = None, None
        if frames is not None:
            pf, _, kf, _ = _input("frames", frames, np.float64, self.device, n=9 * K, dev=dev)
        h = C.c_void_p()
        self.check(self.lib.obb_layer_init(self.h, lat.h, pa, pp, int(K), pf, dev, C.byref(h)))
        return Layer(self, h, lat, K)

    def lloyd_step(self, layer, rounds=16, refit=True, stats=True, descent_steps=0, graph=False):
        """refit: False/0 none, True/1 covariance frame, 2 rotation descent, 3 both;
        graph: run the iteration as one CUDA graph (device-side round loop)."""
        o = StepOpts(int(rounds), int(refit), int(descent_steps), int(bool(graph)))
        st = StepStats()
        self.check(self.lib.obb_lloyd_step(self.h, layer.h, C.byref(o), C.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def unit_step(self, upper, lower, rounds=16, refit=True, stats=True, descent_steps=0):
        """One Lloyd iteration of `upper` with the clusters of `lower` as units
        (bottom-up merging, Sec. 4.2.2); refit as in lloyd_step."""
        o = StepOpts(int(rounds), int(refit), int(descent_steps), 0)
        st = StepStats()
        self.check(self.lib.obb_unit_step(self.h, upper.h, lower.h, C.byref(o), C.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def flood_partition(self, layer, centres=None, mode=0):
        """Re-partition the layer's triangles by flooding (Sec. 4.2.1 step 1):
        mode 0 the paper's priority order, 1 the wavefront approximation."""
        st = FloodStats()
        c = None
        if centres is not None:
            c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
            if len(c) != layer.K:
                raise ValueError("one centre per box")
        self.check(self.lib.obb_flood_partition(self.h, layer.h, c.ctypes.data_as(C.c_void_p) if c is not None else None,
                                                int(mode), C.byref(st)))
        return {"waves": st.waves, "box_evals": st.box_evals}

    def layer_adjust(self, layer, iters=2, rounds=16, refit=True, descent_steps=0):
        """Re-seat the least important box (Sec. 4.2.1 step 3); kept only if
        the layer's total outer volume drops after `iters` Lloyd iterations."""
        o = StepOpts(int(rounds), int(refit), int(descent_steps), 0)
        st = AdjustStats()
        self.check(self.lib.obb_layer_adjust(self.h, layer.h, C.byref(o), int(iters), C.byref(st)))
        return st.as_dict()

    def layer_parents(self, layer):
        p = np.zeros(layer.K, np.int32)
        self.check(self.lib.obb_layer_parents(self.h, layer.h, p.ctypes.data_as(C.c_void_p)))
        return p

    def layer_read(self, layer, out=None):
        """The layer's state as host arrays; `out` may supply them (e.g. in
        page-locked memory, which the copies reach faster): a dict with
        assign int32 [T], frames float64 [K, 9], qboxes, boxes, obv uint64 [K]."""
        T, K = layer.lat.mesh.nt, layer.K
        if out is not None:
            want = {"assign": ((T,), np.int32), "frames": ((K, 9), np.float64), "qboxes": ((K,), QBOX_DTYPE),
                    "boxes": ((K,), BOX_DTYPE), "obv": ((K,), np.uint64)}
            for k, (shape, dt) in want.items():
                a = out.get(k)
                if not (isinstance(a, np.ndarray) and a.shape == shape and a.dtype == dt and a.flags.c_contiguous
                        and a.flags.writeable):
                    raise ValueError(f"out[{k!r}] must be a writeable contiguous {np.dtype(dt)} array of shape {shape}")
            assign, frames, q, boxes, obv = (out[k] for k in want)
        else:
            assign = np.zeros(T, np.int32)
            frames = np.zeros((K, 9), np.float64)
            q = np.zeros(K, QBOX_DTYPE)
            boxes = np.zeros(K, BOX_DTYPE)
            obv = np.zeros(K, np.uint64)
        self.check(self.lib.obb_layer_read(self.h, layer.h, assign.ctypes.data_as(C.c_void_p),
                                           frames.ctypes.data_as(C.c_void_p), q.ctypes.data_as(C.c_void_p),
                                           boxes.ctypes.data_as(C.c_void_p), obv.ctypes.data_as(C.c_void_p), 0))
        return dict(assign=assign, frames=frames, qboxes=q, boxes=boxes, obv=obv)

    def batch_create(self, layers):
        """A batch of layers (of one or many meshes) stepped together."""
        arr = (C.c_void_p * len(layers))(*[l.h.value for l in layers])
        h = C.c_void_p()
        self.check(self.lib.obb_batch_create(self.h, arr, len(layers), C.byref(h)))
        return Batch(self, h, list(layers))

    def batch_lloyd_step(self, batch, rounds=16, refit=True, descent_steps=0):
        """One Lloyd iteration of every layer of the batch, each round's exact
        counts of all layers in one counting launch; returns a list of stats."""
        o = StepOpts(int(rounds), int(refit), int(descent_steps), 0)
        st = (StepStats * len(batch.layers))()
        self.check(self.lib.obb_batch_lloyd_step(self.h, batch.h, C.byref(o), st))
        return [x.as_dict() for x in st]

    def layer_moments(self, layer, compensated=True):
        """Cluster moments float64 [K, 10] as the refit sums them (compensated
        FP32) or in plain FP32 (compensated=False)."""
        out = np.zeros((layer.K, 10), np.float64)
        self.check(self.lib.obb_layer_moments(self.h, layer.h, 1 if compensated else 0,
                                              out.ctypes.data_as(C.c_void_p)))
        return out

    def layer_members(self, layer):
        """Member lists: (members int32 [n_tris], triangles sorted by cluster,
        ascending within a cluster; start int32 [K + 1])."""
        members = np.zeros(layer.lat.mesh.nt, np.int32)
        start = np.zeros(layer.K + 1, np.int32)
        self.check(self.lib.obb_layer_members(self.h, layer.h, members.ctypes.data_as(C.c_void_p),
                                              start.ctypes.data_as(C.c_void_p)))
        return members, start

    def layer_split(self, layer):
        child = np.zeros(layer.lat.mesh.nt, np.int32)
        self.check(self.lib.obb_layer_split(self.h, layer.h, child.ctypes.data_as(C.c_void_p), 0))
        return child

    # ------------------------------------------------------------- surrogate
    SURROGATE_INPUTS = 524

    def mlp_create(self, seed=0):
        h = C.c_void_p()
        self.check(self.lib.obb_mlp_create(self.h, C.c_uint64(seed), C.byref(h)))
        return Mlp(self, h)

    def mlp_num_params(self):
        return int(self.lib.obb_mlp_num_params())

    def mlp_params(self, mlp):
        out = np.zeros(self.mlp_num_params(), np.float32)
        self.check(self.lib.obb_mlp_params(self.h, mlp.h, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def mlp_set_params(self, mlp, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.mlp_num_params():
            raise ValueError(f"params holds {p.size} values; the network has {self.mlp_num_params()}")
        self.check(self.lib.obb_mlp_set_params(self.h, mlp.h, p.ctypes.data_as(C.c_void_p), 0))

    def surrogate_features(self, lat, qboxes, out=None):
        """[K, 524] float32 features (numpy in -> numpy out, CUDA tensors -> CUDA tensor)."""
        p, dev, keep, K = _input("qboxes", qboxes, QBOX_DTYPE, self.device)
        if out is None:
            if dev:
                import torch
                out = torch.empty((K, self.SURROGATE_INPUTS), dtype=torch.float32, device=f"cuda:{self.device}")
            else:
                out = np.zeros((K, self.SURROGATE_INPUTS), np.float32)
        po = _output("out", out, K * self.SURROGATE_INPUTS, np.float32, dev, self.device)
        self.check(self.lib.obb_surrogate_features(self.h, lat.h, p, K, po, dev))
        return out

    def surrogate_targets(self, qboxes, counts):
        """Training targets: exact outer volume / the box's cell volume (the
        screen's scale), clipped to [0, 1].  CUDA tensors in -> CUDA tensor out
        (qboxes as bytes, counts int64), numpy -> numpy."""
        p, dev, keep, K = _input("qboxes", qboxes, QBOX_DTYPE, self.device)
        pc, _, keepc, _ = _input("counts", counts, np.uint64, self.device, n=K, dev=dev)
        if dev:
            import torch
            out = torch.empty(K, dtype=torch.float32, device=f"cuda:{self.device}")
            po = C.c_void_p(out.data_ptr())
        else:
            out = np.zeros(K, np.float32)
            po = out.ctypes.data_as(C.c_void_p)
        self.check(self.lib.obb_surrogate_targets(self.h, p, pc, K, po, dev))
        return out

    def mlp_forward(self, mlp, feats, half=True):
        """Predicted empty fractions [B] of features [B, 524] (numpy or a CUDA tensor)."""
        p, dev, keep, n = _input("feats", feats, np.float32, self.device, row=self.SURROGATE_INPUTS)
        B = n // self.SURROGATE_INPUTS
        if dev:
            import torch
            out = torch.empty(B, dtype=torch.float32, device=f"cuda:{self.device}")
            po = C.c_void_p(out.data_ptr())
        else:
            out = np.zeros(B, np.float32)
            po = out.ctypes.data_as(C.c_void_p)
        self.check(self.lib.obb_mlp_forward(self.h, mlp.h, p, B, po, 1 if half else 0, dev))
        return out

    def mlp_gradients(self, mlp, feats, target):
        """Gradients of the mean squared error over a host batch: (grads, loss)."""
        px, _, kx, n = _input("feats", feats, np.float32, self.device, dev=0, row=self.SURROGATE_INPUTS)
        B = n // self.SURROGATE_INPUTS
        pt, _, kt, _ = _input("target", target, np.float32, self.device, n=B, dev=0)
        g = np.zeros(self.mlp_num_params(), np.float32)
        loss = np.zeros(1, np.float32)
        self.check(self.lib.obb_mlp_gradients(self.h, mlp.h, px, pt, B, g.ctypes.data_as(C.c_void_p),
                                              loss.ctypes.data_as(C.c_void_p), 0))
        return g, float(loss[0])

    def mlp_train_step(self, mlp, feats, target, lr, want_loss=False):
        """One Adam step; feats [B, 524] / target [B] are both CUDA tensors
        (device; no loss returned) or both host arrays."""
        px, dev, kx, n = _input("feats", feats, np.float32, self.device, row=self.SURROGATE_INPUTS)
        B = n // self.SURROGATE_INPUTS
        pt, _, kt, _ = _input("target", target, np.float32, self.device, n=B, dev=dev)
        if dev:
            self.check(self.lib.obb_mlp_train_step(self.h, mlp.h, px, pt, B, C.c_float(lr), None, 1))
            return None
        loss = np.zeros(1, np.float32)
        self.check(self.lib.obb_mlp_train_step(self.h, mlp.h, px, pt, B, C.c_float(lr),
                                               loss.ctypes.data_as(C.c_void_p), 0))
        return float(loss[0])

    def layer_set_surrogate(self, layer, mlp, topk):
        self.check(self.lib.obb_layer_set_surrogate(self.h, layer.h, mlp.h if mlp is not None else None, int(topk)))

    def layer_last_candidates(self, layer, cap=1 << 20):
        q = np.zeros(cap, QBOX_DTYPE)
        c = np.zeros(cap, np.uint64)
        n = C.c_int64()
        self.check(self.lib.obb_layer_last_candidates(self.h, layer.h, q.ctypes.data_as(C.c_void_p),
                                                      c.ctypes.data_as(C.c_void_p), cap, C.byref(n)))
        m = min(n.value, cap)
        return q[:m].copy(), c[:m].copy()

    # ------------------------------------------------------------------ tree
    def build_tree(self, lat, depth, iters, rounds=16, refit=True):
        o = TreeOpts(int(depth), int(iters), int(rounds), int(refit))
        h = C.c_void_p()
        self.check(self.lib.obb_build_tree(self.h, lat.h, C.byref(o), C.byref(h)))
        return Tree(self, h, lat)

    def tree_read(self, tree, level):
        T = tree.lat.mesh.nt
        K = 1 << level
        assign = np.zeros(T, np.int32)
        frames = np.zeros((K, 9), np.float64)
        q = np.zeros(K, QBOX_DTYPE)
        boxes = np.zeros(K, BOX_DTYPE)
        obv = np.zeros(K, np.uint64)
        self.check(self.lib.obb_tree_read(self.h, tree.h, int(level), assign.ctypes.data_as(C.c_void_p),
                                          frames.ctypes.data_as(C.c_void_p), q.ctypes.data_as(C.c_void_p),
                                          boxes.ctypes.data_as(C.c_void_p), obv.ctypes.data_as(C.c_void_p)))
        return dict(assign=assign, frames=frames, qboxes=q, boxes=boxes, obv=obv)

    def tree_parents(self, tree, level):
        p = np.zeros(1 << level, np.int32)
        self.check(self.lib.obb_tree_parents(self.h, tree.h, int(level), p.ctypes.data_as(C.c_void_p)))
        return p

    def tree_sweep(self, tree, sweeps=1, iters=2, rounds=16, refit=True):
        """Reciprocating bottom-up / top-down sweeps over the tree's levels (Sec. 4.2.2)."""
        o = SweepOpts(int(sweeps), int(iters), int(rounds), int(refit))
        st = SweepStats()
        self.check(self.lib.obb_tree_sweep(self.h, tree.h, C.byref(o), C.byref(st)))
        return st.as_dict()

    def tree_score(self, tree):
        p = C.c_double()
        v = C.c_double()
        self.check(self.lib.obb_tree_score(self.h, tree.h, C.byref(p), C.byref(v)))
        return p.value, v.value


class _Handle:
    _free = None

    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def free(self):
        if getattr(self, "h", None) and self.ctx.h:
            getattr(self.ctx.lib, self._free)(self.h)
            self.h = None


class Mesh(_Handle):
    _free = "obb_mesh_free"

    def __init__(self, ctx, h, nv, nt):
        super().__init__(ctx, h)
        self.nv, self.nt = nv, nt


class Lattice(_Handle):
    _free = "obb_lattice_free"

    def __init__(self, ctx, h, mesh):
        super().__init__(ctx, h)
        self.mesh = mesh
        lo = (C.c_double * 3)()
        hh = (C.c_double * 3)()
        N = C.c_int32()
        W = C.c_int64()
        words = C.c_void_p()
        fixed = C.c_void_p()
        ctx.check(ctx.lib.obb_lattice_desc(h, lo, hh, C.byref(N), C.byref(W), C.byref(words), C.byref(fixed)))
        self.lo = np.array(lo[:])
        self.h_ = np.array(hh[:])
        self.N = N.value
        self.W = W.value
        self._words = words.value
        self._fixed = fixed.value

    @property
    def spacing(self):
        return self.h_

    def words(self):
        """The occupancy words as a torch uint64-typed view (int64 tensor) of library memory."""
        import torch
        return torch.as_tensor(_DevArray(self._words, (self.N * self.N * self.W,), "<i8"),
                               device=f"cuda:{self.ctx.device}")

    def fixed(self):
        import torch
        return torch.as_tensor(_DevArray(self._fixed, (self.mesh.nv, 3), "<i4"), device=f"cuda:{self.ctx.device}")

    def bits(self):
        """Occupancy as a numpy uint8 array [k, j, i] (copies to the host)."""
        w = self.words().cpu().numpy().view(np.uint64).reshape(self.N, self.N, self.W)
        b = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
        return b[..., :self.N]


class Layer(_Handle):
    _free = "obb_layer_free"

    def __init__(self, ctx, h, lat, K):
        super().__init__(ctx, h)
        self.lat = lat
        self.K = K


class Mlp(_Handle):
    _free = "obb_mlp_free"


class Batch(_Handle):
    _free = "obb_batch_free"

    def __init__(self, ctx, h, layers):
        super().__init__(ctx, h)
        self.layers = layers


class Tree(_Handle):
    _free = "obb_tree_free"

    def __init__(self, ctx, h, lat):
        super().__init__(ctx, h)
        self.lat = lat
        self.depth = ctx.lib.obb_tree_depth(h)
