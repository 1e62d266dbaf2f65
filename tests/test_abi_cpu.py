"""CPU-side checks of the C-ABI library: it builds, loads and exports every
entry point declared in include/obbvar.h (no compute call without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "obbvar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(obb_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    import paper_2203_10521_gb300 as P
    from paper_2203_10521_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(P.exported_symbols()) == set(names)


def test_struct_layouts_match_header():
    import paper_2203_10521_gb300 as P
    assert P.BOX_DTYPE.itemsize == 48
    assert P.QBOX_DTYPE.itemsize == 88 and P.QBOX_DTYPE.fields["b"][1] == 40
    assert ctypes.sizeof(P.StepStats) == 56
    assert ctypes.sizeof(P.TreeOpts) == 16
    assert ctypes.sizeof(P.ProfileStats) == 56
    assert ctypes.sizeof(P.SweepOpts) == 16
    assert ctypes.sizeof(P.SweepStats) == 40
    assert ctypes.sizeof(P.FloodStats) == 16
    assert ctypes.sizeof(P.AdjustStats) == 32


def test_no_gpu_means_no_context():
    """Without a device the library refuses to create a context (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2203_10521_gb300 as P
    with pytest.raises(P.ObbError):
        P.Context(0, stream=0)


def test_product_never_imports_oracle():
    """The CUDA package and its binding do not reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2203_10521_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "obb_oracle" not in text and "orc_" not in text, f


def _prototypes():
    """(return type, name, [parameter types]) of every function the header declares."""
    src = open(os.path.join(ROOT, "include", "obbvar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"^\s*#[^\n]*", "", src, flags=re.M)
    out = []
    for ret, name, params in re.findall(r"([A-Za-z_][\w\s\*]*?)\b(obb_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src):
        ps = [] if params.strip() in ("", "void") else [" ".join(p.split()) for p in params.split(",")]
        out.append((" ".join(ret.split()), name, ps))
    return out


def _ctype_of(decl):
    """The ctypes class a C parameter or return declaration marshals as ('ptr' for any pointer)."""
    if "*" in decl or "[" in decl:
        return "ptr"
    base = decl.replace("const ", "").split()[0]
    return {"obb_status": ctypes.c_int32, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
            "uint64_t": ctypes.c_uint64, "float": ctypes.c_float, "double": ctypes.c_double,
            "void": None}[base]


def _same(expected, actual):
    if expected == "ptr":
        return actual is ctypes.c_void_p or actual is ctypes.c_char_p or (
            isinstance(actual, type) and issubclass(actual, ctypes._Pointer))
    return actual is expected


def test_binding_signatures_match_header():
    """Every ctypes signature in the binding has the header's arity, integer widths and return type, so
    no argument is marshalled at the wrong width."""
    import paper_2203_10521_gb300 as P
    L = P.load()
    protos = _prototypes()
    assert sorted(n for _, n, _ in protos) == sorted(P.exported_symbols())
    for ret, name, params in protos:
        f = getattr(L, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == len(params), (name, params, f.argtypes)
        for p, a in zip(params, f.argtypes):
            assert _same(_ctype_of(p), a), (name, p, a)
        assert _same(_ctype_of(ret), f.restype), (name, ret, f.restype)


def test_struct_offsets_and_status_codes_match_compiled_header(tmp_path):
    """A C program compiled against the header prints sizeof and every field offset of the public structs
    and the status codes; the binding's ctypes structures and numpy dtypes must agree field by field (a
    field the binding names that the header lacks fails the compile)."""
    import shutil
    import subprocess
    import paper_2203_10521_gb300 as P
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    ctypes_structs = {"obb_step_opts": P.StepOpts, "obb_step_stats": P.StepStats,
                      "obb_profile_stats": P.ProfileStats, "obb_tree_opts": P.TreeOpts,
                      "obb_flood_stats": P.FloodStats, "obb_adjust_stats": P.AdjustStats,
                      "obb_sweep_opts": P.SweepOpts, "obb_sweep_stats": P.SweepStats}
    dtypes = {"obb_box": P.BOX_DTYPE, "obb_qbox": P.QBOX_DTYPE}
    expect, lines = {}, []
    for cname, S in ctypes_structs.items():
        expect[f"{cname} size"] = ctypes.sizeof(S)
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in S._fields_:
            expect[f"{cname} {f}"] = getattr(S, f).offset
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    for cname, dt in dtypes.items():
        expect[f"{cname} size"] = dt.itemsize
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in dt.names:
            expect[f"{cname} {f}"] = dt.fields[f][1]
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    for code, name in list(P._ERRORS.items()) + [(P.OBB_OK, "OBB_OK")]:
        expect[f"{name} value"] = code
        lines.append(f'printf("{name} value %d\\n", (int){name});')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "obbvar.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        key, val = line.rsplit(" ", 1)
        got[key] = int(val)
    assert got == expect


def test_output_checks_refuse_unusable_arrays():
    """The binding's check of caller-provided outputs (no device needed for
    host arrays): K 8-byte integers, contiguous and writeable, else ValueError."""
    import types
    import paper_2203_10521_gb300 as P
    fake = types.SimpleNamespace(device=0)
    P.Context._check_out(fake, "counts", np.zeros(5, np.uint64), 5, 0)
    P.Context._check_out(fake, "counts", np.zeros(7, np.int64), 5, 0)
    ro = np.zeros(5, np.uint64)
    ro.flags.writeable = False
    for bad in (np.zeros(4, np.uint64), np.zeros(5, np.int32), np.zeros(10, np.uint64)[::2], ro, [0] * 5):
        with pytest.raises(ValueError):
            P.Context._check_out(fake, "counts", bad, 5, 0)
    with pytest.raises(ValueError):
        P.Context._check_out(fake, "counts", np.zeros(5, np.uint64), 5, 1)   # host array for device boxes


def test_input_checks_host_arrays():
    """The binding's check of inputs before any call reads them (host arrays
    and CPU tensors; no device needed): lengths the call reads, one placement
    for all of a call's arrays, whole rows, records from raw bytes."""
    import paper_2203_10521_gb300 as P
    torch = pytest.importorskip("torch")
    p, dev, keep, n = P._input("assign", np.arange(7, dtype=np.int64), np.int32, 0, n=7)
    assert dev == 0 and n == 7 and keep.dtype == np.int32 and np.array_equal(keep, np.arange(7))
    _, _, keep, n = P._input("frames", np.zeros((3, 9)), np.float64, 0, n=27, dev=0)
    assert n == 27
    _, dev, keep, n = P._input("assign", torch.arange(5, dtype=torch.int32), np.int32, 0, n=5)
    assert dev == 0 and n == 5
    with pytest.raises(ValueError, match="reads 8"):
        P._input("assign", np.zeros(7, np.int32), np.int32, 0, n=8)
    with pytest.raises(ValueError, match="a CUDA tensor"):
        P._input("parent", np.zeros(4, np.int32), np.int32, 0, dev=1)
    with pytest.raises(ValueError, match="whole rows of 524"):
        P._input("feats", np.zeros((2, 100), np.float32), np.float32, 0, row=524)
    _, _, _, n = P._input("feats", np.zeros((3, 524), np.float32), np.float32, 0, row=524)
    assert n == 3 * 524


def test_record_inputs_from_bytes_and_rows():
    """Boxes as [K, 12] numbers, quantised boxes as raw bytes: both become
    whole records, never a field-by-field conversion."""
    import paper_2203_10521_gb300 as P
    q = np.zeros(3, P.QBOX_DTYPE)
    q["b"] = np.arange(18).reshape(3, 6)
    q["n"][:, 0] = [5, 6, 7]
    _, _, keep, n = P._input("qboxes", q.view(np.uint8), P.QBOX_DTYPE, 0)
    assert n == 3 and np.array_equal(keep["b"], q["b"]) and np.array_equal(keep["n"], q["n"])
    with pytest.raises(ValueError, match="whole 88-byte records"):
        P._input("qboxes", np.zeros(100, np.uint8), P.QBOX_DTYPE, 0)
    rows = np.arange(24, dtype=np.float64).reshape(2, 12)
    _, _, keep, n = P._input("boxes", rows, P.BOX_DTYPE, 0)
    assert n == 2 and keep["half"][1].tolist() == [21.0, 22.0, 23.0]
    with pytest.raises(ValueError, match="12 numbers"):
        P._input("boxes", np.zeros(13, np.float32), P.BOX_DTYPE, 0)


def test_output_checks_host_arrays():
    """Caller-supplied outputs: room for the elements, the element size of
    plain types, contiguous and writeable, on the inputs' side."""
    import paper_2203_10521_gb300 as P
    P._output("out", np.zeros(4, P.QBOX_DTYPE), 4, P.QBOX_DTYPE, 0, 0)
    P._output("out", np.zeros(4 * 88, np.uint8), 4, P.QBOX_DTYPE, 0, 0)   # records: any element type
    P._output("out", np.zeros((2, 524), np.float32), 2 * 524, np.float32, 0, 0)
    ro = np.zeros(4, P.QBOX_DTYPE)
    ro.flags.writeable = False
    for bad, n, dt in ((np.zeros(3, P.QBOX_DTYPE), 4, P.QBOX_DTYPE), (ro, 4, P.QBOX_DTYPE),
                       (np.zeros((2, 524), np.float64), 2 * 524, np.float32),
                       (np.zeros((2, 600), np.float32)[:, :524], 2 * 524, np.float32)):
        with pytest.raises(ValueError):
            P._output("out", bad, n, dt, 0, 0)
    with pytest.raises(ValueError, match="CUDA tensor"):
        P._output("out", np.zeros(4, P.QBOX_DTYPE), 4, P.QBOX_DTYPE, 1, 0)
