"""Build libobbvar.so (CUDA, sm_103a) in-tree with nvcc.

The translation units compile in parallel; the result goes to
paper_2203_10521_gb300/_build/libobbvar.so (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libobbvar.so")
UNITS = ["runtime.cu", "occupancy.cu", "outer_volume.cu", "lloyd.cu", "tree.cu", "surrogate.cu", "directional.cu", "sweep.cu", "flood.cu", "adjust.cu", "mesh.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(SRC, u) for u in UNITS]
    files += [os.path.join(SRC, "internal.h"), os.path.join(HERE, "..", "include", "obbvar.h")]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), out_dir: str = None) -> str:
    """Compile and link; `extra` adds nvcc flags (e.g. tuning -D values) and
    `out_dir` redirects the objects and the library (default: _build/)."""
    lib = LIB if out_dir is None else os.path.join(out_dir, "libobbvar.so")
    out = OUT if out_dir is None else out_dir
    if not force and out_dir is None and up_to_date():
        return LIB
    os.makedirs(out, exist_ok=True)
    cc = nvcc()

    def one(unit):
        obj = os.path.join(out, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(SRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
