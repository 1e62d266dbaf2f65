"""bench.py's reference arm (the oracle timed on the host) keeps the JSON
contract the benchmark driver reads; ranks other than 0 do no work."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--small", "--steps", "1",
                           "--warmup", "1", "--cpu-seconds", "1"], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=600)


def test_reference_arm_json_line():
    import bench
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_cpu_baseline_and_reference_time_the_same_work():
    """The GPU line's cpu_baseline and the reference arm count the same boxes
    (the oracle's own median-split leaves, in one seeded order) on a fresh
    oracle problem, in in-domain points per second, single thread and on all
    cores."""
    import bench
    import oracle as O
    wl = bench.workload("torus4k-64", 0)
    n1, b1, o1, _ = bench.oracle_setup(wl)
    n2, b2, o2, _ = bench.oracle_setup(wl)
    assert np.array_equal(n1, n2) and np.array_equal(b1, b2) and np.array_equal(o1, o2)
    assert len(n1) == 1 << wl["depth"]
    v, pts, nb, dt, used = bench.oracle_rate(wl["mesh"], wl["N"], n1, b1, o1[:3], 60.0, 1)
    P = O.Problem(wl["mesh"].verts, wl["mesh"].tris, wl["N"])
    _, _, dom = O.outer_volume(P.occ, n1[o1[:3]], b1[o1[:3]], want_domain=True)
    assert nb == 3 and pts == int(dom.sum()) and used == 1
    cb = bench.cpu_baseline(wl, 0.5)
    assert cb["cores"] >= 1 and cb["nproc"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["single_thread_value"] > 0


def test_roofline_inputs_match_the_counting_sources():
    """The committed ncu figures the benchmark reports (DRAM traffic and
    instruction count of the counting kernel's batch launch) were captured
    from the current counting sources: a change to the kernel, the occupancy
    pass that writes its lattice copies or their shared types needs a new
    capture."""
    import bench
    for wl in ("sdf2m-1024", "sdf200k-512"):
        ri = bench.roofline_inputs(wl)
        assert not ri.get("stale"), wl
        assert ri.get("dram_bytes_batch_launch", 0) > 0 and ri.get("warp_inst_batch_launch", 0) > 0, wl


def _profile_commands():
    """The shell commands quoted in profiles/ (code fences of the .md
    summaries, '#' lines of the .txt inputs), continuation lines joined."""
    cmds = []
    pdir = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        text = open(os.path.join(pdir, name)).read()
        if name.endswith(".md"):
            parts = text.split("```")
            lines = [ln for block in parts[1::2] for ln in block.splitlines()]
        else:
            lines = [ln.lstrip("#").strip() for ln in text.splitlines() if ln.startswith("#")]
        cur = ""
        for ln in lines:
            ln = ln.strip()
            cur = (cur + " " + ln[:-1]).strip() if ln.endswith("\\") else (cur + " " + ln).strip()
            if not ln.endswith("\\"):
                if cur.split(" ", 1)[0] in ("python", "ncu", "nvcc"):
                    cmds.append((name, cur))
                cur = ""
    return cmds


def test_profile_commands_run_the_committed_benchmark():
    """Every bench.py command a profile summary quotes is accepted by
    bench.py's own argument parser, and every ncu command leaves the clocks
    alone (--clock-control none)."""
    import shlex
    sys.path.insert(0, ROOT)
    import bench
    cmds = _profile_commands()
    n_bench = n_ncu = 0
    for name, cmd in cmds:
        toks = shlex.split(cmd)
        if toks and toks[0] == "ncu" and "-i" not in toks:   # a capture (-i only reads a saved report)
            n_ncu += 1
            i = toks.index("--clock-control")
            assert toks[i + 1] == "none", (name, cmd)
        for i, t in enumerate(toks):
            if t == "bench.py" and i > 0 and toks[i - 1] == "python":
                n_bench += 1
                old = sys.argv
                try:
                    sys.argv = ["bench.py"] + toks[i + 1:]
                    bench.parse()
                except SystemExit as e:
                    raise AssertionError(f"{name}: bench.py rejects {cmd!r}") from e
                finally:
                    sys.argv = old
    assert n_bench >= 8 and n_ncu >= 4, (n_bench, n_ncu)
