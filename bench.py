#!/usr/bin/env python
"""Benchmark of the outer-volume / Lloyd hot path on one GB300 per rank.

One step = one pass of the whole path over the workload's batch:
  occupancy rebuild of the lattice from the resident mesh (snap, column
  crossings, row scan with the rank tables), exact outer volume of every box
  of the tree (FP32 boxes: quantise + count; Eq. 4), and one Lloyd iteration
  on the leaf layer (partition rounds with exact gains + covariance / Jacobi
  refit, as the library's CUDA graph), whose layer total is the Eq. 7 leaf
  term.
value = in-domain lattice points counted by the outer-volume kernel (every
counting launch of the step, the Lloyd iteration's included) per second of
step time; whole job: summed over ranks, divided by the slowest rank.

Workloads (--workload):
  sdf2m-1024   (default) the seeded SDF union of 200 spheres + 100 capsules +
               50 rounded boxes, 2,029,088 watertight triangles (marching
               tetrahedra), 1024^3 lattice (128 MiB, larger than L2), binary
               tree of depth 14 (16,384 leaves), three reciprocating
               bottom-up / top-down sweeps after the top-down build;
  sdf200k-512  the union of 40 spheres + 20 capsules, 202,244 triangles,
               512^3 lattice, depth 10;
  torus4k-64   (--small) the 4,096-triangle torus on 64^3, depth 4.

--impl reference times the CPU oracle (the plain per-point restatement) on a
bounded sample of the same workload, the same way as the GPU line's
cpu_baseline.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "lattice pts/s in OBB outer-volume eval; Lloyd iter/s plain vs surrogate"
UNIT = "lattice pts/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sdf2m-1024", choices=sorted(WORKLOADS))
    ap.add_argument("--small", action="store_true", help="the 4,096-triangle torus on 64^3 (--workload torus4k-64)")
    ap.add_argument("--setup-iters", type=int, default=2, help="Lloyd iterations per level while building the tree")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="oracle time per thread count in cpu_baseline")
    ap.add_argument("--eager-step", action="store_true",
                    help="host-driven Lloyd rounds in the timed step (default: the step's CUDA graph)")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-topk", type=int, default=5,
                    help="candidates (and rotation probes) per cluster the surrogate keeps for exact counting")
    ap.add_argument("--lloyd-iters", type=int, default=10,
                    help="Lloyd iterations timed for the plain vs surrogate comparison")
    ap.add_argument("--surrogate-pairs", type=int, default=2_000_000,
                    help="training pairs generated on the 202,244-triangle union at 512^3")
    ap.add_argument("--surrogate-steps", type=int, default=2000, help="Adam steps of surrogate training")
    ap.add_argument("--batch-meshes", type=int, default=256, help="meshes of the batched Lloyd comparison (0: skip)")
    ap.add_argument("--batch-iters", type=int, default=3, help="Lloyd iterations timed in the batched comparison")
    ap.add_argument("--no-second-workload", action="store_true",
                    help="skip the plain vs surrogate comparison on the 1M-triangle union at 768^3")
    ap.add_argument("--walk", action="store_true", help="count every row word by word (no rank tables)")
    ap.add_argument("--profile-batch", metavar="BOXES",
                    help="profiling aid: count the tree batch twice and exit; the tree's boxes are read from "
                         "BOXES (.npy) when it exists, else built and written there")
    a = ap.parse_args()
    if a.small:
        a.workload = "torus4k-64"
    return a


def _torus(rank):
    from synth import meshes as M
    return M.torus(1.0, 0.3, 64, 32, jitter=0.002, seed=1000 + rank)


def _sdf200k(rank):
    from synth import meshes as M
    return M.sdf_union_200k(seed=2000 + rank)


def _sdf1m(rank):
    from synth import meshes as M
    return M.sdf_union_1m(seed=4000 + rank)


def _sdf2m(rank):
    from synth import meshes as M
    return M.sdf_union_2m(seed=5000 + rank)


WORKLOADS = {
    "sdf2m-1024": dict(desc="SDF union 200 spheres + 100 capsules + 50 rounded boxes, {T:,} triangles, 1024^3 "
                            "lattice, depth 14 (16,384 leaves), 3 up/down sweeps", mesh=_sdf2m, N=1024, depth=14,
                       sweeps=3),
    "sdf1m-768": dict(desc="SDF union 40 spheres + 20 capsules, {T:,} triangles, 768^3 lattice, depth 12 "
                           "(4,096 leaves)", mesh=_sdf1m, N=768, depth=12, sweeps=0),
    "sdf200k-512": dict(desc="SDF union 40 spheres + 20 capsules, {T:,} triangles, 512^3 lattice, depth 10 "
                             "(1,024 leaves)", mesh=_sdf200k, N=512, depth=10, sweeps=0),
    "torus4k-64": dict(desc="torus R=1 r=0.3, {T:,} triangles, 64^3 lattice, depth 4", mesh=_torus, N=64, depth=4,
                       sweeps=0),
}


def workload(name: str, rank: int):
    w = dict(WORKLOADS[name])
    m = w["mesh"](rank)
    w["mesh"] = m
    w["name"] = w["desc"].format(T=m.n_tris)
    w["key"] = name
    return w


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


COUNTING_SOURCES = ("outer_volume.cu", "occupancy.cu", "internal.h")


def counting_source_hash():
    """First 16 hex digits of the SHA-256 of the counting kernel's sources (the
    kernel, the occupancy pass that writes its lattice copies, their shared
    types), concatenated in that order."""
    h = hashlib.sha256()
    for f in COUNTING_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2203_10521_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def roofline_inputs(workload_key):
    """DRAM bytes and warp instructions per batch launch of the counting kernel
    from the committed ncu summary of this workload; valid only while the
    kernel and the layout of the lattice copies it reads are unchanged (else
    the values are null)."""
    p = os.path.join(ROOT, "profiles", f"k_count_{workload_key}_roofline_inputs.txt")
    if not os.path.exists(p):
        return {}
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != counting_source_hash():
        return {"stale": True}
    out = {}
    for k in ("dram_bytes_batch_launch", "warp_inst_batch_launch", "alu_pipe_pct", "issue_active_pct"):
        try:
            out[k] = float(kv[k])
        except (KeyError, ValueError):
            pass
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_ranks(t_rank, points, launches, world, device):
    """Whole-job figures over ranks: the slowest rank's time, and the summed
    lattice points and kernel launches (one NCCL/gloo all-reduce each; no
    data-path collective -- the ranks run independent meshes)."""
    if world <= 1:
        return float(t_rank), float(points), int(launches)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_rank)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(points), float(launches)], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p[0].item()), int(p[1].item())


def tree_boxes(ctx, tree, depth):
    boxes = []
    for lev in range(depth + 1):
        r = ctx.tree_read(tree, lev)
        b = r["boxes"].view(np.float32).reshape(-1, 12)
        boxes.append(b)
    return np.ascontiguousarray(np.concatenate(boxes))


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_leaf_boxes(P, depth):
    """The oracle's own leaf boxes of the workload: median splits (Sec. 4.2.2
    top-down decomposition, reading R18) of every node down to `depth`, each
    child's frame from the area-weighted covariance and its tight slab bounds.
    No counting happens here."""
    import oracle as O
    T = P.F.shape[0]
    assign = np.zeros(T, np.int32)
    fr = O.cluster_frames(P.V, P.F, assign, 1, P.center)
    n = O.frame_normals(fr, P.h)
    L = O.Layer(assign, np.zeros(1, np.int32), fr, n, O.tight_bounds(P.U, P.F, assign, 1, n), np.zeros(1, np.uint64))
    K = 1
    for _ in range(depth):
        child = O.median_split(P, L)
        K *= 2
        fr = O.cluster_frames(P.V, P.F, child, K, P.center, fallback=np.repeat(L.frames, 2, axis=0))
        n = O.frame_normals(fr, P.h)
        L = O.Layer(child, (np.arange(K) // 2).astype(np.int32), fr, n, O.tight_bounds(P.U, P.F, child, K, n),
                    np.zeros(K, np.uint64))
    return L.n, L.bnd


def oracle_rate(m, N, n, bnd, order, budget_s, threads):
    """The oracle as it stands on a fresh Problem (no column computed yet):
    leaf boxes in the seeded order, each one per-point occupancy of the
    columns it covers + per-point count (Eq. 4), until the time budget is
    spent.  Returns (in-domain points/s, points, boxes, seconds, threads)."""
    import oracle as O
    used = O.set_threads(threads)
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    pts = nb = 0
    t0 = time.perf_counter()
    for k in order:
        _, _, dom = O.outer_volume(P.occ, n[k:k + 1], bnd[k:k + 1], want_domain=True)
        pts += int(dom[0])
        nb += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    O.set_threads(1)
    return pts / dt, pts, nb, dt, used


def oracle_setup(wl):
    import oracle as O
    O.build()
    m = wl["mesh"]
    P = O.Problem(m.verts, m.tris, wl["N"], adj=np.zeros((m.n_tris, 3), np.int32))
    t0 = time.perf_counter()
    n, bnd = oracle_leaf_boxes(P, wl["depth"])
    order = np.random.Generator(np.random.PCG64(7)).permutation(len(n))
    return n, bnd, order, time.perf_counter() - t0


def cpu_baseline(wl, budget_s):
    n, bnd, order, tree_s = oracle_setup(wl)
    cores = os.cpu_count() or 1
    v1, p1, nb1, dt1, _ = oracle_rate(wl["mesh"], wl["N"], n, bnd, order, budget_s, 1)
    va, pa, nba, dta, used = oracle_rate(wl["mesh"], wl["N"], n, bnd, order, budget_s, cores)
    return {"value": va, "unit": UNIT, "cores": used, "kind": "oracle",
            "single_thread_value": v1, "nproc": cores,
            "sample": (f"leaf boxes of the oracle's own depth-{wl['depth']} median-split tree in a seeded order, each "
                       f"per-point occupancy of its columns + per-point count, in-domain points: {nba} boxes "
                       f"({pa:,} points) in {dta:.1f} s on {used} threads; {nb1} boxes ({p1:,} points) in "
                       f"{dt1:.1f} s on 1 thread; oracle tree {tree_s:.1f} s (untimed)")}


def run_reference(args):
    """Reference arm: the CPU oracle on this host's cores, rank 0 only; each
    step a bounded sample of the workload, timed as the GPU line's
    cpu_baseline times it (all cores)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload, 0)
    n, bnd, order, tree_s = oracle_setup(wl)
    cores = os.cpu_count() or 1
    per_step = max(min(args.cpu_seconds, 120.0 / max(args.steps + args.warmup, 1)), 0.5)
    vals, times, pts_all, nb_all, used = [], [], 0, 0, 1
    at = 0
    for s in range(args.warmup + args.steps):
        sl = np.roll(order, -at)
        v, pts, nb, dt, used = oracle_rate(wl["mesh"], wl["N"], n, bnd, sl, per_step, cores)
        at = (at + nb) % len(order)
        if s >= args.warmup:
            vals.append(v)
            times.append(dt)
            pts_all += pts
            nb_all += nb
    v = float(np.sum(pts_all) / np.sum(times))
    sample = (f"{nb_all} leaf boxes of the oracle's own depth-{wl['depth']} median-split tree over {args.steps} "
              f"steps of about {per_step:.1f} s, each box per-point occupancy of its columns + per-point count, "
              f"in-domain points, {used} threads (nproc {cores})")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(times)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": wl["name"]},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def profile_batch(args):
    """Two counts of the tree batch on the resident lattice (for ncu); the
    boxes come from the file when it exists (few launches before the
    counts), else from the tree built here, which is then saved."""
    import torch
    import paper_2203_10521_gb300 as P
    torch.cuda.set_device(0)
    wl = workload(args.workload, 0)
    m = wl["mesh"]
    ctx = P.Context(0)
    if args.walk:
        ctx.set_counting_rank(0)
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, wl["N"])
    path = args.profile_batch
    if os.path.exists(path):
        boxes = np.load(path)
    else:
        tree = ctx.build_tree(lat, wl["depth"], args.setup_iters)
        if wl["sweeps"]:
            ctx.tree_sweep(tree, sweeps=wl["sweeps"], iters=1)
        boxes = tree_boxes(ctx, tree, wl["depth"])
        np.save(path, boxes)
        tree.free()
    ctx.tune_counting(lat, ctx.quantize_boxes(lat, boxes))   # the tile height the benchmark runs with
    d = torch.from_numpy(boxes).cuda()
    c = ctx.outer_volume(lat, d)
    torch.cuda.nvtx.range_push("profile_batch")
    ctx.outer_volume(lat, d, counts=c)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"boxes": len(boxes), "total_obv": int(c.sum().item())}))
    lat.free()
    mesh.free()
    ctx.close()


def train_surrogate(ctx, args):
    """The surrogate network trained on (box, exact outer volume) pairs from
    runs of the method on the 202,244-triangle union at 512^3 (a depth-10
    tree: Lloyd candidate boxes of every level and perturbed tree boxes),
    features and targets by the library; returns (mlp, training record)."""
    from paper_2203_10521_gb300 import surrogate as S
    t0 = time.perf_counter()
    w = workload("sdf200k-512", 0)
    mesh = ctx.mesh_create(w["mesh"].verts, w["mesh"].tris)
    lat = ctx.build_occupancy(mesh, w["N"])
    tree = ctx.build_tree(lat, w["depth"], 2)
    q, c = S.collect_pairs(ctx, lat, tree, w["depth"], iters=2, perturb=6, seed=3, target_pairs=args.surrogate_pairs)
    t1 = time.perf_counter()
    mlp = ctx.mlp_create(7)
    _, mse0, mse1 = S.train(ctx, mlp, lat, q, c, steps=args.surrogate_steps, batch=1024, lr=2e-3, seed=4)
    rec = {"pairs": int(len(q)), "pairs_from": w["name"], "heldout_mse_before": mse0, "heldout_mse_after": mse1,
           "steps": args.surrogate_steps, "batch": 1024, "collect_s": t1 - t0, "train_s": time.perf_counter() - t1}
    tree.free()
    lat.free()
    mesh.free()
    return mlp, rec


def lloyd_comparison(ctx, lat, tree, depth, args, flush, stream, mlp=None):
    """Lloyd iterations per second on the same freshly split leaf layer: plain
    host-driven, plain as one CUDA graph, and (with a trained surrogate)
    screening candidates and probes (rotation-descent box update, 2 steps);
    final layer totals and exact box counts compared."""
    import torch
    lloyd = {}
    up = ctx.tree_read(tree, depth - 1)
    Kp = 1 << (depth - 1)
    K = 1 << depth
    parent = (np.arange(K) // 2).astype(np.int32)
    up_layer = ctx.layer_init(lat, up["assign"], (np.arange(Kp) // 2).astype(np.int32), up["frames"])
    child = ctx.layer_split(up_layer)
    up_layer.free()
    modes = ["plain", "plain_graph"] + (["surrogate"] if mlp is not None else [])
    for mode in modes:
        lay = ctx.layer_init(lat, child, parent)
        if mode == "surrogate":
            ctx.layer_set_surrogate(lay, mlp, args.surrogate_topk)
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        evals = 0
        torch.cuda.nvtx.range_push("lloyd_" + mode)
        for _ in range(args.lloyd_iters):
            st = ctx.lloyd_step(lay, rounds=16, refit=2, descent_steps=2, graph=(mode == "plain_graph"))
            evals += st["box_evals"]
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        lms = e0.elapsed_time(e1)
        lloyd[mode] = {"iter_per_s": 1000.0 * args.lloyd_iters / lms, "final_total_obv": int(st["total_obv"]),
                       "exact_box_counts": int(evals)}
        lay.free()
    if "surrogate" in lloyd:
        a, b = lloyd["plain"]["final_total_obv"], lloyd["surrogate"]["final_total_obv"]
        lloyd["final_obv_rel_diff"] = (b - a) / a
        lloyd["surrogate_topk"] = args.surrogate_topk
        lloyd["surrogate_vs_plain_iter_ratio"] = lloyd["surrogate"]["iter_per_s"] / lloyd["plain"]["iter_per_s"]
    return lloyd


def lloyd_on_workload(ctx, key, args, flush, stream, mlp):
    """The plain vs screened comparison on another workload (its own mesh,
    lattice and tree, freed afterwards)."""
    w = workload(key, 0)
    mesh = ctx.mesh_create(w["mesh"].verts, w["mesh"].tris)
    lat = ctx.build_occupancy(mesh, w["N"])
    tree = ctx.build_tree(lat, w["depth"], args.setup_iters)
    out = lloyd_comparison(ctx, lat, tree, w["depth"], args, flush, stream, mlp)
    out["workload"] = w["name"]
    tree.free()
    lat.free()
    mesh.free()
    return out


def batch_depths(meshes, seed):
    """Tree depth per mesh of the batched workload: log-uniform in 6..9 and at
    most log2(T / 16)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m, _ in meshes:
        d = int(np.floor(np.exp(rng.uniform(np.log(6), np.log(10)))))
        out.append(max(2, min(d, int(np.log2(m.n_tris / 16)))))
    return out


def batched_lloyd(ctx, args, flush, stream):
    """The batched workload: seeded SDF unions of uneven size (about 1k to
    185k triangles, lattices 128^3 to 384^3, depths 6 to 9), the leaf level of
    each freshly split from its parent level; Lloyd iterations (covariance
    refit) of all of them as one batch -- every round's exact counts of all
    meshes in one counting launch -- against the same iterations mesh by mesh,
    from identical states."""
    import torch
    from synth import meshes as M
    t0 = time.perf_counter()
    meshes = M.sdf_batch(args.batch_meshes, seed=3000)
    depths = batch_depths(meshes, 31)
    objs, A, B = [], [], []
    for (m, N), d in zip(meshes, depths):
        mesh = ctx.mesh_create(m.verts, m.tris)
        lat = ctx.build_occupancy(mesh, N)
        tree = ctx.build_tree(lat, d - 1, 1)
        up = ctx.tree_read(tree, d - 1)
        Kp = 1 << (d - 1)
        up_layer = ctx.layer_init(lat, up["assign"], (np.arange(Kp) // 2).astype(np.int32), up["frames"])
        child = ctx.layer_split(up_layer)
        up_layer.free()
        tree.free()
        parent = (np.arange(2 * Kp) // 2).astype(np.int32)
        A.append(ctx.layer_init(lat, child, parent))
        B.append(ctx.layer_init(lat, child, parent))
        objs.append((mesh, lat))
    batch = ctx.batch_create(A)
    # one untimed iteration in both modes (the batch captures its per-layer
    # graphs on first use); both sides stay in identical states
    ctx.batch_lloyd_step(batch, rounds=16, refit=1)
    for L in B:
        ctx.lloyd_step(L, rounds=16, refit=1)
    setup_s = time.perf_counter() - t0
    res = {}
    for mode in ("batched", "per_mesh"):
        flush.fill_(1)
        torch.cuda.synchronize()
        ctx.profile_enable(2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        moves = 0
        for _ in range(args.batch_iters):
            if mode == "batched":
                st = ctx.batch_lloyd_step(batch, rounds=16, refit=1)
            else:
                st = [ctx.lloyd_step(L, rounds=16, refit=1) for L in B]
            moves += sum(x["moves"] for x in st)
        e1.record(stream)
        torch.cuda.synchronize()
        pr = ctx.profile_read()
        ctx.profile_enable(0)
        sec = e0.elapsed_time(e1) / 1000.0
        res[mode] = {"iter_per_s": args.batch_iters / sec, "points_per_s": pr["count_points_in_domain"] / sec,
                     "counting_launches_per_iter": pr["count_launches"] / args.batch_iters, "moves": int(moves),
                     "final_total_obv": int(sum(x["total_obv"] for x in st))}
    same = all(np.array_equal(ctx.layer_read(a)["obv"], ctx.layer_read(b)["obv"]) for a, b in zip(A, B))
    out = {"meshes": len(meshes), "triangles": int(sum(m.n_tris for m, _ in meshes)),
           "triangles_range": [int(min(m.n_tris for m, _ in meshes)), int(max(m.n_tris for m, _ in meshes))],
           "lattices": sorted({int(N) for _, N in meshes}), "depths": sorted(set(depths)),
           "leaves": int(sum(1 << d for d in depths)), "iters": args.batch_iters, "warmup_iters": 1,
           "setup_s": setup_s,
           "batched": res["batched"], "per_mesh": res["per_mesh"],
           "speedup": res["batched"]["iter_per_s"] / res["per_mesh"]["iter_per_s"],
           "identical_results": bool(same)}
    batch.free()
    for L in A + B:
        L.free()
    for mesh, lat in objs:
        lat.free()
        mesh.free()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_batch:
        profile_batch(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    import paper_2203_10521_gb300 as P

    wl = workload(args.workload, rank)
    m = wl["mesh"]
    N, depth = wl["N"], wl["depth"]
    ctx = P.Context(local)
    if args.walk:
        ctx.set_counting_rank(0)
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    t0 = time.perf_counter()
    tree = ctx.build_tree(lat, depth, args.setup_iters)
    torch.cuda.synchronize()
    tree_s = time.perf_counter() - t0
    sweep = None
    if wl["sweeps"]:
        t0 = time.perf_counter()
        sweep = ctx.tree_sweep(tree, sweeps=wl["sweeps"], iters=1)
        torch.cuda.synchronize()
        sweep["seconds"] = time.perf_counter() - t0
    boxes = tree_boxes(ctx, tree, depth)
    # the counting kernel's rows per tile, chosen by the library's autotuner on this batch
    tile_k, tune_ms = ctx.tune_counting(lat, ctx.quantize_boxes(lat, boxes))
    d_boxes = torch.from_numpy(boxes).cuda()
    d_counts = torch.empty(len(boxes), dtype=torch.int64, device="cuda")
    d_points = torch.empty(len(boxes), dtype=torch.int64, device="cuda")
    leaf = ctx.tree_read(tree, depth)
    K = 1 << depth
    parent = (np.arange(K) // 2).astype(np.int32)
    layer = ctx.layer_init(lat, leaf["assign"], parent, leaf["frames"])
    # the batch's algorithmic bytes, rows and in-domain points (constant: the
    # same boxes on the same lattice every step), from one profiled launch
    ctx.profile_enable(1)
    _, pts0 = ctx.outer_volume(lat, boxes, want_points=True)
    batch_prof = ctx.profile_read()
    ctx.profile_enable(0)
    batch_points = int(pts0.sum())
    batch_dom = int(batch_prof["count_points_in_domain"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    stream = torch.cuda.current_stream()

    def step():
        ctx.occupancy_rebuild(lat)
        ctx.outer_volume(lat, d_boxes, counts=d_counts, points=d_points)
        return ctx.lloyd_step(layer, rounds=16, refit=True, graph=not args.eager_step)

    for _ in range(args.warmup):
        step()
        flush.fill_(1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    # events around every counting launch outside a CUDA graph (the batch
    # launch of each step), the kernel without its profiling counters; the
    # in-domain point total covers every counting launch
    ctx.profile_enable(2)
    launches0 = ctx.profile_read()["launches"]
    evs = []
    lloyd_steps = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")
        e0.record(stream)
        st = step()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        evs.append((e0, e1))
        lloyd_steps.append(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    prof = ctx.profile_read()
    ctx.profile_enable(0)
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    t_rank = sum(ms) / 1000.0
    launches = prof["launches"] - launches0
    pts_dom = prof["count_points_in_domain"]
    t_max, pts_all, launches_all = reduce_ranks(t_rank, pts_dom, launches, world, "cuda")
    value = pts_all / t_max

    mlp, training = (None, None) if args.no_surrogate else train_surrogate(ctx, args)
    lloyd = lloyd_comparison(ctx, lat, tree, depth, args, flush, stream, mlp)
    lloyd["workload"] = wl["name"]
    lloyd_other = None
    if mlp is not None and wl["key"] == "sdf2m-1024" and not args.no_second_workload:
        lloyd_other = lloyd_on_workload(ctx, "sdf1m-768", args, flush, stream, mlp)
    if mlp is not None:
        mlp.free()
    batched = batched_lloyd(ctx, args, flush, stream) if args.batch_meshes > 0 else None

    # roofline of the counting kernel: algorithmic bytes of the batch launch
    # over its event-timed duration in the timed region
    peak, peak_kind = measured_peaks()
    n_batch = prof["count_launches"]
    batch_ms = prof["count_ms"] / max(n_batch, 1)
    achieved = batch_prof["count_bytes"] / (batch_ms / 1000.0) / 1e9 if batch_ms > 0 else 0.0
    ri = {} if args.eager_step or args.walk else roofline_inputs(wl["key"])
    traffic = ri.get("dram_bytes_batch_launch")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_count (outer-volume counting)", "peak_kind": peak_kind,
                "launches_timed": (f"the {len(boxes):,}-box tree batch launch of each step (the Lloyd iteration's "
                                   "counting launches run inside its CUDA graph)"),
                "batch_launch_ms": batch_ms, "batch_bytes": batch_prof["count_bytes"],
                "batch_rows": batch_prof["count_rows"], "batch_rows_rank": batch_prof["count_rows_rank"],
                "batch_share_of_step_time": prof["count_ms"] / sum(ms)}
    if traffic:
        roofline["dram_gbs"] = traffic / (batch_ms / 1000.0) / 1e9
        roofline["dram_frac"] = roofline["dram_gbs"] / peak
    if ri.get("warp_inst_batch_launch"):
        # integer issue: 152 SMs x 4 schedulers x 1 warp instruction per cycle at the sampled SM clock
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        ceiling = 152 * 4 * mhz * 1e6
        roofline["issue"] = {"warp_inst_per_launch": ri["warp_inst_batch_launch"], "ceiling_per_s": ceiling,
                             "frac": ri["warp_inst_batch_launch"] / (batch_ms / 1000.0) / ceiling,
                             "alu_pipe_pct": ri.get("alu_pipe_pct"), "issue_active_pct": ri.get("issue_active_pct")}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e_t, h2d, d2h, e2e_pts = [], 0, 0, []

        def pinned(a):
            # the step's inputs live in page-locked host memory, as a caller
            # streaming meshes to the GPU would keep them
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

        def pinned_like(a):
            # a page-locked array of a's dtype (structured ones included) and shape
            buf = torch.empty(a.nbytes, dtype=torch.uint8).pin_memory().numpy()
            return buf.view(a.dtype).reshape(a.shape)

        p_verts, p_tris, p_boxes = pinned(m.verts), pinned(m.tris), pinned(boxes)
        p_assign, p_parent, p_frames = pinned(leaf["assign"]), pinned(parent), pinned(leaf["frames"])
        # the step's results land in page-locked host arrays too
        p_out = {k: pinned_like(v) for k, v in ctx.layer_read(layer).items()}
        p_cnt, p_pts = pinned_like(np.zeros(len(boxes), np.uint64)), pinned_like(np.zeros(len(boxes), np.uint64))
        for _ in range(max(2, min(args.steps, 5))):
            torch.cuda.synchronize()
            ctx.profile_enable(2)
            t0 = time.perf_counter()
            mh = ctx.mesh_create(p_verts, p_tris)
            lt_ = ctx.build_occupancy(mh, N)
            cnt, pt = ctx.outer_volume(lt_, p_boxes, counts=p_cnt, points=p_pts)
            ly = ctx.layer_init(lt_, p_assign, p_parent, p_frames)
            st = ctx.lloyd_step(ly, rounds=16, refit=True)
            out = ctx.layer_read(ly, out=p_out)
            e2e_t.append(time.perf_counter() - t0)
            e2e_pts.append(ctx.profile_read()["count_points_in_domain"])
            ctx.profile_enable(0)
            h2d = (m.verts.nbytes + m.tris.nbytes + boxes.nbytes + leaf["assign"].nbytes + parent.nbytes
                   + leaf["frames"].nbytes)
            d2h = cnt.nbytes + pt.nbytes + sum(v.nbytes for v in out.values())
            ly.free()
            lt_.free()
            mh.free()
        tm = statistics.median(e2e_t)
        e2e = {"value": statistics.median(e2e_pts) / tm, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * tm,
               "includes": "mesh upload from pinned host memory + device-side validation, occupancy, outer volume "
                           "of the tree batch (pinned host boxes -> host counts), layer init from pinned host "
                           "arrays, one Lloyd iteration, layer read-back"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, args.cpu_seconds)

    if rank == 0:
        last = lloyd_steps[-1]
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
               "config": {"workload": wl["name"], "triangles": m.n_tris, "lattice": N, "tree_depth": depth,
                          "batch_boxes": len(boxes), "sweeps": wl["sweeps"], "lloyd_rounds_per_iter": 16,
                          "lloyd_step": "host-driven rounds" if args.eager_step else "CUDA graph (conditional rounds)",
                          "row_counting": "every word" if args.walk else "rank tables for long rows",
                          "tile_rows_autotuned": tile_k, "autotune_ms": tune_ms,
                          "l2": "flushed between steps (256 MiB write)", "per_rank": "independent mesh (seed + rank)"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_all,
               "clocks": clocks,
               "points": {"in_domain_per_step": pts_dom / args.steps, "batch_in_domain": batch_dom,
                          "batch_out_of_domain": batch_points - batch_dom,
                          "note": "value counts in-domain points only; out-of-domain points are empty by "
                                  "definition and read no memory"},
               "lloyd_iter_per_s": lloyd["plain"]["iter_per_s"],
               "lloyd_graph_iter_per_s": lloyd["plain_graph"]["iter_per_s"],
               "surrogate_lloyd_iter_per_s": lloyd["surrogate"]["iter_per_s"] if "surrogate" in lloyd else None,
               "lloyd_comparison": lloyd, "lloyd_comparison_1m_768": lloyd_other,
               "surrogate_training": training, "batched_lloyd": batched, "lloyd_last_step": last,
               "setup": {"tree_s": tree_s, "sweeps": sweep}, "wall_s_timed": wall}
        print(json.dumps(out), flush=True)
    layer.free()
    tree.free()
    lat.free()
    mesh.free()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
