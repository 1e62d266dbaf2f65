#!/usr/bin/env python
"""Benchmark of the outer-volume / Lloyd hot path on one GB300 per rank.

One step = one pass of the whole path over the workload's batch:
  occupancy rebuild of the 512^3 lattice from the resident mesh (snap,
  column crossings, row scan), exact outer volume of every box of the
  depth-10 tree (2047 FP32 boxes: quantise + count), and one Lloyd iteration
  on the 1,024-leaf layer (partition rounds with exact gains + covariance /
  Jacobi refit), whose layer total is the Eq. 7 leaf term.
value = lattice points counted by the outer-volume kernel per second of
step time (whole job: summed over ranks, divided by the slowest rank).

Workload: the seeded SDF union of 40 spheres + 20 capsules, ~200k
watertight triangles (marching tetrahedra), 512^3 lattice, binary tree of
depth 10.  --small runs the 4,096-triangle torus on 64^3, depth 4.

--impl reference times the CPU oracle (the plain per-point restatement) on a
bounded sample of the same workload.
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
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--small", action="store_true", help="4,096-triangle torus on 64^3 (the oracle-sized case)")
    ap.add_argument("--setup-iters", type=int, default=2, help="Lloyd iterations per level while seeding the tree")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--eager-step", action="store_true",
                    help="host-driven Lloyd rounds in the timed step (default: the step's CUDA graph)")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-topk", type=int, default=5,
                    help="candidates (and rotation probes) per cluster the surrogate keeps for exact counting")
    ap.add_argument("--lloyd-iters", type=int, default=10,
                    help="Lloyd iterations timed for the plain vs surrogate comparison")
    return ap.parse_args()


def workload(small: bool, rank: int):
    from synth import meshes as M
    if small:
        m = M.torus(1.0, 0.3, 64, 32, jitter=0.002, seed=1000 + rank)
        return dict(name="torus R=1 r=0.3, 4,096 triangles, 64^3 lattice, depth 4", mesh=m, N=64, depth=4,
                    iters=10)
    m = M.sdf_union_200k(seed=2000 + rank)
    return dict(name=f"SDF union 40 spheres + 20 capsules, {m.n_tris:,} triangles, 512^3 lattice, depth 10 "
                     f"(1,024 leaves)", mesh=m, N=512, depth=10, iters=20)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def count_kernel_traffic(key="dram_bytes_per_launch"):
    """DRAM bytes per launch of the counting kernel from the committed ncu
    summary (`key`: the average over a step's launches, or the batch launch
    alone), valid only while the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "k_count_roofline_inputs.txt")
    src = os.path.join(ROOT, "paper_2203_10521_gb300", "csrc", "outer_volume.cu")
    if not os.path.exists(p):
        return None, None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            kv[k.strip()] = v.strip()
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if kv.get("source_sha256_16") != h:
        return None, kv.get("workload")
    try:
        return float(kv[key]), kv.get("workload")
    except (KeyError, ValueError):
        return None, None


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


def cpu_oracle_sample(wl, boxes_q_n, boxes_q_b, budget_s):
    """The oracle as it stands, single threaded: per-point occupancy of the
    columns a box needs, then the per-point count, box by box until the time
    budget is spent.  Returns (points/s, points, boxes, seconds)."""
    import oracle as O
    m = wl["mesh"]
    P = O.Problem(m.verts, m.tris, wl["N"], adj=np.zeros((m.n_tris, 3), np.int32))
    pts = 0
    nb = 0
    t0 = time.perf_counter()
    for i in range(len(boxes_q_n)):
        cnt, tot = O.outer_volume(P.occ, boxes_q_n[i:i + 1], boxes_q_b[i:i + 1])
        pts += int(tot[0])
        nb += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return pts / dt, pts, nb, dt


def run_reference(args):
    """Reference arm: the CPU oracle, timed on this host, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.build()
    wl = workload(args.small, 0)
    m = wl["mesh"]
    N = wl["N"]
    # boxes: leaf-sized boxes of the workload -- the oracle's own tree is far too
    # slow at this size, so use median-split boxes of the oracle's root frame
    P = O.Problem(m.verts, m.tris, N, adj=np.zeros((m.n_tris, 3), np.int32))
    T = m.n_tris
    fr = O.cluster_frames(P.V, P.F, np.zeros(T, np.int32), 1, P.center)
    L = O.Layer(np.zeros(T, np.int32), np.zeros(1, np.int32), fr, O.frame_normals(fr, P.h),
                O.tight_bounds(P.U, P.F, np.zeros(T, np.int32), 1, O.frame_normals(fr, P.h)), np.zeros(1, np.uint64))
    assign = np.zeros(T, np.int32)
    K = 1
    for _ in range(wl["depth"]):
        child = O.median_split(P, L)
        K *= 2
        fr = np.repeat(L.frames, 2, axis=0)
        n = O.frame_normals(fr, P.h)
        L = O.Layer(child, (np.arange(K) // 2).astype(np.int32), fr, n, O.tight_bounds(P.U, P.F, child, K, n),
                    np.zeros(K, np.uint64))
    rng = np.random.Generator(np.random.PCG64(7))
    order = rng.permutation(K)
    per_step = max(args.cpu_seconds / max(args.steps + args.warmup, 1), 0.5)
    vals, times = [], []
    i = 0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pts = 0
        while time.perf_counter() - t0 < per_step:
            k = order[i % K]
            i += 1
            cnt, tot = O.outer_volume(P.occ, L.n[k:k + 1], L.bnd[k:k + 1])
            pts += int(tot[0])
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            vals.append(pts / dt)
            times.append(dt)
    v = float(np.mean(vals))
    sample = (f"{i} leaf boxes (median-split seeds of the {K:,}-leaf level), per-point occupancy of their "
              f"columns + per-point count, single thread, about {per_step:.1f} s per step")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(times)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": wl["name"]},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
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

    wl = workload(args.small, rank)
    m = wl["mesh"]
    N, depth = wl["N"], wl["depth"]
    ctx = P.Context(local)
    mesh = ctx.mesh_create(m.verts, m.tris)
    lat = ctx.build_occupancy(mesh, N)
    t0 = time.perf_counter()
    tree = ctx.build_tree(lat, depth, args.setup_iters)
    torch.cuda.synchronize()
    tree_s = time.perf_counter() - t0
    boxes = tree_boxes(ctx, tree, depth)
    d_boxes = torch.from_numpy(boxes).cuda()
    d_counts = torch.empty(len(boxes), dtype=torch.int64, device="cuda")
    d_points = torch.empty(len(boxes), dtype=torch.int64, device="cuda")
    leaf = ctx.tree_read(tree, depth)
    K = 1 << depth
    parent = (np.arange(K) // 2).astype(np.int32)
    layer = ctx.layer_init(lat, leaf["assign"], parent, leaf["frames"])
    # lattice points of the batch (constant: same boxes on the same lattice)
    _, pts0 = ctx.outer_volume(lat, boxes, want_points=True)
    batch_points = int(pts0.sum())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    stream = torch.cuda.current_stream()

    def step():
        ctx.occupancy_rebuild(lat)
        ctx.outer_volume(lat, d_boxes, counts=d_counts, points=d_points)
        st = ctx.lloyd_step(layer, rounds=16, refit=True, graph=not args.eager_step)
        return st

    for _ in range(args.warmup):
        step()
        flush.fill_(1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ctx.profile_enable(True)
    launches0 = ctx.profile_read()["launches"]
    evs = []
    pts_total = 0
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
        pts_total += batch_points + st["points_counted"]
        lloyd_steps.append(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    t_rank = sum(ms) / 1000.0
    launches = prof["launches"] - launches0
    t_max, pts_all, launches_all = reduce_ranks(t_rank, pts_total, launches, world, "cuda")
    value = pts_all / t_max

    # Lloyd iterations per second, plain vs surrogate-screened: the same freshly
    # split leaf layer, the rotation-descent box update (6 probes per cluster,
    # 2 steps), timed with CUDA events; final layer totals compared
    lloyd = {}
    up = ctx.tree_read(tree, depth - 1)
    Kp = 1 << (depth - 1)
    up_layer = ctx.layer_init(lat, up["assign"], (np.arange(Kp) // 2).astype(np.int32), up["frames"])
    child = ctx.layer_split(up_layer)
    up_layer.free()
    mlp = None
    modes = ["plain", "plain_graph"] if args.no_surrogate else ["plain", "plain_graph", "surrogate"]
    if not args.no_surrogate:
        from paper_2203_10521_gb300 import surrogate as S
        t0 = time.perf_counter()
        mlp = ctx.mlp_create(7)
        q, c = S.collect_pairs(ctx, lat, tree, depth, iters=2, perturb=6, seed=3)
        _, mse0, mse1 = S.train(ctx, mlp, lat, q, c, steps=400, batch=1024, lr=2e-3, seed=4)
        lloyd["surrogate_training"] = {"pairs": int(len(q)), "heldout_mse_before": mse0, "heldout_mse_after": mse1,
                                       "seconds": time.perf_counter() - t0}
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
    lloyd_iter_per_s = lloyd["plain"]["iter_per_s"]
    lloyd_graph_iter_per_s = lloyd["plain_graph"]["iter_per_s"]
    surrogate_iter_per_s = lloyd["surrogate"]["iter_per_s"] if "surrogate" in lloyd else None
    if "surrogate" in lloyd:
        a, b = lloyd["plain"]["final_total_obv"], lloyd["surrogate"]["final_total_obv"]
        lloyd["final_obv_rel_diff"] = (b - a) / a
        lloyd["surrogate_topk"] = args.surrogate_topk
    if mlp is not None:
        mlp.free()

    # roofline of the counting kernel (the dominant kernel), live over the timed region
    peak, peak_kind = measured_peaks()
    achieved = prof["count_bytes"] / (prof["count_ms"] / 1000.0) / 1e9 if prof["count_ms"] > 0 else 0.0
    # with the Lloyd step as a CUDA graph, its counting launches run inside the
    # graph and only the batch launch of each step is bracketed by events
    traffic, traffic_wl = count_kernel_traffic("dram_bytes_per_launch" if args.eager_step
                                               else "dram_bytes_batch_launch")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_count (outer-volume counting)", "peak_kind": peak_kind,
                "launches_timed": ("every counting launch of each step" if args.eager_step else
                                   f"the {len(boxes):,}-box batch launch of each step (the Lloyd step's "
                                   "counting launches run inside its CUDA graph)"),
                "count_launches": prof["count_launches"], "count_ms_total": prof["count_ms"],
                "count_bytes_total": prof["count_bytes"], "count_rows": prof["count_rows"],
                "count_share_of_step_time": prof["count_ms"] / sum(ms)}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e_t, e2e_pts, h2d, d2h = [], 0, 0, 0

        def pinned(a):
            # the step's inputs live in page-locked host memory, as a caller
            # streaming meshes to the GPU would keep them
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

        p_verts, p_tris, p_boxes = pinned(m.verts), pinned(m.tris), pinned(boxes)
        p_assign, p_parent, p_frames = pinned(leaf["assign"]), pinned(parent), pinned(leaf["frames"])
        for _ in range(max(2, min(args.steps, 5))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mh = ctx.mesh_create(p_verts, p_tris)
            lt_ = ctx.build_occupancy(mh, N)
            cnt, pt = ctx.outer_volume(lt_, p_boxes, want_points=True)
            ly = ctx.layer_init(lt_, p_assign, p_parent, p_frames)
            st = ctx.lloyd_step(ly, rounds=16, refit=True)
            out = ctx.layer_read(ly)
            e2e_t.append(time.perf_counter() - t0)
            e2e_pts = int(pt.sum()) + st["points_counted"]
            h2d = (m.verts.nbytes + m.tris.nbytes + boxes.nbytes + leaf["assign"].nbytes + parent.nbytes
                   + leaf["frames"].nbytes)
            d2h = cnt.nbytes + pt.nbytes + sum(v.nbytes for v in out.values())
            ly.free()
            lt_.free()
            mh.free()
        e2e = {"value": e2e_pts / statistics.median(e2e_t), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * statistics.median(e2e_t),
               "includes": "mesh upload from pinned host memory + device-side validation, occupancy, outer volume "
                           "of the tree batch (pinned host boxes -> host counts), layer init from pinned host "
                           "arrays, one Lloyd iteration, layer read-back"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        q = leaf["qboxes"]
        rng = np.random.Generator(np.random.PCG64(7))
        order = rng.permutation(len(q))
        v, p_, nb, dt = cpu_oracle_sample(wl, q["n"][order], q["b"][order], args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nb} leaf boxes of the 1,024-leaf layer ({p_:,} lattice points): per-point occupancy "
                         f"of their columns + per-point count, single thread, {dt:.1f} s"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
               "config": {"workload": wl["name"], "triangles": m.n_tris, "lattice": N, "tree_depth": depth,
                          "batch_boxes": len(boxes), "lloyd_rounds_per_iter": 16,
                          "lloyd_step": "host-driven rounds" if args.eager_step else "CUDA graph (conditional rounds)",
                          "l2": "flushed between steps (256 MiB write)", "per_rank": "independent mesh (seed + rank)"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_all,
               "clocks": clocks, "lloyd_iter_per_s": lloyd_iter_per_s,
               "lloyd_graph_iter_per_s": lloyd_graph_iter_per_s,
               "surrogate_lloyd_iter_per_s": surrogate_iter_per_s, "lloyd_comparison": lloyd,
               "lloyd_last_step": lloyd_steps[-1], "tree_setup_s": tree_s, "wall_s_timed": wall}
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
