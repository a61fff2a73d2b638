"""Benchmark: tomogram build + evaluate on one GB300 (or N replicas).

Workload: the five-level parking structure (5M points over 100 x 100 x 20 m,
grid 1000 x 1000 at 0.1 m, 40 slices, robot of height 0.5 m, maximum slope
30 deg, inflation 0.3 m), generated from seed 2.  One step is one
tct_build_evaluate call: partition of the points, the per-tile slice stack
(ground, ceiling, costs, inflation, mask, uniqueness bits) and the
simplification chain, with the points already resident in HBM.  L2 is
flushed (a 256 MB write) before every timed step; the flush is outside the
timed interval.

Printed: one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The benchmark robot, written out here (not read from the library) so that
# the reference arm never loads the CUDA library: Table I of the paper
# (d_min 0.5, d_ref 0.65, theta_b 1.70, theta_p 0.20, c^B 50, alpha_d 20,
# alpha_b 20, alpha_s 15), a maximum slope of 30 deg (theta_s = tan 30 deg),
# an inflation radius d_inf = 0.3 m with the Fig. 3 safe margin d_sm = 0.4 m,
# and a 5 x 5 p_s patch.
ROBOT_PARAMS = dict(d_min=0.5, d_ref=0.65, theta_b=1.70, theta_s=0.5773502691896257,
                    theta_p=0.20, c_b=50.0, alpha_d=20.0, alpha_b=20.0, alpha_s=15.0,
                    d_inf=0.3, d_sm=0.4, patch_radius=2, flags=0)

METRIC = "tomogram build+eval Mpoints/s & slice-cells/s, % HBM roofline; batched vs plain"
UNIT = "Mpoints/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["parking", "parking-small", "building"],
                    default="parking")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-map batched-versus-plain measurement")
    ap.add_argument("--no-planner", action="store_true",
                    help="skip the path search across slices and the refinement of its paths")
    ap.add_argument("--no-stress", action="store_true",
                    help="skip the 60M-point cave-terrain measurement")
    return ap.parse_args()


def workload(name):
    from paper_2403_07631_gb300 import scenes
    if name == "parking":
        return scenes.parking_structure()
    if name == "parking-small":
        # the same structure on 60 x 60 m, pillars and beams scaled with the area
        # (600 x 600 x 40 outputs: 187 MB, above L2)
        return scenes.parking_structure(n_points=1_800_000, side_cells=600, n_pillars=144,
                                        n_beams=108)
    sc = scenes.two_storey_building()
    sc.n_slices = 12
    return sc


def config_of(sc, params):
    return {"workload": sc.name, "points": int(len(sc.points)), "grid": [sc.H, sc.W],
            "res_m": sc.res, "slices": sc.n_slices, "d_s_m": sc.d_s,
            "robot": {"d_min": params["d_min"], "theta_s": round(params["theta_s"], 6),
                      "d_inf": params["d_inf"], "d_sm": params["d_sm"]},
            "seed": sc.meta.get("seed"), "l2": "flushed before each timed step (256 MB write)",
            "inputs": "resident in HBM"}


def algorithmic_bytes(P, N, H, W):
    # xyz read once, e^G, e^C, c^T (float32) and the mask (uint8) written
    # once per slice-cell, the keep flags once per slice
    return 12 * P + 13 * N * H * W + N


def stack_bytes(P, N, H, W):
    # the slice-stack kernel's algorithmic bytes: the per-slice-cell figure of
    # the path (e^G, e^C, c^T float32 and the mask byte written, 13 B) times
    # the slice-cells one launch produces; the point heights it reads back
    # belong to the partition's 12 B per point and are not counted again
    return 13 * N * H * W


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def source_digest(text: str) -> str:
    """First 16 hex digits of the SHA-256 of a CUDA source with its // comments
    and blank lines removed: an edit of the comments keeps the digest, any
    change to the code changes it."""
    import hashlib
    import re
    code = [re.sub(r"//.*$", "", line).rstrip() for line in text.split("\n")]
    return hashlib.sha256("\n".join(c for c in code if c.strip()).encode()).hexdigest()[:16]


def stack_profile():
    """DRAM bytes per launch and issue / ALU activity of the stack kernel from
    the committed ncu summary; an empty dict when the kernel source changed
    since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "k_stack_batched_parking.txt")
    src = os.path.join(ROOT, "paper_2403_07631_gb300", "csrc", "tct_stack_inc.cuh")
    try:
        rec = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        with open(src) as f:
            digest = source_digest(f.read())
        if rec.get("kernel_source_sha256_16") != digest:
            return {}
        return {"traffic": int(rec["traffic_bytes_per_launch"]),
                "issue_active_pct": float(rec["issue_active_pct"]),
                "alu_pipe_active_pct": float(rec["alu_pipe_active_pct"])}
    except (OSError, KeyError, ValueError):
        return {}


def max_over_ranks(ms: float, device) -> float:
    """The step time of the whole job: the slowest rank's (a collective for timing
    only; the ranks exchange no data)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput in millions of units per second: every rank builds its
    own replica of the workload, so the job processes world x units per step."""
    return units_per_rank * world / (ms * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def cpu_baseline(sc, params, min_seconds=10.0, max_runs=20):
    """The FP64 oracle as it stands, on the same workload, on the host cores:
    whole runs (build, evaluate with fragility bounds, chain) repeated until
    `min_seconds` have passed; the value is the mean over the runs."""
    import oracle
    oracle.compile_library()
    op = {k: params[k] for k in oracle.PARAM_FIELDS}
    runs = []
    while not runs or (len(runs) < max_runs and sum(runs) < min_seconds):
        g = oracle.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, 0.0, sc.n_slices)
        t0 = time.perf_counter()
        eG, eC, g, _, _ = oracle.build(sc.points, g, True)
        cT, mask, frag = oracle.evaluate(g, op, eG, eC)
        oracle.simplify(eG, cT, op["c_b"], frag)
        runs.append(time.perf_counter() - t0)
    dt = statistics.mean(runs)
    return {"value": len(sc.points) / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": round(dt, 3), "runs": len(runs),
            "sample": "%d whole runs of the workload (build, evaluate with fragility bounds, "
                      "chain), mean time per run" % len(runs)}


def sampler_paths(dev, grid, params, cost, ground, mask, stats, steps, paths=256, L=512,
                  refine_steps=50, label="the parking structure"):
    """`paths` x `L` waypoints on the evaluated tomogram: straight lines between
    random traversable cells of the most traversable kept slice plus N(0, 0.2 m)
    noise.  Times the query + adjoint kernels and the fused refinement."""
    import torch
    from paper_2403_07631_gb300 import scenes, tct
    st = tct.stats_from(stats)
    g = tct.Grid(grid.x0, grid.y0, grid.res, grid.W, grid.H, grid.d_s, grid.n_slices,
                 float(st.z_min), True)
    k = int(max(range(grid.n_slices), key=lambda i: st.trav_cells[i]))
    xy = torch.from_numpy(scenes.straight_paths(mask[k].cpu().numpy() != 0, grid.x0, grid.y0,
                                                grid.res, paths, L)).to(dev)
    sl = torch.full((paths, L), k, dtype=torch.int32, device=dev)
    q = paths * L
    c_out = torch.empty(paths, L, device=dev)
    e_out = torch.empty(paths, L, device=dev)
    gxy = torch.empty_like(xy)
    ones = torch.ones(paths, L, device=dev)
    stream = torch.cuda.current_stream()

    def fwd_bwd():
        tct.tct_sample_cost(g, cost, ground, xy, sl, c_out, e_out)
        tct.tct_sample_cost_backward(g, cost, ground, xy, sl, ones, None, gxy)

    def timed(fn, n):
        out = []
        for i in range(n + 3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if i >= 3:
                out.append(a.elapsed_time(b))
        return statistics.median(out)

    t_fb = timed(fwd_bwd, max(steps, 10))
    out = {"workload": "%d paths x %d waypoints on slice %d of %s" % (paths, L, k, label),
           "query_fwd_bwd_ms": t_fb, "waypoints_per_s_fwd_bwd": q / (t_fb * 1e-3)}
    if refine_steps:
        tct.tct_sample_cost(g, cost, None, xy, sl, c_out, None)
        before = float(c_out.mean())
        work = xy.clone()

        def refine():
            work.copy_(xy)
            tct.tct_refine_paths(g, cost, sl, work, refine_steps, 1e-3, 1.0)

        t_ref = timed(refine, max(steps, 5))
        tct.tct_sample_cost(g, cost, None, work, sl, c_out, None)
        out.update({"refine_%d_steps_ms" % refine_steps: t_ref,
                    "waypoint_steps_per_s": refine_steps * q / (t_ref * 1e-3),
                    "mean_cost_before": before, "mean_cost_after": float(c_out.mean())})
    return out


def planned_paths(dev, grid, params, ground, cost, keep, stats, n_paths=256, L=512, steps=50):
    """Path search across the kept slices (the library's host stage) between
    random traversable cells of the kept slices, on the host cores; the
    found paths, resampled to L waypoints by arc length, are then refined by
    the fused descent kernel."""
    import numpy as np
    import torch
    from paper_2403_07631_gb300 import tct
    st = tct.stats_from(stats)
    g = tct.Grid(grid.x0, grid.y0, grid.res, grid.W, grid.H, grid.d_s, grid.n_slices,
                 float(st.z_min), True)
    t0 = time.perf_counter()
    h_ground, h_cost, h_keep = ground.cpu().numpy(), cost.cpu().numpy(), keep.cpu().numpy()
    t_copy = time.perf_counter() - t0
    c_b = float(np.float32(params["c_b"]))
    rng = np.random.default_rng(4)
    kept = np.flatnonzero(h_keep)
    trav = [np.flatnonzero(h_cost[k].reshape(-1) < c_b) for k in kept]
    weights = np.array([len(t) for t in trav], np.float64)
    ends = []
    for _ in range(2 * n_paths):
        m = rng.choice(len(kept), p=weights / weights.sum())
        c = int(rng.choice(trav[m]))
        ends.append((c // grid.W, c % grid.W, int(kept[m])))
    starts, goals = ends[:n_paths], ends[n_paths:]
    planner = tct.Planner(g, h_ground, h_cost, h_keep, c_b)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    paths, costs, expanded = planner.plan(starts, goals, max_len=1 << 16, n_threads=threads)
    t_plan = time.perf_counter() - t0
    planner.close()
    reached = [p for p in paths if len(p) >= 2]
    out = {"workload": "%d start/goal pairs on traversable cells of the kept slices" % n_paths,
           "threads": threads, "plan_s": t_plan, "copy_to_host_s": t_copy,
           "paths_per_s": n_paths / t_plan, "reached": len(reached),
           "mean_states_expanded": float(np.mean(expanded)),
           "mean_path_states": float(np.mean([len(p) for p in reached])) if reached else 0.0,
           "paths_crossing_slices": sum(int(len(set(p[:, 2].tolist())) > 1) for p in reached)}
    if not reached:
        return out
    # arc-length resampling of the cell-centre polylines
    xy = np.empty((len(reached), L, 2), np.float32)
    sl = np.empty((len(reached), L), np.int32)
    for r, p in enumerate(reached):
        pts = np.stack([grid.x0 + (p[:, 1] + 0.5) * grid.res,
                        grid.y0 + (p[:, 0] + 0.5) * grid.res], 1)
        s = np.concatenate([[0.0], np.cumsum(np.hypot(*np.diff(pts, axis=0).T))])
        u = np.linspace(0.0, s[-1], L)
        xy[r, :, 0] = np.interp(u, s, pts[:, 0])
        xy[r, :, 1] = np.interp(u, s, pts[:, 1])
        sl[r] = p[np.minimum(np.searchsorted(s, u, side="right") - 1, len(p) - 1), 2]
    d_xy = torch.from_numpy(xy).to(dev)
    d_sl = torch.from_numpy(sl).to(dev)
    c_out = torch.empty(d_sl.shape, device=dev)
    tct.tct_sample_cost(g, cost, None, d_xy, d_sl, c_out, None)
    before = float(c_out.mean())
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    a.record(stream)
    tct.tct_refine_paths(g, cost, d_sl, d_xy, steps, 1e-3, 1.0)
    b.record(stream)
    b.synchronize()
    tct.tct_sample_cost(g, cost, None, d_xy, d_sl, c_out, None)
    out.update({"refine_%d_steps_ms" % steps: a.elapsed_time(b),
                "mean_cost_before": before, "mean_cost_after": float(c_out.mean())})
    return out


def e2e_host(dev, sc, grid, params, steps, kept_only, rounds=3):
    """Host cloud in, host layers out, through tct_build_evaluate_host, on two
    streams with two sets of buffers (device and pinned host): each step
    uploads the points, builds and evaluates, and copies the layers back.
    After one untimed round, times `rounds` rounds of `steps` steps and
    returns the median round's mean time per step (the host link is shared
    with the machine's other GPUs, so one round can see less of it), every
    round's, and the bytes moved per step."""
    import torch
    from paper_2403_07631_gb300 import tct
    P, N, H, W = len(sc.points), sc.n_slices, sc.H, sc.W
    h_xyz = torch.from_numpy(sc.points).pin_memory()
    sets = []
    for _ in range(2):
        d = tct.alloc_outputs(grid, P, dev, params)
        host = [torch.empty(grid.shape, dtype=torch.float32).pin_memory() for _ in range(3)]
        host += [torch.empty(grid.shape, dtype=torch.uint8).pin_memory(),
                 torch.empty(N, dtype=torch.uint8).pin_memory()]
        sets.append((torch.cuda.Stream(), torch.empty_like(h_xyz, device=dev), d, host))
    moved = [0]

    def run(i):
        st, d_xyz, d, host = sets[i & 1]
        with torch.cuda.stream(st):
            m = tct.tct_build_evaluate_host(h_xyz, grid, params, d[0], d_xyz, *d[1:], *host,
                                            kept_only=kept_only)
        moved[0] += m * H * W * 13 + N

    main = torch.cuda.current_stream()
    for i in range(steps):               # an untimed round: first use of the host buffers
        run(i)
    torch.cuda.synchronize()
    per_round = []
    for _ in range(rounds):
        moved[0] = 0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        for st, *_ in sets:
            st.wait_event(a)
        for i in range(steps):
            run(i)
        for st, *_ in sets:
            main.wait_stream(st)
        b.record(main)
        b.synchronize()
        per_round.append(a.elapsed_time(b) / steps)
    return {"ms": statistics.median(per_round), "rounds_ms": per_round, "h2d": P * 12,
            "d2h": moved[0] // steps}


def host_link(dev, nbytes=256 << 20, reps=5):
    """The host link as the copy engines see it, in the same run: pinned host
    to device, device to pinned host, and both at once on two streams (best of
    `reps` copies of `nbytes`, CUDA events)."""
    import torch
    h_src = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_dst = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_a = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_b = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def best(fn):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            s1.wait_event(a)
            s2.wait_event(a)
            fn()
            torch.cuda.current_stream().wait_stream(s1)
            torch.cuda.current_stream().wait_stream(s2)
            b.record()
            b.synchronize()
            out.append(a.elapsed_time(b))
        return min(out)

    def h2d():
        with torch.cuda.stream(s1):
            d_a.copy_(h_src, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            h_dst.copy_(d_b, non_blocking=True)

    def both():
        h2d()
        d2h()

    t1, t2, t3 = best(h2d), best(d2h), best(both)
    return {"h2d_gbs": nbytes / (t1 * 1e-3) / 1e9, "d2h_gbs": nbytes / (t2 * 1e-3) / 1e9,
            "both_gbs": 2 * nbytes / (t3 * 1e-3) / 1e9, "bytes_per_copy": nbytes,
            "how": "pinned host buffers, cudaMemcpyAsync through torch copies, best of %d" % reps}


def separate_calls(dev, sc, grid, params, steps, ground, ceil):
    """The construction alone (tct_build, the paper's T_p) and the evaluation
    alone on the built layers (tct_evaluate, its T_e; Sec. IV-A, Table III),
    each timed with CUDA events, L2 flushed before every call, with its own
    roofline: tct_build moves 12 B per point and writes 8 B per slice-cell,
    tct_evaluate reads those 8 B and writes 5 B per slice-cell."""
    import torch
    from paper_2403_07631_gb300 import tct
    P, N, H, W = len(sc.points), sc.n_slices, sc.H, sc.W
    pts = torch.from_numpy(sc.points).to(dev)
    ws_b = torch.empty(tct.tct_workspace_bytes(grid, P), dtype=torch.uint8, device=dev)
    ws_e = torch.empty(tct.tct_workspace_bytes(grid, 0, params), dtype=torch.uint8, device=dev)
    g2 = torch.empty_like(ground)
    c2 = torch.empty_like(ceil)
    cost2 = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    mask2 = torch.empty(grid.shape, dtype=torch.uint8, device=dev)
    keep2 = torch.empty(N, dtype=torch.uint8, device=dev)
    st_b = torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device=dev)
    st_e = torch.zeros(tct.STATS_BYTES, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    egrid = tct.Grid(grid.x0, grid.y0, grid.res, W, H, grid.d_s, N, 0.0, False)

    def build():
        tct.tct_build(pts, grid, ws_b, g2, c2, st_b)

    def evaluate():
        tct.tct_evaluate(egrid, params, g2, c2, ws_e, cost2, mask2, keep2, None, st_e)

    def timed(fn, n):
        out = []
        for i in range(n + 3):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if i >= 3:
                out.append(a.elapsed_time(b))
        return statistics.median(out)

    t_b = timed(build, steps)
    t_e = timed(evaluate, steps)
    peak, _ = measured_peak_gbs()
    bb = 12 * P + 8 * N * H * W
    eb = 13 * N * H * W + N
    same = bool(torch.equal(g2, ground) and torch.equal(c2, ceil))
    return {"workload": sc.name, "build_ms": t_b, "evaluate_ms": t_e,
            "build_roofline_frac": bb / (t_b * 1e-3) / 1e9 / peak,
            "evaluate_roofline_frac": eb / (t_e * 1e-3) / 1e9 / peak,
            "build_bytes": bb, "evaluate_bytes": eb,
            "layers_equal_fused": same,
            "kernels": "tct_build: partition + per-cell elevation walk; "
                       "tct_evaluate: slice stack on given layers + chain"}


def small_map_graph(dev, params, steps):
    """The two-storey building (200k points, 200 x 200 x 12): a map this small
    is launch-bound, so beside the plain call it is timed as a replay of a
    CUDA graph that captured the call."""
    import torch
    from paper_2403_07631_gb300 import tct
    sc = workload("building")
    grid = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, 0.0, True)
    pts = torch.from_numpy(sc.points).to(dev)
    bufs = tct.alloc_outputs(grid, len(sc.points), dev, params)
    stream = torch.cuda.current_stream()
    tct.tct_timing_enable(False)

    def call():
        tct.tct_build_evaluate(pts, grid, params, *bufs)

    def timed(fn, n):
        out = []
        for i in range(n + 3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if i >= 3:
                out.append(a.elapsed_time(b))
        return statistics.median(out)

    t_plain = timed(call, steps)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        call()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        call()
    t_graph = timed(graph.replay, steps)
    tct.tct_timing_enable(True)          # the later measurements read the phase times
    P, SC = len(sc.points), sc.n_slices * sc.H * sc.W
    return {"workload": sc.name, "plain_us": t_plain * 1e3, "graph_replay_us": t_graph * 1e3,
            "graph_speedup": t_plain / t_graph, "mpoints_per_s_graph": P / (t_graph * 1e-3) / 1e6,
            "slice_cells_per_s_graph": SC / (t_graph * 1e-3)}


def batched_vs_plain(dev, params, steps):
    """64 maps of uneven size (points log-uniform 50k-4M, sides 128-1024 cells,
    4-48 slices): sequential single-map calls against one batched call (tuned by
    the library's autotuner) and against a CUDA-graph replay of that call."""
    import torch
    from paper_2403_07631_gb300 import scenes, tct
    scs = scenes.batched_maps()
    maps = []
    for sc in scs:
        g = tct.Grid(sc.x0, sc.y0, sc.res, sc.W, sc.H, sc.d_s, sc.n_slices, 0.0, True)
        maps.append(tct.MapBuffers.allocate(torch.from_numpy(sc.points).to(dev), g))
    P = sum(len(sc.points) for sc in scs)
    SC = sum(sc.W * sc.H * sc.n_slices for sc in scs)
    ws_plain = torch.empty(max(tct.tct_workspace_bytes(m.grid, m.xyz.shape[0], params) for m in maps),
                           dtype=torch.uint8, device=dev)
    ws = torch.empty(tct.tct_workspace_bytes_batched(maps, params), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def plain():
        for m in maps:
            tct.tct_build_evaluate(m.xyz, m.grid, params, ws_plain, m.ground, m.ceil, m.cost,
                                   m.mask, m.keep, m.stats)

    tuning = tct.tct_autotune_batched(maps, params, ws)

    def batched():
        tct.tct_build_evaluate_batched(maps, params, ws, tuning)

    def timed(fn, n):
        out = []
        for i in range(n + 2):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if i >= 2:
                out.append(a.elapsed_time(b))
        return statistics.median(out)

    t_plain = timed(plain, steps)
    t_batch = timed(batched, steps)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batched()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        batched()
    t_graph = timed(graph.replay, steps)
    return {"workload": "64 buildings, seeds 3000-3063, %.1fM points, %.0fM slice-cells" % (P / 1e6, SC / 1e6),
            "plain_ms": t_plain, "batched_ms": t_batch, "graph_replay_ms": t_graph,
            "batched_speedup": t_plain / t_batch, "graph_speedup": t_plain / t_graph,
            "batched_mpoints_per_s": P / (t_graph * 1e-3) / 1e6,
            "batched_slice_cells_per_s": SC / (t_graph * 1e-3),
            "path_roofline_frac": (12 * P + 13 * SC) / (t_graph * 1e-3) / 1e9 / measured_peak_gbs()[0],
            "tuning": {"tile": {1: "64x64", 2: "32x32", 3: "64x56", 4: "64x40",
                                5: "128x56"}.get(tuning.tile, "auto"),
                       "ctas_per_sm": tuning.ctas_per_sm,
                       "points_per_block": tuning.points_per_block}}


def stress(dev, params, steps):
    """Cave terrain: 60M points over 200 x 200 x 40 m, 4000 x 4000 cells at
    0.05 m (inflation radius 12 cells), 80 slices; one build + evaluate per
    step (inputs resident, L2 flushed before each), then 4096 paths x 512
    waypoints queried forward and backward on the result."""
    import torch
    from paper_2403_07631_gb300 import scenes, tct
    sc = scenes.cave_terrain()
    P, N, H, W = len(sc.points), sc.n_slices, sc.H, sc.W
    grid = tct.Grid(sc.x0, sc.y0, sc.res, W, H, sc.d_s, N, 0.0, True)
    pts = torch.from_numpy(sc.points).to(dev)
    del sc.points
    ws, ground, ceil, cost, mask, keep, stats = tct.alloc_outputs(grid, P, dev, params)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    times, phase = [], []
    for i in range(steps + 2):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tct.tct_build_evaluate(pts, grid, params, ws, ground, ceil, cost, mask, keep, stats)
        b.record(stream)
        ph = tct.tct_timing_read()
        b.synchronize()
        if i >= 2:
            times.append(a.elapsed_time(b))
            phase.append(ph)
    ms = statistics.median(times)
    st = tct.stats_from(stats)
    peak = measured_peak_gbs()[0]
    del ws, ceil, pts
    torch.cuda.empty_cache()
    q = sampler_paths(dev, grid, params, cost, ground, mask, stats, steps, paths=4096, L=512,
                      refine_steps=0, label="the cave terrain")
    stack_ms = statistics.median(p[1] for p in phase)
    return {"workload": sc.name, "points": P, "grid": [H, W], "res_m": sc.res, "slices": N,
            "ms_per_step": ms, "mpoints_per_s": P / (ms * 1e-3) / 1e6,
            "slice_cells_per_s": N * H * W / (ms * 1e-3),
            "path_roofline_frac": algorithmic_bytes(P, N, H, W) / (ms * 1e-3) / 1e9 / peak,
            "phases_ms": {"partition": statistics.median(p[0] for p in phase),
                          "stack": stack_ms, "chain": statistics.median(p[2] for p in phase)},
            "stack_roofline_frac": stack_bytes(P, N, H, W) / (stack_ms * 1e-3) / 1e9 / peak,
            "kept_slices": int(st.n_kept), "dropped_points": int(st.n_dropped),
            "valid_cells": int(sum(st.valid_cells[:N])), "trav_cells": int(sum(st.trav_cells[:N])),
            "queries": q}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    tct_params = dict(ROBOT_PARAMS)
    sc = workload(args.workload)
    times = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(sc, tct_params, min_seconds=0.0, max_runs=1)
        if i >= args.warmup:
            times.append(cb["seconds"])
    t = statistics.mean(times)
    P, N, H, W = len(sc.points), sc.n_slices, sc.H, sc.W
    value = P / t / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config_of(sc, tct_params),
           "slice_cells_per_s": N * H * W / t,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                            "sample": cb["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_2403_07631_gb300 import build as libbuild
    from paper_2403_07631_gb300 import tct

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    libbuild.build()

    params = dict(ROBOT_PARAMS)
    sc = workload(args.workload)
    P, N, H, W = len(sc.points), sc.n_slices, sc.H, sc.W
    grid = tct.Grid(sc.x0, sc.y0, sc.res, W, H, sc.d_s, N, 0.0, True)
    pts = torch.from_numpy(sc.points).to(dev)
    ws, ground, ceil, cost, mask, keep, stats = tct.alloc_outputs(grid, P, dev, params)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        tct.tct_build_evaluate(pts, grid, params, ws, ground, ceil, cost, mask, keep, stats)

    tct.tct_timing_enable(True)
    for _ in range(max(3, args.warmup)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = tct.tct_launch_count()
    phase = []
    for i in range(args.steps):
        flush.fill_(1)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        phase.append(tct.tct_timing_read())
    torch.cuda.synchronize()
    launches = tct.tct_launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms, dev)
    stack_ms = statistics.mean(p[1] for p in phase)
    part_ms = statistics.mean(p[0] for p in phase)
    chain_ms = statistics.mean(p[2] for p in phase)

    # end to end through the C ABI with host buffers: pinned host points in,
    # host layers out (tct_build_evaluate_host), two buffer sets on two streams
    # so that one map's copies overlap the next map's upload and compute
    e2e = e2e_host(dev, sc, grid, params, args.steps, kept_only=False)
    e2e_kept = e2e_host(dev, sc, grid, params, args.steps, kept_only=True)
    link = host_link(dev)

    st = tct.stats_from(stats)
    peak, peak_src = measured_peak_gbs()
    units = P * world
    value = job_value(P, world, ms)
    path_gbs = algorithmic_bytes(P, N, H, W) / (ms * 1e-3) / 1e9
    sb = stack_bytes(P, N, H, W)
    stack_gbs = sb / (stack_ms * 1e-3) / 1e9
    # the committed ncu record is of the parking structure: other workloads get none
    prof = stack_profile() if sc.name.startswith("parking structure 5M") else {}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(sc, params),
        "slice_cells_per_s": N * H * W * world / (ms * 1e-3),
        "path_roofline": {"bound": "hbm", "achieved": path_gbs, "peak": peak, "unit": "GB/s",
                          "frac": path_gbs / peak, "bytes_per_step": algorithmic_bytes(P, N, H, W),
                          "peak_source": peak_src},
        "roofline": {"kernel": "k_stack_batched (per-tile incremental slice stack; 128 x 56 tiles "
                               "of 8-row strips, one CTA of 28 warps per SM, on the parking "
                               "structure)",
                     "bound": "hbm",
                     "achieved": stack_gbs, "peak": peak, "unit": "GB/s", "frac": stack_gbs / peak,
                     "traffic": prof.get("traffic"), "algorithmic_bytes": sb, "ms": stack_ms,
                     "peak_source": peak_src,
                     "issue_active_pct_ncu": prof.get("issue_active_pct"),
                     "alu_pipe_active_pct_ncu": prof.get("alu_pipe_active_pct")},
        "phases_ms": {"partition": part_ms, "stack": stack_ms, "chain": chain_ms},
        "e2e": {"value": units / (e2e["ms"] * 1e-3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                "ms_per_step": e2e["ms"], "rounds_ms": e2e["rounds_ms"],
                "api": "tct_build_evaluate_host, all layers",
                "pipelined": "two streams, two buffer sets",
                "host_link": link,
                # the copies alone at the measured link: the larger direction
                # when both overlap (two streams), the floor of any host path
                "link_floor_ms": max(e2e["h2d"] / (link["h2d_gbs"] * 1e9),
                                     e2e["d2h"] / (link["d2h_gbs"] * 1e9)) * 1e3,
                "frac_of_link": max(e2e["h2d"] / (link["h2d_gbs"] * 1e9),
                                    e2e["d2h"] / (link["d2h_gbs"] * 1e9)) * 1e3 / e2e["ms"]},
        "e2e_kept_slices": {"value": units / (e2e_kept["ms"] * 1e-3) / 1e6, "unit": UNIT,
                            "h2d_bytes_per_step": e2e_kept["h2d"],
                            "d2h_bytes_per_step": e2e_kept["d2h"], "ms_per_step": e2e_kept["ms"],
                            "rounds_ms": e2e_kept["rounds_ms"],
                            "api": "tct_build_evaluate_host, TCT_HOST_KEPT_ONLY (the kept slices)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "kept_slices": int(st.n_kept),
        "paper_context": {"hardware": "RTX 3080 Ti + i9-12900KF (Table III)",
                          "build_plus_eval_ms": "4.4-32.5 on the paper's scenes",
                          "slice_cells_per_s": "about 0.2-0.7 G/s (derived; point counts not given)",
                          "note": "other hardware and scenes: context, not the target"},
        "valid_frac_per_slice": [round(st.valid_cells[k] / (H * W), 4) for k in range(N)],
        "trav_frac_per_slice": [round(st.trav_cells[k] / (H * W), 4) for k in range(N)],
    }
    # the single-GPU measurements beside the headline (queries, small-map graph,
    # path search, batches, stress) run at N = 1 only; at N > 1 every rank
    # would repeat them on shared host cores
    if world == 1:
        out["separate"] = separate_calls(dev, sc, grid, params, min(args.steps, 10), ground, ceil)
        out["sampler"] = sampler_paths(dev, grid, params, cost, ground, mask, stats, args.steps)
        out["small_map"] = small_map_graph(dev, params, args.steps)
        if not args.no_planner:
            out["planned_paths"] = planned_paths(dev, grid, params, ground, cost, keep, stats)
        if not args.no_batched:
            del ws, ground, ceil, cost, mask, keep
            torch.cuda.empty_cache()
            out["batched_vs_plain"] = batched_vs_plain(dev, params, min(args.steps, 5))
            torch.cuda.empty_cache()
        if not args.no_stress:
            if args.no_batched:
                del ws, ground, ceil, cost, mask, keep
                torch.cuda.empty_cache()
            out["stress"] = stress(dev, params, min(args.steps, 3))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sc, params)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
