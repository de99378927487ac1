#!/usr/bin/env python3
"""Throughput of the ORCA step on GB300: agent-steps/s.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload clusters_1m|shared_space_65k|open_square_1k]

A step is one synchronous ORCA update of every agent of the workload (grid
binning, k-nearest neighbours, ORCA half-planes, velocity LP with the
least-penetration fallback, integration), through the C ABI, from
device-resident state.  Default workload: 1,000,000 agents in 64 Gaussian
clusters over 2 x 2 km (10,000 vehicles).  L2 (129 MB) is flushed before
every timed step by writing a 256 MB buffer outside the timed events.

Under torchrun every rank runs an independent replica (weak scaling, no
collective on the data path); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle on this host's cores on a
bounded sample of agents per step (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "agent-steps/s"

# Algorithmic FP32 operations per counted item (add/sub/mul/div/sqrt/compare
# = 1, fused multiply-add = 2):
#   candidate key test: 2 sub, 2 mul, 1 add, 1 compare with R_n^2      =  6
#   ORCA half-plane: relative state, obstacle test, cut-off or leg
#     construction with one sqrt and one or two divides, leg side
#     filter, placement (50-64 by branch)                            = 60
#   LP pair evaluation: 2 determinants, 1 divide, 1 bound           = 10
#   per agent: preferred velocity 10, disc clip 6, integration 4,
#     1D set-ups amortised 10                                       = 30
FLOPS_CAND, FLOPS_LINE, FLOPS_PAIR, FLOPS_AGENT = 6, 60, 10, 30
# Algorithmic DRAM bytes of binning per agent (the method's per-unit figure
# for binning and reorder): cell key written and read 8, permutation written
# and read 8, the 36-byte agent state read and written in sorted order 72.
BIN_BYTES_METHOD = 88
# The binning kernel's own traffic, for comparison (first step of a call;
# the bench times one-step calls, so every timed step is a first step):
#   cell keys: order entry 4, caller state (position 8, velocity 8, radius 4,
#     type 1) 21 read, key + slot 8 and the staged state 24 written, cell
#     counter 8 (atomic read-modify-write)                           = 65 / agent
#   cell order: key + slot 8, cell start 4, x 4 read, (x key, index) 8 written
#                                                                    = 24 / agent
#   order by x: (x key, index) 8, key 4, cell range 8 read, staged state 24
#     read, sorted state 24 written                                  = 68 / agent
#   scan: count read 4, count cleared 4, start written 4              = 12 / cell
# Later steps of a call skip the cell-key phase (the solve kernel bins the
# new positions) and read the previous step's state instead of the staged one.
BIN_BYTES_KERNEL_FIRST, BIN_BYTES_KERNEL_LATER, BIN_BYTES_CELL = 65 + 24 + 68, 24 + 68, 12
FP32_LANES = 128    # FP32 lanes per SM (sm_103a)
N_COUNTERS = 13     # work tallies of the counting solve variant (layout in orca.h)


def _source_hash():
    import hashlib
    root = os.path.join(ROOT, "paper_2008_11578_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(root)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(root, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "orca.h"), "rb").read())
    return h.hexdigest()[:16]


def _profiled(workload, kernel="solve_kernel"):
    """Figures of the committed ncu capture of a kernel (DRAM bytes per
    launch, and for the solve kernel issue-slot and SIMT utilisation), or {}
    when the CUDA sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload.split('_', 1)[0]}_1m.md")
    try:
        txt = open(path).read()
    except OSError:
        return {}
    keys = ("kernel_source_hash", "traffic_bytes_per_launch", "issue_active_pct",
            "simt_efficiency_pct", "warp_instructions_per_launch")
    vals = dict(line.split(": ", 1) for line in txt.splitlines()
                if line.startswith(tuple(k + ": " for k in keys)))
    if vals.get("kernel_source_hash", "").strip() != _source_hash():
        return {}
    out = {}
    for k, conv in (("traffic_bytes_per_launch", int), ("issue_active_pct", float),
                    ("simt_efficiency_pct", float), ("warp_instructions_per_launch", int)):
        try:
            out[k] = conv(vals[k])
        except (KeyError, ValueError):
            pass
    return out


def _profiled_traffic(workload):
    """DRAM bytes per solve launch from the committed ncu summary, or None
    when the CUDA sources changed since that capture."""
    return _profiled(workload).get("traffic_bytes_per_launch")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def _scene(name):
    from paper_2008_11578_gb300 import scenes
    if name == "clusters_1m":
        return scenes.clusters(), dict(workload="clusters_1m", agents=1_000_000,
                                       vehicles=10_000, area_m="2000x2000",
                                       clusters=64, sigma_m=20.0)
    if name == "shared_space_65k":
        return scenes.shared_space(), dict(workload="shared_space_65k", agents=65_000,
                                           vehicles=1_000, area_m="500x500")
    if name == "open_square_1k":
        return scenes.open_square(), dict(workload="open_square_1k", agents=1_000,
                                          vehicles=0, area_m="50x50")
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu_index), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.remove(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_throughput(local_seconds, units, world, device=None):
    """Whole-job throughput of `world` independent replicas.

    Each rank processed `units` units in `local_seconds`; the job takes as long
    as its slowest rank, so the rate is world * units / max over ranks.
    Returns (rate, slowest seconds).  Collective only when world > 1.
    """
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slowest = float(t.item())
    return units * world / slowest, slowest


def run_reference(args):
    """The FP64 CPU oracle on this host's cores, bounded sample per step."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    import oracle
    scene, cfg = _scene(args.workload)
    oracle.build()
    cores = oracle.num_threads()
    rng = np.random.default_rng(0)
    # size the per-step sample so one step takes about 2 s of CPU time
    probe = np.sort(rng.choice(scene.n, min(scene.n, 256), replace=False))
    t0 = time.perf_counter()
    oracle.step(scene, sel=probe)
    per_agent = (time.perf_counter() - t0) / len(probe)
    m = int(min(scene.n, max(64, 2.0 / max(per_agent, 1e-9))))
    for _ in range(args.warmup):
        oracle.step(scene, sel=np.sort(rng.choice(scene.n, min(m, 256), replace=False)))
    times = []
    for _ in range(args.steps):
        sel = np.sort(rng.choice(scene.n, m, replace=False))
        t0 = time.perf_counter()
        oracle.step(scene, sel=sel)
        times.append(time.perf_counter() - t0)
    value = m * args.steps / sum(times)
    sample = (f"{m} agents drawn per step from the {cfg['agents']}-agent workload, "
              f"FP64 oracle (brute-force neighbours), {args.steps} steps from the initial state")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step_sample": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _parity_stats(scene, r, gpu, sel):
    """One GPU step against the oracle's results ``r`` for agents ``sel``:
    neighbour lists (bit-exact), velocity and position errors, and the
    ill-conditioned agents (active-set condition number > 1e3) apart."""
    import numpy as np
    k = int(scene.params.max_neighbors)
    nb_same = np.array_equal(gpu["cnt"][sel], r.cnt) and \
        np.array_equal(gpu["nbr"][sel][:, :k], r.nbr)
    dv = np.abs(gpu["vel"][sel].astype(np.float64) - r.vel).max(1)
    p32 = np.abs(r.pos.astype(np.float32))
    half_ulp = 0.5 * (np.nextafter(p32, np.float32(np.inf)) - p32).astype(np.float64)
    dp = np.maximum(np.abs(gpu["pos"][sel].astype(np.float64) - r.pos) - half_ulp, 0.0).max(1)
    ill = r.cond > 1e3
    w = int(np.argmax(dv)) if len(dv) else 0
    worst = {"agent": int(sel[w]), "dv_m_s": float(dv[w]), "cond": float(r.cond[w]),
             "tstar_oracle": float(r.tstar[w]), "flags_oracle": int(r.flags[w]),
             "flags_gpu": int(gpu["flags"][sel[w]])} if len(dv) else None
    return {"agents": int(len(sel)), "neighbour_lists_bit_exact": bool(nb_same),
            "worst": worst,
            "max_dv_m_s": float(dv.max(initial=0.0)),
            "p9999_dv_m_s": float(np.quantile(dv, 0.9999)) if len(dv) else 0.0,
            "max_dp_beyond_half_ulp_m": float(dp.max(initial=0.0)),
            "ill_conditioned": int(ill.sum()),
            "ill_conditioned_max_dv_m_s": float(dv[ill].max(initial=0.0)),
            "ill_conditioned_p9999_dv_m_s": float(np.quantile(dv[ill], 0.9999))
            if ill.any() else 0.0,
            "least_penetration_agents": int((r.flags & 1).sum()),
            "tolerance": {"dv_m_s": 1e-4, "dp_m": 1e-5}}


def cpu_baseline(scene, cfg, gpu=None, budget_s=2.5, reps=5):
    """The FP64 oracle timed on a bounded sample of the same workload (rank 0,
    N=1): best of ``reps`` runs after a warm-up, on all host cores, and the
    same on one core with a smaller sample.  ``gpu`` is one GPU step from
    ``scene``'s state (numpy pos, vel, nbr, cnt, flags); the timed oracle
    results of the all-core sample are compared with it agent by agent."""
    import numpy as np

    import oracle
    oracle.build()
    cores = oracle.num_threads()
    rng = np.random.default_rng(1)
    # a probe large enough to keep every host core busy, so that the
    # per-agent cost it measures holds for the sample
    probe = np.sort(rng.choice(scene.n, min(scene.n, 4000), replace=False))
    t0 = time.perf_counter()
    oracle.step(scene, sel=probe)
    per_agent = (time.perf_counter() - t0) / len(probe)

    def best_of(m):
        sel = np.sort(rng.choice(scene.n, m, replace=False))
        oracle.step(scene, sel=sel[:max(1, m // 4)])          # warm-up
        times, r = [], None
        for _ in range(reps):
            t0 = time.perf_counter()
            r = oracle.step(scene, sel=sel)
            times.append(time.perf_counter() - t0)
        return sel, r, min(times)

    m = int(min(scene.n, max(100, budget_s / max(per_agent, 1e-12))))
    sel, r, t_all = best_of(m)
    oracle.set_num_threads(1)
    try:
        m1 = int(min(scene.n, max(10, budget_s / max(per_agent * cores, 1e-12))))
        _, _, t_one = best_of(m1)
    finally:
        oracle.set_num_threads(cores)
    out = {"value": m / t_all, "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": f"{m} agents drawn from the {cfg['agents']}-agent workload, one step "
                     f"(FP64, brute-force neighbours), best of {reps} after a warm-up",
           "single_core": {"value": m1 / t_one, "unit": METRIC, "cores": 1,
                           "sample": f"{m1} agents, best of {reps} after a warm-up"}}
    parity = _parity_stats(scene, r, gpu, sel) if gpu is not None else None
    out["other_workloads"] = _cpu_baseline_other(reps)
    return out, parity


def _cpu_baseline_other(reps, budget_s=1.0):
    """The oracle on the other workloads' initial states (all host cores,
    one step, best of ``reps`` after a warm-up, a bounded sample where a
    whole step would take longer than ``budget_s``)."""
    import numpy as np

    import oracle
    from paper_2008_11578_gb300 import scenes
    rng = np.random.default_rng(2)
    out = {}
    sl = scenes.batched()
    for name, sc in (("open_square_1k", scenes.open_square()),
                     ("shared_space_65k", scenes.shared_space()),
                     ("batched_512_largest_scene", max(sl, key=lambda x: x.n)),
                     ("waypoint_square_4k", scenes.waypoint_square())):
        probe = np.sort(rng.choice(sc.n, min(sc.n, 500), replace=False))
        t0 = time.perf_counter()
        oracle.step(sc, sel=probe)
        per_agent = (time.perf_counter() - t0) / len(probe)
        m = int(min(sc.n, max(50, budget_s / max(per_agent, 1e-12))))
        sel = None if m == sc.n else np.sort(rng.choice(sc.n, m, replace=False))
        oracle.step(sc, sel=sel)
        best = min(_timed(lambda: oracle.step(sc, sel=sel)) for _ in range(reps))
        out[name] = {"value": m / best, "unit": METRIC, "agents": sc.n,
                     "sample": m, "cores": oracle.num_threads()}
    return out


def _timed(fn):
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def measure_batched(dev, flush, n_steps=50, tune=True):
    """512 independent scenes (log-uniform sizes in [100, 20,000]): one CUDA
    graph of ``n_steps`` batched steps against two per-scene baselines from
    the same state: the plain loop that calls orca_step(n_steps) scene by
    scene (its host enqueue time and GPU time reported apart), and the same
    loop with every scene's ``n_steps`` captured as its own CUDA graph (no
    per-launch host cost).  All three must end bit-identical."""
    import torch

    from paper_2008_11578_gb300 import api, autotune, scenes
    sl = scenes.batched()
    total = sum(s.n for s in sl)
    stream = torch.cuda.current_stream()
    tuned = None
    cells = heights = None
    block = 0
    if tune:
        tuned = autotune.tune_batch(sl, dev, alphas=(0.25, 0.375, 0.5, 0.75, 1.0),
                                    aspects=(1.0, 2.0, 4.0), steps=3, warmup=1)
        cells = tuned.cell_sizes(sl)
        heights = tuned.cell_heights(sl)
        block = tuned.block_size
    b = api.DeviceBatch(sl, dev, cell_sizes=cells, cell_heights=heights, block_size=block)
    pos0, vel0 = b.pos.clone(), b.vel.clone()
    b.capture(n_steps)
    b.replay()                                   # warm-up replay
    torch.cuda.synchronize()
    b.pos.copy_(pos0)
    b.vel.copy_(vel0)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.replay(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1)
    status = b.sync_status()

    plain = [api.DeviceScene(s, dev, cell_size=None if cells is None else cells[i],
                             cell_height=None if heights is None else heights[i],
                             block_size=block) for i, s in enumerate(sl)]
    for ds in plain:                             # warm-up call per scene
        ds.step(1)
    torch.cuda.synchronize()

    def reset():
        for ds, s in zip(plain, sl):
            ds.set_state(pos=s.pos, vel=s.vel)
        torch.cuda.synchronize()
        flush.zero_()

    reset()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    h0 = time.perf_counter()
    for ds in plain:
        ds.step(n_steps)
    host_ms = 1e3 * (time.perf_counter() - h0)
    p1.record(stream)
    torch.cuda.synchronize()
    loop_ms = p0.elapsed_time(p1)
    same = all(torch.equal(ds.pos, b.pos[b.scene_slice(i)]) and
               torch.equal(ds.vel, b.vel[b.scene_slice(i)]) for i, ds in enumerate(plain))

    # the same loop, every scene's steps replayed from its own CUDA graph
    for ds in plain:
        ds.capture(n_steps)
    reset()
    for ds in plain:                             # warm-up replay
        ds.replay(stream)
    reset()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    h0 = time.perf_counter()
    for ds in plain:
        ds.replay(stream)
    graph_host_ms = 1e3 * (time.perf_counter() - h0)
    q1.record(stream)
    torch.cuda.synchronize()
    loop_graph_ms = q0.elapsed_time(q1)
    same_graph = all(torch.equal(ds.pos, b.pos[b.scene_slice(i)]) and
                     torch.equal(ds.vel, b.vel[b.scene_slice(i)]) for i, ds in enumerate(plain))
    graph_launches = b.launch_count(n_steps)
    loop_launches = sum(ds.launch_count(n_steps) for ds in plain)
    for ds in plain:
        ds.close()
    b.close()
    return {"workload": "batched_512", "scenes": len(sl), "agents": total,
            "steps": n_steps, "graph_value": total * n_steps / (graph_ms / 1e3),
            "plain_loop_value": total * n_steps / (loop_ms / 1e3), "unit": METRIC,
            "graph_ms": graph_ms, "plain_loop_ms": loop_ms,
            "plain_loop_host_enqueue_ms": host_ms,
            "plain_loop_us_per_launch": 1e3 * loop_ms / loop_launches,
            "plain_loop_graph_ms": loop_graph_ms,
            "plain_loop_graph_host_ms": graph_host_ms,
            "speedup_vs_plain_loop": loop_ms / graph_ms,
            "speedup_vs_plain_loop_graph": loop_graph_ms / graph_ms,
            "bitwise_equal": bool(same and same_graph),
            "graph_launches": graph_launches, "plain_loop_launches": loop_launches,
            "status": status,
            "autotune": None if tuned is None else
            {"height_factor": tuned.alpha, "aspect": tuned.aspect,
             "block_size": tuned.block_size,
             "candidates": [[a, asp, bs, ms] for a, asp, bs, ms in tuned.table]}}


def measure_adjoint(dev, n_steps=40, ckpt_every=8, reps=5):
    """The adjoint workload (4,000 pedestrians + 64 vehicles with 8 waypoints,
    100 x 100 m): the checkpointing forward (orca_rollout) and the adjoint
    (orca_adjoint: segment replays + reverse steps), CUDA events on the
    launching stream, median of ``reps``."""
    import torch

    from paper_2008_11578_gb300 import api, scenes
    from paper_2008_11578_gb300.adjoint import Rollout, workload_loss
    s = scenes.waypoint_square()
    roll = Rollout(s, n_steps, ckpt_every, device=dev)
    stream = torch.cuda.current_stream()
    d = torch.zeros((n_steps, s.n, 2), dtype=torch.float32, device=dev)
    goal = torch.as_tensor(s.goal, device=dev)
    veh = torch.as_tensor(s.type == 1, device=dev)
    fw, bw, plain = [], [], []
    for r in range(reps + 1):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        roll.forward_raw(d)
        e[1].record(stream)
        pos_T = roll.ds.pos.clone().requires_grad_(True)
        vt = roll.vel_traj.clone().requires_grad_(True)
        gp, gv = torch.autograd.grad(workload_loss(pos_T, vt, goal, veh), [pos_T, vt])
        e[2].record(stream)
        roll.backward_raw(d, gp, gv)
        e[3].record(stream)
        roll.reset()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        roll.ds.step(n_steps, d)
        p1.record(stream)
        torch.cuda.synchronize()
        if r > 0:                                   # the first pass is warm-up
            fw.append(e[0].elapsed_time(e[1]))
            bw.append(e[2].elapsed_time(e[3]))
            plain.append(p0.elapsed_time(p1))
    f, b, pl = statistics.median(fw), statistics.median(bw), statistics.median(plain)
    out = {"workload": "waypoint_square_4k", "agents": s.n, "vehicles": int((s.type == 1).sum()),
           "steps": n_steps, "ckpt_every": ckpt_every, "forward_ms": f, "adjoint_ms": b,
           "plain_steps_ms": pl, "adjoint_over_forward": b / f,
           "forward_value": s.n * n_steps / (f / 1e3), "unit": METRIC,
           "adjoint_launches": api.orca_adjoint_launch_count(roll.ds.handle, n_steps,
                                                             ckpt_every)}
    roll.close()
    return out


def measure_vehicle_share(dev, flush, cell, cell_h, block, steps=10, warmup=3):
    """The paper's claim that the vehicle share costs nothing (one code path
    for every agent type, Sec. 3.1 and Sec. 4): the 1M-agent cluster step at
    0, 1, 5 and 50 % vehicles, same positions and goals, same launch shape.
    Each share: ``warmup`` steps from the initial state, then ``steps``
    one-step calls from that one state (restored before each, L2 flushed),
    median; then one counting step from the same state gives the work per
    agent (candidates, LP pair evaluations, least-penetration fraction), so
    that a difference in time can be told apart from a difference in the
    crowd's physics (vehicles are larger and faster, so they change the
    overlaps and the LPs, not the code path)."""
    import numpy as np
    import torch

    from paper_2008_11578_gb300 import api, scenes
    stream = torch.cuda.current_stream()
    out = {}
    for label, every in (("0%", 0), ("1%", 100), ("5%", 20), ("50%", 2)):
        sc = scenes.clusters(vehicle_every=every if every else 100)
        if every == 0:
            sc.type[:] = 0
        veh = sc.type == 1
        sc.radius = np.where(veh, 1.5, 0.5).astype(np.float32)
        sc.max_speed = np.where(veh, 5.0, 1.5).astype(np.float32)
        ds = api.DeviceScene(sc, dev, cell_size=cell, cell_height=cell_h, block_size=block)
        for _ in range(warmup):
            ds.step(1)
        saved = (ds.pos.clone(), ds.vel.clone())
        ts = []
        for _ in range(steps):
            ds.pos.copy_(saved[0])
            ds.vel.copy_(saved[1])
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ds.step(1)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ds.pos.copy_(saved[0])
        ds.vel.copy_(saved[1])
        counters = torch.zeros(N_COUNTERS, dtype=torch.int64, device=dev)
        api.orca_scene_set_counters(ds.handle, counters)
        ds.step(1)
        api.orca_scene_set_counters(ds.handle, None)
        assert ds.sync_status() == 0
        c = counters.cpu().numpy().astype(np.float64) / ds.n
        ds.close()
        out[label] = {"vehicles": int(veh.sum()), "ms_per_step": statistics.median(ts),
                      "per_agent": {"candidates": c[0], "lp_pairs": c[2],
                                    "least_penetration_frac": c[3]}}
    ms = [v["ms_per_step"] for v in out.values()]
    t0 = out["0%"]["ms_per_step"]
    for v in out.values():
        v["vs_people_only"] = v["ms_per_step"] / t0 - 1.0
    return {"workload": "clusters_1m", "shares": out,
            "spread": (max(ms) - min(ms)) / statistics.mean(ms),
            "max_dev_from_people_only": max(abs(v["vs_people_only"]) for v in out.values()),
            "state": f"{warmup} warm-up steps from the initial state, then every timed "
                     f"step from that state"}


def measure_removal(dev, arrive_every=10, reps=3):
    """Removal at goal (Sec. 4) on the 1M-agent cluster scene: every
    ``arrive_every``-th agent has its goal at its own position, so one call of
    orca_scene_remove_arrived flags, scans and compacts all agent arrays.  The
    call synchronises (the host needs the new count); CUDA events bracket it
    on the launching stream, median of ``reps`` calls on fresh scenes."""
    import torch

    from paper_2008_11578_gb300 import api, scenes
    s = scenes.clusters()
    s.goal[::arrive_every] = s.pos[::arrive_every]
    stream = torch.cuda.current_stream()
    ts, kept = [], None
    for _ in range(reps + 1):
        ds = api.DeviceScene(s, dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kept = ds.remove_arrived()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
        ds.close()
    ms = statistics.median(ts[1:])
    n, nk = s.n, len(kept)
    # flags: position, goal, radius read, flag written (20 B per agent); the
    # compaction gathers and writes 38 B per kept agent (two passes)
    alg = 20 * n + 2 * 38 * nk
    hbm = float(_peaks().get("hbm_gbs", 6681.5))
    return {"workload": "clusters_1m", "agents": n, "kept": nk, "ms": ms,
            "bytes": alg, "achieved_gbs": alg / (ms / 1e3) / 1e9,
            "frac": alg / (ms / 1e3) / 1e9 / hbm,
            "kernels": "arrived_kernel, scan kernels, compact_gather_kernel, "
                       "compact_scatter_kernel",
            "note": "one call with its host synchronisation (the new count)"}


def measure_lp_schemes(scene, dev, cell, cell_h, block, pos, vel, steps=5):
    """The per-thread incremental LP against the paper's work-unit batch LP
    (Sec. 3), the warp-cooperative LP and active-set enumeration, same
    workload, launch shape and start state (``pos``/``vel``): median
    solve-kernel time over ``steps`` single steps (all agree to FP32
    rounding)."""
    import torch

    from paper_2008_11578_gb300 import api
    out = {}
    for name, flags in (("per_thread", 0), ("work_units", api.LP_WORK_UNITS),
                        ("warp", api.LP_WARP), ("enumeration", api.LP_ENUMERATION)):
        ds = api.DeviceScene(scene, dev, cell_size=cell, cell_height=cell_h, block_size=block,
                             flags=flags)
        p0, v0 = pos.clone(), vel.clone()
        b, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        api.orca_scene_set_solve_events(ds.handle, b, e)
        ts = []
        for r in range(steps + 1):
            ds.pos.copy_(p0)
            ds.vel.copy_(v0)
            ds.step(1)
            torch.cuda.synchronize()
            if r:
                ts.append(api.event_elapsed_ms(b, e))
        out[name + "_solve_ms"] = statistics.median(ts)
        ds.close()
    out["work_units_over_per_thread"] = out["work_units_solve_ms"] / out["per_thread_solve_ms"]
    out["warp_over_per_thread"] = out["warp_solve_ms"] / out["per_thread_solve_ms"]
    out["enumeration_over_per_thread"] = out["enumeration_solve_ms"] / out["per_thread_solve_ms"]
    return out


def _sm_count(dev):
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def _time_one_step_calls(ds, flush, steps, stream, solve_ev=None, bin_ev=None):
    """Per-call CUDA-event times of ``steps`` one-step calls (L2 flushed
    before each, outside the events); optionally the library's solve and
    binning kernel events of every call."""
    import torch

    from paper_2008_11578_gb300 import api
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        if solve_ev is not None:
            api.orca_scene_set_solve_events(ds.handle, *solve_ev[k])
            api.orca_scene_set_bin_events(ds.handle, *bin_ev[k])
        ev[k][0].record(stream)
        ds.step(1)
        ev[k][1].record(stream)
    return ev


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2008_11578_gb300 import api, autotune, build

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build()
    scene, cfg = _scene(args.workload)
    n = scene.n
    tuned = None
    cell, cell_h, block = args.cell_size, args.cell_height, args.block_size
    if cell is None and not args.no_tune:
        # launch shape only: every candidate computes bit-identical states
        tuned = autotune.tune_scene(scene, dev, steps=3, warmup=1)
        cell_h = tuned.alpha * float(scene.params.cell_size)
        cell = tuned.aspect * cell_h
        block = tuned.block_size
    ds = api.DeviceScene(scene, dev, cell_size=cell, cell_height=cell_h, block_size=block)
    cell_w_m, cell_h_m = float(ds.params.cell_size), float(ds.params.cell_height)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ds.step(1)
    torch.cuda.synchronize()
    assert ds.sync_status() == 0, "non-finite state after warm-up"

    # ---- timed region: K one-step calls, device-resident state ----
    sv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    bv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
        if "CUDA_VISIBLE_DEVICES" in os.environ else local
    barrier()
    with ClockSampler(gpu_index) as clk:
        ev = _time_one_step_calls(ds, flush, args.steps, stream, sv, bv)
        barrier()
    api.orca_scene_set_solve_events(ds.handle, None, None)
    api.orca_scene_set_bin_events(ds.handle, None, None)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    solve_ms = [api.event_elapsed_ms(a, b) for a, b in sv]
    bin_ms = [api.event_elapsed_ms(a, b) for a, b in bv]
    total_s = sum(step_ms) / 1e3
    value, total_max = replica_throughput(total_s, n * args.steps, world, dev)
    clocks = clk.summary()

    # ---- algorithmic FLOPs of the solve kernel (untimed counting step) ----
    counters = torch.zeros(N_COUNTERS, dtype=torch.int64, device=dev)
    saved = (ds.pos.clone(), ds.vel.clone())
    api.orca_scene_set_counters(ds.handle, counters)
    ds.step(1)
    api.orca_scene_set_counters(ds.handle, None)
    ds.pos.copy_(saved[0])
    ds.vel.copy_(saved[1])
    c = counters.cpu().numpy().astype(np.float64)
    flops = FLOPS_CAND * c[0] + FLOPS_LINE * c[1] + FLOPS_PAIR * c[2] + FLOPS_AGENT * c[4]
    prof = _profiled(args.workload) if args.workload == "clusters_1m" else {}
    solve_avg_s = statistics.mean(solve_ms) / 1e3
    sms = _sm_count(dev)
    peaks = _peaks()
    sm_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    peak_tflops = 2 * FP32_LANES * sms * float(sm_mhz) * 1e6 / 1e12
    achieved = flops / solve_avg_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops,
                "traffic": prof.get("traffic_bytes_per_launch"),
                # why the fraction is small (same ncu capture, null when stale):
                # issue slots busy, and active lanes per issued instruction
                "ncu_issue_active_pct": prof.get("issue_active_pct"),
                "ncu_simt_efficiency_pct": prof.get("simt_efficiency_pct"),
                # the issue-slot ceiling: warp instructions of one launch (same
                # capture) over the live launch time, against one instruction
                # per scheduler per cycle (4 per SM)
                "issue": None if "warp_instructions_per_launch" not in prof else {
                    "achieved_warp_inst_per_s":
                        prof["warp_instructions_per_launch"] / solve_avg_s,
                    "peak_warp_inst_per_s": 4.0 * sms * float(sm_mhz) * 1e6,
                    "frac": prof["warp_instructions_per_launch"] / solve_avg_s
                            / (4.0 * sms * float(sm_mhz) * 1e6)},
                "kernel": "solve_kernel", "solve_ms": statistics.mean(solve_ms),
                "solve_share_of_step": statistics.mean(solve_ms) / statistics.mean(step_ms),
                "flops_per_agent_step": flops / n,
                "counts_per_agent": {"candidates": c[0] / n, "neighbours": c[1] / n,
                                     "lp_pairs": c[2] / n, "fallback_frac": c[3] / n,
                                     "klist_admissions": c[9] / n, "klist_shifts": c[10] / n,
                                     "rows_scanned": c[11] / n, "row_loop_iterations": c[12] / n},
                # share of a solve thread's clock cycles in each phase (counting
                # variant, stalls included)
                "phase_split": {"search": c[5] / c[8], "half_planes": c[6] / c[8],
                                "lp": c[7] / c[8], "rest": 1.0 - (c[5] + c[6] + c[7]) / c[8]},
                "peak_source": f"FP32 FMA: {sms} SMs (queried) x {FP32_LANES} lanes x 2 x "
                               f"{sm_mhz:.0f} MHz (maximum SM clock, nvidia-smi)"}

    # ---- binning kernel: HBM bound ----
    ncells = int(ds.params.grid_nx) * int(ds.params.grid_ny)
    hbm = float(peaks.get("hbm_gbs", 6681.5))
    bin_s = statistics.mean(bin_ms) / 1e3

    # DRAM bytes of a first-step binning launch from the committed capture
    # (same workload and launch shape), while the sources match it
    bin_traffic = (_profiled(args.workload, "bin_kernel").get("traffic_bytes_per_launch")
                   if args.workload == "clusters_1m" else None)

    def bin_roof(sec, kernel_bytes_agent, first):
        method_bytes = BIN_BYTES_METHOD * n
        kernel_bytes = kernel_bytes_agent * n + BIN_BYTES_CELL * ncells
        return {"bound": "hbm", "achieved": method_bytes / sec / 1e9, "peak": hbm,
                "unit": "GB/s", "frac": method_bytes / sec / 1e9 / hbm,
                "traffic": bin_traffic if first else None,
                "kernels": "bin_kernel (cooperative: cell keys, scan, cell order, order by x)",
                "ms": 1e3 * sec, "bytes_per_step": method_bytes,
                "bytes_basis": f"{BIN_BYTES_METHOD} B per agent (the method's per-unit figure)",
                "kernel_bytes_per_step": kernel_bytes,
                "kernel_frac": kernel_bytes / sec / 1e9 / hbm,
                "cells": ncells, "cell_bytes": BIN_BYTES_CELL * ncells,
                "first_step_of_call": first, "launches_per_step": 1,
                "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"}
    roofline_binning = bin_roof(bin_s, BIN_BYTES_KERNEL_FIRST, True)

    # later steps of one multi-step call (no cell-key phase; the previous
    # step's state is read in nearly sorted order): the last binning kernel
    # of a 4-step call, L2 flushed before the call only
    later = []
    bb, be = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        ds.pos.copy_(saved[0])
        ds.vel.copy_(saved[1])
        flush.zero_()
        api.orca_scene_set_bin_events(ds.handle, bb, be)
        ds.step(4)
        api.orca_scene_set_bin_events(ds.handle, None, None)
        torch.cuda.synchronize()
        later.append(api.event_elapsed_ms(bb, be))
    ds.pos.copy_(saved[0])
    ds.vel.copy_(saved[1])
    roofline_binning_steady = bin_roof(statistics.median(later) / 1e3, BIN_BYTES_KERNEL_LATER,
                                       False)
    roofline_binning_steady["note"] = ("4th step of a 4-step call, median of 3; L2 is flushed "
                                       "before the call, not between its steps")

    # ---- end to end through the public API from pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        # the caller's state as one pinned host block (positions then
        # velocities), the layout of the scene's device state: one copy each way
        hs = torch.empty((2, n, 2), dtype=torch.float32, pin_memory=True)
        os_ = torch.empty((2, n, 2), dtype=torch.float32, pin_memory=True)
        hs.copy_(ds.state)
        eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        for k in range(args.steps):
            flush.zero_()
            eev[k][0].record(stream)
            ds.state.copy_(hs, non_blocking=True)
            ds.step(1)
            os_.copy_(ds.state, non_blocking=True)
            eev[k][1].record(stream)
        barrier()
        e_total = sum(a.elapsed_time(b) for a, b in eev) / 1e3
        e2e = {"value": replica_throughput(e_total, n * args.steps, world, dev)[0],
               "unit": METRIC,
               "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 2 * 8 * n}

    status = ds.sync_status()
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": dict(cfg, l2="flushed before every timed step (256 MB write)",
                           parallelism=f"replicas{world}" if world > 1 else "single",
                           cell_w_m=cell_w_m, cell_h_m=cell_h_m,
                           solve_block=int(ds.params.block_size) or 128,
                           autotune=None if tuned is None else
                           [[a * float(scene.params.cell_size), asp, bs, ms]
                            for a, asp, bs, ms in tuned.table],
                           autotune_columns=["cell_h_m", "aspect", "block", "ms_per_step"],
                           neighbor_dist_m=10.0, max_neighbors=10, tau_s=5.0, dt_s=0.25),
            "clocks": clocks, "gpu_launches": ds.launch_count(1) * args.steps,
            "roofline": roofline, "roofline_binning": roofline_binning,
            "roofline_binning_steady": roofline_binning_steady, "e2e": e2e,
            "status": status, "hbm_peak_gbs": peaks.get("hbm_gbs"), "sms": sms}
    if not args.no_ablation:
        line["lp_scheme_ablation"] = dict(
            measure_lp_schemes(scene, dev, cell_w_m, cell_h_m, int(ds.params.block_size),
                               ds.pos, ds.vel),
            workload=cfg["workload"],
            state=f"after the {args.warmup + args.steps} warm-up and timed steps")
    if not args.no_vehicle_share and args.workload == "clusters_1m":
        line["vehicle_share_sweep"] = measure_vehicle_share(dev, flush, cell_w_m, cell_h_m,
                                                            int(ds.params.block_size))
    if not args.no_batched:
        line["batched"] = measure_batched(dev, flush)
    if not args.no_adjoint:
        line["adjoint"] = measure_adjoint(dev)
    if not args.no_removal:
        line["removal"] = measure_removal(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # one more GPU step from the current state, with its neighbour lists,
        # for the parity statistics of the oracle sample timed below
        ref = scene.copy()
        ref.pos, ref.vel = ds.pos.cpu().numpy(), ds.vel.cpu().numpy()
        ds.enable_debug()
        ds.step(1)
        torch.cuda.synchronize()
        gpu = dict(pos=ds.pos.cpu().numpy(), vel=ds.vel.cpu().numpy(),
                   **{k: v.cpu().numpy() for k, v in ds.dbg.items()})
        api.orca_scene_set_debug(ds.handle)
        ds.dbg = None
        line["cpu_baseline"], line["parity"] = cpu_baseline(ref, cfg, gpu)
    tg = {"agent_steps_per_s": {"target": 5e8, "value": value, "met": value >= 5e8},
          "binning_hbm_frac": {"target": 0.5, "value": roofline_binning["frac"],
                               "steady": roofline_binning_steady["frac"],
                               "met": roofline_binning["frac"] >= 0.5}}
    if "batched" in line:
        sp = line["batched"]["speedup_vs_plain_loop"]
        tg["batched_over_plain_loop"] = {"target": 3.0, "value": sp, "met": sp >= 3.0}
    if "adjoint" in line:
        r_ = line["adjoint"]["adjoint_over_forward"]
        tg["adjoint_over_forward"] = {"target": 3.0, "value": r_, "met": r_ <= 3.0}
    if line.get("parity"):
        pr = line["parity"]
        tg["velocity_parity_m_s"] = {"target": 1e-4, "value": pr["max_dv_m_s"],
                                     "met": pr["max_dv_m_s"] <= 1e-4}
        tg["position_parity_m"] = {"target": 1e-5, "value": pr["max_dp_beyond_half_ulp_m"],
                                   "met": pr["max_dp_beyond_half_ulp_m"] <= 1e-5}
    line["targets"] = tg
    if rank == 0:
        print(json.dumps(line), flush=True)
    ds.close()
    if world > 1:
        dist.destroy_process_group()


def run_only(args):
    import torch

    from paper_2008_11578_gb300 import build
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build()
    if args.only == "adjoint":
        out = measure_adjoint(dev)
    elif args.only == "batched":
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        out = measure_batched(dev, flush, tune=not args.no_tune)
    else:
        out = measure_removal(dev)
    print(json.dumps({args.only: out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clusters_1m")
    ap.add_argument("--cell-size", type=float, default=None,
                    help="cell width in m (skips the autotuner)")
    ap.add_argument("--cell-height", type=float, default=None,
                    help="cell height in m with --cell-size (default: square)")
    ap.add_argument("--block-size", type=int, default=0,
                    help="solve block size with --cell-size (0: the library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-vehicle-share", action="store_true")
    ap.add_argument("--no-removal", action="store_true")
    ap.add_argument("--only", choices=["adjoint", "batched", "removal"], default=None,
                    help="run one secondary measurement alone (for profiling); prints "
                         "its JSON object, not the benchmark line")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
