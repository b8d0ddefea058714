"""Benchmark of the flock environment step on GB300.

Default (one GPU): the plain single-instance step at 50,000 agents (side
707.1, density 0.1, view radius 5, 8 sectors, field of view 250 degrees,
uniform random actions), W warm-up steps then K timed steps, each timed with
CUDA events on the library's stream, with L2 flushed (a 512 MiB write)
between timed steps.  Prints one JSON line: agent-steps/s, p50/p99 step
latency, the roofline of the dominant kernel (the neighbour scan), the same
metric end to end through host buffers, GPU clocks sampled during the timed
region, and the CPU oracle timed on this host as a reported baseline.

--gpus N (under torchrun): every rank runs its own 50,000-agent instance
(instances are independent, no collective on the data path); the value is
the agent-steps of all ranks over the slowest rank's time.

--impl reference: times the CPU oracle (the reference arm of this project:
the plain O(N^2) statement of the step) on this host's cores."""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import flock_inputs as fi  # noqa: E402

METRIC = "flock agent-steps/sec at 50k agents, batched vs plain; p99 step latency"
UNIT = "agent-steps/s"
N_AGENTS = 50000
# the headline workload, the same words in both arms' config
PLAIN_WORKLOAD = ("plain flock step, 1 instance, %d agents, side %.1f, density 0.1, view radius "
                  "5, 8 sectors, fov 250 deg, uniform random actions")
BYTES_PER_AGENT_STEP = 116  # state in 16 + action 4 + state out 16 + obs 72 + reward 4 + coll 4
# neighbour scan: reads the agent's sorted position (8), heading and speed (8)
# and index (4); writes its observation (72), reward (4) and collisions (4)
NEIGH_BYTES_PER_AGENT = 100
# DRAM traffic per launch from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum), valid while the kernel sources are unchanged
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
CSRC = os.path.join(ROOT, "paper_2207_03945_gb300", "csrc")


def _code_only(text: str) -> str:
    """C/C++ source without comments and blank lines (comment edits do not
    change a kernel)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def sources_digest() -> str:
    """SHA-256 over the code (comments removed) of the kernel sources and the
    public header."""
    import hashlib
    h = hashlib.sha256()
    files = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h")))
    paths = [(f, os.path.join(CSRC, f)) for f in files]
    paths.append(("flock.h", os.path.join(ROOT, "include", "flock.h")))
    for name, path in paths:
        with open(path, encoding="utf-8") as fh:
            h.update(name.encode() + b"\0" + _code_only(fh.read()).encode())
    return h.hexdigest()


def batch_traffic(key: str, mode: int):
    """DRAM bytes of one batched step from the committed table: the sum over
    the step's kernels in that form (None unless all are in the table)."""
    kernels = {2: ["k_batch_step"], 3: ["k_batch_step", "k_batch_neigh"],
               4: ["k_bbin_apply", "k_bbin_scan", "k_bbin_scatter", "k_batch_neigh"]}
    vals = [measured_traffic(k, key) for k in kernels.get(mode, [])]
    return None if not vals or any(v is None for v in vals) else sum(vals)


def pair_counts(params: dict, state, stencil: int = 1):
    """(candidate tests, in-range pairs) of one step of the square at these
    positions: candidates are the other agents in each agent's stencil cells
    (the library's cell list), pairs the ordered pairs closer than the view
    radius (counted in float64: a throughput figure, not a parity check)."""
    from scipy.spatial import cKDTree
    import paper_2207_03945_gb300 as F
    d = F.flock_derive(params, {"stencil": stencil})
    nc, h, invw = int(d["cells_per_side"]), int(d["stencil"]), np.float32(d["inv_cell_width"])
    xy = np.asarray(state, dtype=np.float32)[:, :2]
    cells = np.clip((xy * invw).astype(np.int64), 0, nc - 1)
    grid = np.zeros((nc, nc), np.int64)
    np.add.at(grid, (cells[:, 1], cells[:, 0]), 1)
    box = np.zeros_like(grid)
    for dy in range(-h, h + 1):
        for dx in range(-h, h + 1):
            box += np.roll(np.roll(grid, dy, axis=0), dx, axis=1)
    cand = int(box[cells[:, 1], cells[:, 0]].sum()) - len(xy)
    L = float(params["side"])
    tree = cKDTree(np.mod(xy.astype(np.float64), L), boxsize=L)
    pairs = int(tree.count_neighbors(tree, float(params["view_radius"]))) - len(xy)
    return cand, pairs


def tuning_tag(t: dict) -> str:
    """Short name of a launch shape, e.g. m2-s1-b128-l2."""
    tag = "m%d-s%d-b%d" % (t["mode"], t["stencil"], t["block"])
    if t["mode"] == 1:
        return tag + "-t%dx%d" % (t["tile_w"], t["tile_h"])
    return tag + "-l%d" % t.get("lanes", 1)


def measured_traffic(kernel: str, workload: str):
    """Bytes per launch of `kernel` on `workload` from the committed ncu
    table, or None when there is no entry or the sources changed since."""
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    digest = sources_digest()
    for ln in lines:
        if not ln.strip() or ln.startswith("#"):
            continue
        f = [x.strip() for x in ln.split("|")]
        if len(f) >= 5 and f[0] == kernel and f[1] == workload and f[4] == digest:
            return int(f[2]) + int(f[3])
    return None


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device=None) -> float:
    """Largest x over the ranks of the default process group (x itself when
    there is none).  NCCL needs a device tensor, gloo a host one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of x over the ranks of the default process group (x itself when
    there is none); a reporting reduction, outside any timed region."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def weak_scaling_value(world: int, agents_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job agent-steps per second: every rank advanced its own
    agents_per_rank agents `steps` times; the job took the slowest rank's time."""
    return world * agents_per_rank * steps / (max_ms * 1e-3)


def rank_seed(rank: int) -> int:
    """Seed of a rank's replica: ranks run independent instances."""
    return 1000 * rank


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n=N_AGENTS, steps=2, seed=0):
    """The oracle, as it stands, on this host's cores: full O(N^2) steps of
    the same workload (a bounded sample of `steps` steps)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    side = fi.side_for(n)
    p = fi.default_params(side)
    st = fi.initial_state(n, side, seed)
    acts = fi.random_actions(n, steps, seed)
    cores = os.cpu_count() or 1
    oracle.step(p, st, None, threads=cores)  # page in / warm
    t0 = time.perf_counter()
    for a in acts:
        st = oracle.step(p, st, a, threads=cores)[0]
    dt = time.perf_counter() - t0
    return {"value": n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d full O(N^2) steps of the %d-agent workload (seed %d), %d OpenMP threads"
                      % (steps, n, seed, cores), "seconds": dt}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on all host cores.  Each
    step applies the actions of all agents and observes a bounded sample of
    them (rotating through the agents), sized so that the whole run takes
    about two minutes; the rate is sampled agent-steps per second."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    n = N_AGENTS
    side = fi.side_for(n)
    p = fi.default_params(side)
    st = fi.initial_state(n, side, 0)
    total = args.steps + args.warmup
    acts = fi.random_actions(n, total, 0)
    cores = os.cpu_count() or 1
    # size the per-step sample from one probe of 512 rows
    probe = np.arange(512, dtype=np.int32)
    t0 = time.perf_counter()
    oracle.observe_rows(p, st, probe, threads=cores)
    per_row = (time.perf_counter() - t0) / len(probe)
    budget = 120.0 / max(total, 1)
    m = int(max(256, min(n, budget / max(per_row, 1e-9))))
    times = []
    off = 0
    for k in range(total):
        rows = (np.arange(m, dtype=np.int64) + off) % n
        off = (off + m) % n
        t0 = time.perf_counter()
        st, _ = oracle.apply(p, st, acts[k])
        oracle.observe_rows(p, st, rows.astype(np.int32), threads=cores)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = m * len(times) / tot
    sample = ("each step: actions applied to all %d agents, observation of %d of them "
              "(rotating), O(N) candidates per observed agent, %d OpenMP threads" % (n, m, cores))
    line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": PLAIN_WORKLOAD % (n, fi.side_for(n)),
                       "agents": n, "parallelism": "single",
                       "form": "CPU oracle (O(N^2) per observed agent), sampled rows"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


BATCH_FORMS = {2: "every phase in one persistent cooperative kernel",
               3: "binning in a persistent cooperative kernel, then the neighbour launch",
               4: "binning by three kernels (apply and count, scan, scatter), then the "
                  "neighbour launch"}
BATCH_KERNELS = {2: "k_batch_step", 3: "k_batch_step + k_batch_neigh",
                 4: "k_bbin_apply + k_bbin_scan + k_bbin_scatter + k_batch_neigh"}


def run_batched(F, torch, dev, stream, steps, warmup, flush, seed=0, n_inst=256, sizes=None,
                world=1, tune=True, tuning=None):
    """The batched form: n_inst instances with agent counts log-uniform in
    [100, 20000] (density 0.1 each), all advanced by one persistent kernel
    per step, replayed from a CUDA graph.  With `sizes`, those instances
    instead.  Returns a dict for the JSON line."""
    mix = sizes is None
    if mix:
        sizes = fi.batch_sizes(n_inst, 100, 20000, seed)
    n_inst = len(sizes)
    params = [fi.default_params(fi.side_for(n)) for n in sizes]
    total = sum(sizes)
    cells = sum(F.flock_instance_cells(p) for p in params)
    arena = torch.empty((total, 4), dtype=torch.float32, device=dev)
    states, off = [], 0
    for k, n in enumerate(sizes):
        arena[off:off + n] = torch.from_numpy(fi.initial_state(n, fi.side_for(n), seed + k))
        states.append(arena[off:off + n])
        off += n
    if tune and tuning is None:
        from paper_2207_03945_gb300.autotune import autotune_batch
        host_states = [s_.cpu().numpy() for s_ in states]
        tuning, _ = autotune_batch(params, sizes, host_states, device=dev)
    cells = sum(F.flock_instance_cells(p, tuning) for p in params)
    b = F.FlockBatch(n_inst, total, cells, 18, device=dev, stream=stream, tuning=tuning)
    b.set(params, sizes, states, reset=[1] * n_inst)
    acts = torch.from_numpy(fi.random_actions(total, steps + warmup + 1, seed + 1)).to(dev)
    act_buf = torch.empty(total, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        act_buf.copy_(acts[0])
        b.step(act_buf)  # initial observation (reset)
        for k in range(warmup):
            act_buf.copy_(acts[1 + k])
            flush.zero_()
            b.step(act_buf)
    torch.cuda.synchronize()
    for k in range(steps):
        with torch.cuda.stream(stream):
            act_buf.copy_(acts[1 + warmup + k])
            flush.zero_()
            ev0[k].record(stream)
            b.step(act_buf)
            ev1[k].record(stream)
    torch.cuda.synchronize()
    # kernel duration from events recorded inside the step graph
    F.env_batch_set_timing(b.batch, True)
    kern = []
    for k in range(steps):
        with torch.cuda.stream(stream):
            act_buf.copy_(acts[1 + warmup + k])
            flush.zero_()
            b.step(act_buf)
        kern.append(F.env_batch_get_time(b.batch))
    F.env_batch_set_timing(b.batch, False)
    torch.cuda.synchronize()
    err = b.error()
    assert err == 0, "device error bits %d" % err
    ms = [ev0[k].elapsed_time(ev1[k]) for k in range(steps)]
    tot = max_over_ranks(sum(ms), dev)
    grid, block = F.env_batch_get_launch(b.batch)
    bmode = (tuning or {}).get("mode", 4) or 4  # the library's default form is 4
    traffic_key = "batched-%d-%d-s%d-m%d" % (n_inst, total, (tuning or {}).get("stencil", 1), bmode)
    kern_ms = float(np.mean(kern))
    peak, peak_kind = peaks()
    achieved = BYTES_PER_AGENT_STEP * total / (kern_ms * 1e-3) / 1e9
    b.close()
    return {"value": weak_scaling_value(world, total, steps, tot), "unit": UNIT,
            "instances": n_inst, "agents": total, "cells": cells, "ms_per_step": tot / steps,
            "tuning": tuning,
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "grid": grid, "block": block,
            "workload": "batched: %d flock instances, agent counts %s (seed %d, %d agents), "
                        "density 0.1, view radius 5, 8 sectors, fov 250 deg, %s, one CUDA "
                        "graph per step"
                        % (n_inst, "log-uniform in [100, 20000]" if mix else
                           "%d x %d" % (n_inst, sizes[0]) if len(set(sizes)) == 1 else str(sizes),
                           seed, total, BATCH_FORMS.get(bmode, "form %d" % bmode)),
            "roofline": {"bound": "hbm",
                         "kernel": BATCH_KERNELS.get(bmode, "batch"),
                         "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_kind,
                         "traffic": batch_traffic(traffic_key, bmode),
                         "bytes_per_agent": BYTES_PER_AGENT_STEP}}


def run_plain(F, torch, dev, stream, n, steps, warmup, flush, seed=0, world=1, what=""):
    """The plain single-instance step at n agents (density 0.1, side
    sqrt(n / 0.1), the defaults): `steps` consecutive steps of uniform random
    actions, each timed with CUDA events on the library's stream, L2 flushed
    between steps.  Returns agent-steps/s and p50/p99 step latency."""
    side = fi.side_for(n)
    p = fi.default_params(side)
    env = F.FlockEnv(p, n, device=dev, stream=stream)
    acts = torch.from_numpy(fi.random_actions(n, steps + warmup, seed)).to(dev)
    act_buf = torch.empty(n, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        env.reset(torch.from_numpy(fi.initial_state(n, side, seed)).to(dev))
        for k in range(warmup):
            act_buf.copy_(acts[k])
            flush.zero_()
            env.step(act_buf)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            act_buf.copy_(acts[warmup + k])
            flush.zero_()
            ev0[k].record(stream)
            env.step(act_buf)
            ev1[k].record(stream)
    torch.cuda.synchronize()
    assert env.error() == 0
    tun = env.tuning()
    env.close()
    ms = [ev0[k].elapsed_time(ev1[k]) for k in range(steps)]
    tot = max_over_ranks(sum(ms), dev)
    return {"value": weak_scaling_value(world, n, steps, tot), "unit": UNIT, "agents": n,
            "steps": steps, "ms_per_step": tot / steps, "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "tuning": tun,
            "workload": "plain flock step%s: %d agents, side %.1f, density 0.1, view radius 5, "
                        "8 sectors, fov 250 deg, uniform random actions, seed %d, %d steps, "
                        "L2 flushed between steps" % (what, n, side, seed, steps)}


POLICY_BYTES_PER_AGENT = 48  # state 16 in + 16 out, action 4 in + 4 out, reward 4, coll 4


def run_policy(F, torch, dev, stream, steps, warmup, flush, n=100000, seed=0, world=1):
    """Step + fused policy at 100,000 agents (side 1000): the greedy actions
    of each step drive the next; observations stay on chip."""
    side = fi.side_for(n)
    p = fi.default_params(side)
    env = F.FlockEnv(p, n, device=dev, stream=stream)
    w = fi.policy_weights(seed)
    blob = torch.from_numpy(w["blob"].view(np.int16)).to(dev)
    act = torch.from_numpy(fi.random_actions(n, 1, seed)[0]).to(dev)
    rew = torch.empty(n, dtype=torch.float32, device=dev)
    coll = torch.empty(n, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        env.reset(torch.from_numpy(fi.initial_state(n, side, seed)).to(dev))
        for _ in range(warmup):
            flush.zero_()
            F.env_step_policy(env.env, blob, act, rew, coll)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev0[k].record(stream)
            F.env_step_policy(env.env, blob, act, rew, coll)
            ev1[k].record(stream)
    torch.cuda.synchronize()
    assert env.error() == 0
    ms = [ev0[k].elapsed_time(ev1[k]) for k in range(steps)]
    tot = max_over_ranks(sum(ms), dev)
    # second pass: events between the step's kernels give each one's time
    F.env_set_timing(env.env, True)
    phase = []
    for k in range(min(steps, 20)):
        with torch.cuda.stream(stream):
            flush.zero_()
            F.env_step_policy(env.env, blob, act, rew, coll)
        phase.append(F.env_get_phase_times(env.env))
    F.env_set_timing(env.env, False)
    ph = np.array(phase).mean(axis=0)
    env.close()
    peak, peak_kind = peaks()
    achieved = POLICY_BYTES_PER_AGENT * n / (tot / steps * 1e-3) / 1e9
    return {"value": weak_scaling_value(world, n, steps, tot), "unit": UNIT, "agents": n,
            "ms_per_step": tot / steps, "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)),
            "workload": "step + fused policy: %d agents, side %.0f, MLP 18-64-64-9 tanh, BF16 "
                        "weights N(0, 0.1) and activations on tensor cores (mma.sync), FP32 "
                        "accumulate, greedy actions feed the next step" % (n, side),
            "kernel_ms": {"apply_bin_and_weight_image": float(ph[0]), "scan": float(ph[1]),
                          "scatter": float(ph[2]), "neighbours_and_network": float(ph[3])},
            "roofline": {"bound": "hbm", "kernel": "whole step (4 kernels; the network runs "
                                                   "in the neighbour scan's epilogue)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": None,  # a whole-step figure; see profiles/ for the kernel
                         "bytes_per_agent": POLICY_BYTES_PER_AGENT}}


def run_paper_variant(F, torch, dev, stream, steps, warmup, flush, n=16000, seed=0, world=1):
    """The paper's own flock (Section 4.1, Section 5): 16,000 agents (its
    largest flock run), 128 sectors, view a tenth of the side (side 400, view
    40: about 500 neighbours in range), field of view 250 degrees, continuous
    (acceleration, rotation) actions, the 129-value view-only observation."""
    p = fi.paper_params(n)
    env = F.FlockEnv(p, n, device=dev, stream=stream)
    acts = torch.from_numpy(fi.random_cont_actions(n, steps + warmup, seed, p["speed_step"],
                                                   p["turn_step"])).to(dev)
    act_buf = torch.empty((n, 2), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        env.reset(torch.from_numpy(fi.initial_state(n, p["side"], seed)).to(dev))
        for k in range(warmup):
            act_buf.copy_(acts[k])
            flush.zero_()
            env.step_continuous(act_buf)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            act_buf.copy_(acts[warmup + k])
            flush.zero_()
            ev0[k].record(stream)
            env.step_continuous(act_buf)
            ev1[k].record(stream)
    torch.cuda.synchronize()
    assert env.error() == 0
    tun = env.tuning()
    cand, pairs = pair_counts(p, env.state().cpu().numpy(), tun["stencil"])
    env.close()
    ms = [ev0[k].elapsed_time(ev1[k]) for k in range(steps)]
    tot = max_over_ranks(sum(ms), dev)
    peak, peak_kind = peaks()
    v = int(p["num_segments"])
    bpa = 16 + 8 + 16 + 4 * (v + 1) + 4 + 4  # state in, action, state out, obs, reward, coll
    achieved = bpa * n / (tot / steps * 1e-3) / 1e9
    return {"value": weak_scaling_value(world, n, steps, tot), "unit": UNIT, "agents": n,
            "ms_per_step": tot / steps, "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "tuning": tun,
            "workload": "the paper's flock: %d agents, side %.0f, view %.0f (a tenth of the "
                        "side), 128 sectors, fov 250 deg, continuous (acceleration, rotation) "
                        "actions, observation 128 distances + speed" % (n, p["side"],
                                                                         p["view_radius"]),
            "pairs": pair_rates(cand, pairs, n, tot / steps),
            "roofline": {"bound": "hbm", "kernel": "whole step (4 kernels)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": None, "bytes_per_agent": bpa}}


def pair_rates(cand: int, pairs: int, n: int, ms_per_step: float):
    """Pair throughput of a pair-bound workload (a view of hundreds of
    neighbours): candidate tests and in-range pairs per second and per
    agent, at the step time given."""
    s_ = ms_per_step * 1e-3
    return {"candidate_tests_per_s": cand / s_, "in_range_pairs_per_s": pairs / s_,
            "candidates_per_agent": cand / max(n, 1), "in_range_per_agent": pairs / max(n, 1),
            "counted": "at the last timed step's positions; pairs closer than the view radius "
                       "(float64)"}


def run_tag(F, torch, dev, stream, steps, warmup, flush, n=17600, seed=0, world=1):
    """The tag environment at the paper's size (Section 4.2, Section 5: 16,000
    runners and 1,600 chasers): two colour channels of 64 sectors, view a
    tenth of the side, (speed, rotation) actions."""
    p = fi.tag_params(n)
    env = F.FlockEnv(p, n, device=dev, stream=stream)
    acts = torch.from_numpy(fi.tag_actions(n, steps + warmup, seed, p["speed_max"],
                                           p["turn_step"])).to(dev)
    act_buf = torch.empty((n, 2), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        env.set_types(torch.from_numpy(fi.tag_types(n, seed)).to(dev))
        env.reset(torch.from_numpy(fi.initial_state(n, p["side"], seed)).to(dev))
        for k in range(warmup):
            act_buf.copy_(acts[k])
            flush.zero_()
            env.step_continuous(act_buf)
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            act_buf.copy_(acts[warmup + k])
            flush.zero_()
            ev0[k].record(stream)
            env.step_continuous(act_buf)
            ev1[k].record(stream)
    torch.cuda.synchronize()
    assert env.error() == 0
    tun = env.tuning()
    cand, pairs = pair_counts(p, env.state().cpu().numpy(), tun["stencil"])
    env.close()
    ms = [ev0[k].elapsed_time(ev1[k]) for k in range(steps)]
    tot = max_over_ranks(sum(ms), dev)
    return {"value": weak_scaling_value(world, n, steps, tot), "unit": UNIT, "agents": n,
            "pairs": pair_rates(cand, pairs, n, tot / steps),
            "chasers": int(round(0.1 * n)), "ms_per_step": tot / steps,
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "tuning": tun,
            "workload": "tag: %d agents (a tenth chasers), side %.0f, view %.0f, 2 x 64 sectors, "
                        "fov 250 deg, (speed, rotation) actions" % (n, p["side"],
                                                                    p["view_radius"])}


def run_rollout(F, torch, dev, stream, reps, flush, n=16000, T=128, seed=0, world=1):
    """One training step's experience collection of the paper (Section 5:
    t = 128 environment updates of all agents), as a single graph launch of
    128 steps of the paper's flock (16,000 agents, continuous actions), then
    the advantages over the 128 x 16,000 trajectory (generalised advantage
    estimation, gamma 0.99, lambda 0.95) with seeded values standing in for
    the critic."""
    p = fi.paper_params(n)
    env = F.FlockEnv(p, n, device=dev, stream=stream)
    acts = torch.from_numpy(fi.random_cont_actions(n, T, seed, p["speed_step"],
                                                   p["turn_step"])).to(dev)
    obs = torch.empty((T, n, env.obs_dim), dtype=torch.float32, device=dev)
    rew = torch.empty((T, n), dtype=torch.float32, device=dev)
    coll = torch.empty((T, n), dtype=torch.int32, device=dev)
    val = torch.from_numpy(np.random.Generator(np.random.PCG64(seed + 5)).normal(
        0.0, 1.0, (T + 1, n)).astype(np.float32)).to(dev)
    adv = torch.empty((T, n), dtype=torch.float32, device=dev)
    ret = torch.empty((T, n), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        env.reset(torch.from_numpy(fi.initial_state(n, p["side"], seed)).to(dev))
        F.env_rollout(env.env, None, obs, rew, coll, actions2=acts)  # warm-up, graph capture
        F.flock_gae(rew, val, 0.99, 0.95, adv, ret, stream=stream)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
    for k in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
            F.env_rollout(env.env, None, obs, rew, coll, actions2=acts)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    # the advantage kernel timed on its own, each run after an L2 flush
    gae_ms = []
    for k in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            F.flock_gae(rew, val, 0.99, 0.95, adv, ret, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        gae_ms.append(e0.elapsed_time(e1))
    assert env.error() == 0
    env.close()
    roll_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(reps)]
    tot = max_over_ranks(sum(roll_ms), dev)
    g_ms = float(np.mean(gae_ms))
    peak, peak_kind = peaks()
    gae_bytes = 16 * T * n + 4 * n  # reward and value in, advantage and target out
    return {"value": weak_scaling_value(world, n * T, reps, tot), "unit": UNIT,
            "agents": n, "steps_per_rollout": T, "ms_per_rollout": tot / reps,
            "launches_per_rollout": 4 * T,
            "workload": "rollout of the paper's flock: %d agents x %d steps in one graph "
                        "launch (continuous actions, 128 sectors, view a tenth of the side), "
                        "outputs kept for every step" % (n, T),
            "gae": {"ms": g_ms, "elements": T * n, "gamma": 0.99, "lambda": 0.95,
                    "roofline": {"bound": "hbm", "kernel": "k_gae",
                                 "achieved": gae_bytes / (g_ms * 1e-3) / 1e9, "peak": peak,
                                 "unit": "GB/s",
                                 "frac": gae_bytes / (g_ms * 1e-3) / 1e9 / peak,
                                 "peak_source": peak_kind, "traffic": None,
                                 "bytes_per_element": 16}}}


def device_initial_state(dev):
    """Clients' initial states drawn on the device from each session's seed by
    the library's flock_seed_states: x, y ~ U[0, side), theta ~ U[0, 2 pi),
    speed 0.5 (the distribution of flock_inputs.initial_state), one launch."""
    import torch
    import paper_2207_03945_gb300 as F

    def fn(s):
        st = torch.empty((s.n, 4), dtype=torch.float32, device=dev)
        F.flock_seed_states(st, float(s.params["side"]), int(s.seed), 0.5)
        return st
    return fn


def bare_set_rate(dev, sessions, max_instances, max_agents, max_cells, steps=100, warmup=5):
    """Agent-steps/s of the batched kernels alone on the given serving
    sessions' instances: one batch of them with the serving loop's capacities
    and default launch shape, uniform random actions drawn on the device each
    step as the loop draws them, `steps` steps back to back timed with CUDA
    events."""
    import torch
    import paper_2207_03945_gb300 as F
    sizes = [s.n for s in sessions]
    params = [s.params for s in sessions]
    total = sum(sizes)
    cells = sum(F.flock_instance_cells(p) for p in params)
    b = F.FlockBatch(max_instances, max_agents, max_cells, 18, device=dev)
    init = device_initial_state(dev)
    arena = torch.empty((total, 4), dtype=torch.float32, device=dev)
    views, off = [], 0
    for s_ in sessions:
        arena[off:off + s_.n] = init(s_)
        views.append(arena[off:off + s_.n])
        off += s_.n
    b.set(params, sizes, views, reset=[1] * len(sizes))
    acts = torch.empty(total, dtype=torch.int32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(12345)
    for _ in range(warmup):
        acts.random_(0, 9, generator=gen)
        b.step(acts)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        acts.random_(0, 9, generator=gen)
        b.step(acts)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    err = b.error()
    assert err == 0, "device error bits %d" % err
    b.close()
    return {"agent_steps_per_s": total * steps / (ms * 1e-3), "agents": total,
            "instances": len(sizes), "ms_per_step": ms / steps, "steps": steps}


def run_serving(dev, seconds, seed=0, rate=50.0, budget=100 * 10 ** 9, backlog=0, rank=0,
                world=1):
    """Serving loop with continuous batching: Poisson session arrivals, agent
    counts log-uniform in [500, 50000], episodes of 100..2000 steps, admission
    by a device-memory budget, all admitted sessions stepped together by the
    batched kernel each iteration.  backlog > 0 adds that many sessions at
    t = 0 (saturation).  With several ranks (one GPU each) the job's single
    arrival stream is placed across them on the host (serve.place_sessions,
    the same on every rank, no exchange) and each rank serves its share; the
    rate is the job's agent-steps over the slowest rank's time."""
    from paper_2207_03945_gb300 import serve
    arrivals = fi.session_stream(rate, seconds, seed)
    if backlog:
        rng = np.random.Generator(np.random.PCG64(seed + 99))
        for k in range(backlog):
            n = int(round(math.exp(math.log(500) + rng.random() * (math.log(50000) - math.log(500)))))
            arrivals.append((0.0, n, int(rng.integers(100, 2001)), 10 ** 6 + k))
    arrivals = sorted(arrivals)
    offered = len(arrivals)
    if world > 1:
        ranks = serve.place_sessions(arrivals, world)
        arrivals = [a for a, r in zip(arrivals, ranks) if r == rank]
    caps = {"max_slots": 512, "arena_agents": 8_000_000, "max_cells": 4_000_000}
    srv = serve.FlockServer(budget, state_fn=device_initial_state(dev), device=dev, **caps)
    st = srv.run(arrivals, duration=seconds)
    err = srv.batch.error()
    assert err == 0, "device error bits %d" % err
    active = list(srv.sched.active)
    srv.close()
    if backlog and active:
        # the sessions running at the end, stepped by the batch alone (same
        # instances, same default launch shape, actions drawn the same way,
        # steps back to back): the serving loop's cost over the bare kernels
        bare = bare_set_rate(dev, active, caps["max_slots"], caps["arena_agents"],
                             caps["max_cells"])
        st["bare_same_set"] = bare
        st["vs_bare_same_set"] = st["agent_steps_per_s"] / bare["agent_steps_per_s"]
    if world > 1:
        wall = max_over_ranks(st["wall_s"], dev)
        st["agent_steps_per_s"] = sum_over_ranks(st["agent_steps"], dev) / wall
        st["placement"] = {"ranks": world, "sessions_this_rank": len(arrivals),
                           "rule": "least placed work (agents x steps), same on every rank"}
    st.update({"rate_per_s": rate, "budget_bytes": budget, "backlog": backlog,
               "seconds": seconds, "sessions_offered": offered})
    return st


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--agents", type=int, default=N_AGENTS)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-policy", action="store_true")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the 1,000- and 5,000-agent plain steps")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the paper's own flock variant (16,000 agents, 128 sectors)")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--tuning", default=None,
                    help='launch shape as JSON, e.g. {"mode": 2, "stencil": 1, "block": 128}')
    ap.add_argument("--batch-tuning", default=None,
                    help='batched form: launch shape as JSON instead of the autotuner\'s, '
                         'e.g. {"stencil": 1, "mode": 3}')
    ap.add_argument("--autotune", action="store_true",
                    help="plain step: launch shape from the autotuner instead of the default")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    import paper_2207_03945_gb300 as F

    n = args.agents
    side = fi.side_for(n)
    p = fi.default_params(side)
    seed = rank_seed(rank)
    st0 = fi.initial_state(n, side, seed)
    total = args.warmup + args.steps
    acts_h = fi.random_actions(n, total, seed)
    acts = torch.from_numpy(acts_h).to(dev)
    act_buf = torch.empty(n, dtype=torch.int32, device=dev)  # fixed pointer: one graph capture
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    if args.tuning:
        tuning = json.loads(args.tuning)
        tuned_by = "command line"
    elif args.autotune:
        from paper_2207_03945_gb300.autotune import autotune
        tuning, _ = autotune(p, st0, device=dev, use_cache=False)
        tuned_by = "autotuner (bit-identical candidates, fastest kept)"
    else:
        tuning = None
        tuned_by = "library default (direct form, 3 x 3 cells, lanes per agent by agent count)"
    env = F.FlockEnv(p, n, device=dev, stream=stream, tuning=tuning)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        env.reset(torch.from_numpy(st0).to(dev))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(total)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(total)]
    stream.synchronize()
    for k in range(args.warmup):
        with torch.cuda.stream(stream):
            act_buf.copy_(acts[k])
            flush.zero_()
            starts[k].record(stream)
            env.step(act_buf)
            ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    # timed region: K steps, each bracketed by events on the library's
    # stream, the L2 flush and the action copy outside the events
    with ClockSampler(local) as clk:
        for k in range(args.warmup, total):
            with torch.cuda.stream(stream):
                act_buf.copy_(acts[k])
                flush.zero_()  # L2 flush between timed steps (outside the events)
                starts[k].record(stream)
                env.step(act_buf)
                ends[k].record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    # second pass, same workload: CUDA events recorded inside the step graph
    # around each kernel give the per-kernel durations for the roofline
    F.env_set_timing(env.env, True)
    phase = []
    for k in range(args.warmup, total):
        with torch.cuda.stream(stream):
            act_buf.copy_(acts[k])
            flush.zero_()
            env.step(act_buf)
        phase.append(F.env_get_phase_times(env.env))
    F.env_set_timing(env.env, False)
    step_ms = [starts[k].elapsed_time(ends[k]) for k in range(args.warmup, total)]
    tot_ms = max_over_ranks(sum(step_ms), dev)
    err = env.error()
    assert err == 0, "device error bits %d" % err
    value = weak_scaling_value(world, n, args.steps, tot_ms)
    ph = np.array(phase)
    neigh_ms = float(ph[:, 3].mean())
    peak, peak_kind = peaks()
    # the step's algorithmic bytes per agent (116) over the dominant kernel's time
    achieved = BYTES_PER_AGENT_STEP * n / (neigh_ms * 1e-3) / 1e9
    step_gbs = BYTES_PER_AGENT_STEP * n / (tot_ms / args.steps * 1e-3) / 1e9

    # end to end through host buffers (pinned): actions in, outputs out
    act_h = torch.from_numpy(acts_h[args.warmup]).pin_memory()
    obs_h = torch.empty((n, env.obs_dim), dtype=torch.float32).pin_memory()
    rew_h = torch.empty(n, dtype=torch.float32).pin_memory()
    coll_h = torch.empty(n, dtype=torch.int32).pin_memory()
    # the host step bound to these buffers (checked once; the same C call each step)
    host_step = F.env_step_host_bind(env.env, act_h, obs_h, rew_h, coll_h)
    for _ in range(3):
        host_step()
    e2e_steps = max(10, min(args.steps, 100))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_step()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * n * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": n * 4, "d2h_bytes_per_step": n * (env.obs_dim + 2) * 4,
           "call": "env_step_host through env_step_host_bind (pinned host buffers: the "
                   "actions read in place over NVLink-C2C, the outputs written into the "
                   "mapped buffers by the neighbour scan in agent order; one graph; "
                   "synchronous)"}

    batched = batch_of_one = None
    if not args.no_batched:
        batched = run_batched(F, torch, dev, stream, args.steps, args.warmup, flush,
                              seed=rank_seed(rank), world=world,
                              tuning=json.loads(args.batch_tuning) if args.batch_tuning else None)
        # the same 50,000-agent instance as the headline, as a batch of one
        batch_of_one = run_batched(F, torch, dev, stream, args.steps, args.warmup, flush,
                                   seed=rank_seed(rank), sizes=[n], world=world, tune=False)
        # like for like with the headline: its agents as ten 5,000-agent instances
        # the mix's tuned form and block; lanes per agent by these instances' size
        ten_tuning = {k: v for k, v in (batched["tuning"] or {}).items() if k != "lanes"}
        ten = run_batched(F, torch, dev, stream, args.steps, args.warmup, flush,
                          seed=rank_seed(rank), sizes=[n // 10] * 10, world=world, tune=False,
                          tuning=ten_tuning)
    serving = None
    if args.serve_seconds > 0:
        serving = {
            "as_specified": run_serving(dev, args.serve_seconds, seed=0, rank=rank,
                                        world=world),
            "saturated_small_budget": run_serving(dev, max(5.0, args.serve_seconds / 2),
                                                  seed=1, budget=10 ** 8, backlog=5000 * world,
                                                  rank=rank, world=world),
            "workload": "serving: Poisson arrivals 50/s, agents log-uniform in [500, 50000], "
                        "episodes uniform in [100, 2000] steps, 100 GB budget, random actions; "
                        "plus a saturated run (5,000 sessions queued at t=0, more than the run "
                        "serves, 100 MB budget so that admission binds); initial states drawn "
                        "on the device from each session's seed at admission; with N ranks one "
                        "job-wide arrival stream is placed across them on the host (least placed "
                        "work) and the saturated backlog is 5,000 per rank"}
    # the other plain-step configurations: 1,000 agents for 100 steps, 5,000
    # agents (the same density) for 1,000 steps
    small = None
    if not args.no_small:
        small = {"n1000_100_steps": run_plain(F, torch, dev, stream, 1000, 100, args.warmup, flush,
                                              seed=rank_seed(rank), world=world),
                 "n5000_1000_steps": run_plain(F, torch, dev, stream, 5000, 1000, args.warmup,
                                               flush, seed=rank_seed(rank), world=world)}
    policy = plain100k = None
    if not args.no_policy:
        policy = run_policy(F, torch, dev, stream, args.steps, args.warmup, flush,
                            seed=rank_seed(rank), world=world)
        # the plain step on the policy's 100,000 agents, like for like
        plain100k = run_plain(F, torch, dev, stream, 100000, args.steps, args.warmup, flush,
                              seed=rank_seed(rank), world=world,
                              what=" (the fused policy's agent count, observations written)")
        policy["plain_step_same_agents"] = {k: plain100k[k] for k in
                                            ("value", "ms_per_step", "p50_ms", "p99_ms")}
    paper = rollout = tag = None
    if not args.no_paper:
        paper = run_paper_variant(F, torch, dev, stream, min(args.steps, 50), args.warmup, flush,
                                  seed=rank_seed(rank), world=world)
        rollout = run_rollout(F, torch, dev, stream, 3, flush, seed=rank_seed(rank), world=world)
        tag = run_tag(F, torch, dev, stream, min(args.steps, 50), args.warmup, flush,
                      seed=rank_seed(rank), world=world)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": PLAIN_WORKLOAD % (n, side),
                       "form": "CUDA graph of 4 kernels",
                       "agents": n, "tuning": env.tuning(), "tuned_by": tuned_by,
                       "l2": "flushed (512 MiB write) between timed steps",
                       "parallelism": "replicas" if world > 1 else "single"},
            "step_hbm_gbs": step_gbs,
            "phase_ms": {"apply_bin": float(ph[:, 0].mean()), "scan": float(ph[:, 1].mean()),
                         "scatter": float(ph[:, 2].mean()), "neighbours": neigh_ms},
            "roofline": {"bound": "hbm", "kernel": "k_neighbours_direct", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_kind,
                         "traffic": measured_traffic("k_neighbours_direct", "plain-%d-%s" % (
                             n, tuning_tag(env.tuning()))),
                         "bytes_per_agent": BYTES_PER_AGENT_STEP,
                         "kernel_own_bytes_per_agent": NEIGH_BYTES_PER_AGENT},
            "e2e": e2e,
            "clocks": clk.summary(),
            # kernels of this library launched inside the timed region (four per step)
            "gpu_launches": 4 * args.steps,
        }
        if batched is not None:
            line["batched"] = batched
            line["batch_of_one"] = batch_of_one
            line["batched_10_instances"] = ten
        if small is not None:
            line["plain_small"] = small
        if policy is not None:
            line["policy"] = policy
        if paper is not None:
            line["paper_variant"] = paper
            line["rollout"] = rollout
            line["tag"] = tag
        if serving is not None:
            if batched is not None:
                # saturated serving against the bare batched form (per agent-step)
                sat = serving["saturated_small_budget"]
                sat["vs_batched_form"] = sat["agent_steps_per_s"] / batched["value"]
            line["serving"] = serving

        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    env.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
