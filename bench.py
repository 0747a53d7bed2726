"""Benchmark: prime paths emitted per second on the 2^22-path diamond chain.

One step = the whole hot path on one graph: load + validate + predecessor CSR
+ all-pairs BFS tables (device-resident input), the level-synchronous
frontier with compaction and primality, canonical ordering and
materialisation of the prime paths, and test-path assembly with canonical
sort/dedup.  Workload: a chain of k=22 if-else diamonds (67 vertices, 88
arcs), 4,194,304 prime paths of 45 vertices, 67,108,695 simple paths.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chain|batch]

--workload batch times the 4096-graph batch (graphs of 10-150 vertices, loop
nesting 0-4, switch fan-out 2-6): one persistent frontier launch over all
graphs with the whole hot path captured in a CUDA graph (tile shape from the
autotuner), compared with host-driven batched calls and with per-graph plain
launches.

Prints one JSON line.  Under torchrun each rank runs an independent replica
(the single graph is not sharded), so per-GPU work is fixed: weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "prime paths emitted/sec"
UNIT = "PP/s"
K_DIAMONDS = 22
ALG_BYTES_PER_NODE = 16  # lean frontier: int32 parent + int32 last vertex, written once and read once
PROFILE = os.path.join(ROOT, "profiles", "enumerate_kernel_diamond22_traffic.txt")


def workload():
    from paper_2210_16998_gb300 import cfggen

    return cfggen.diamond_chain(K_DIAMONDS)


def chain_sizes(k):
    return 3 * k + 1, 4 * k, 2 ** k, 2 * k + 1


def config_dict(extra=None):
    n, m, P, L = chain_sizes(K_DIAMONDS)
    d = {"workload": f"diamond-chain k={K_DIAMONDS} ({n} vertices, {m} arcs, {P:,} PPs x {L} vertices)",
         "graphs": 1, "vertices": n, "arcs": m,
         "step": "load+validate+BFS tables, frontier/compaction/primality, canonical order, PP materialise, "
                 "TP assembly + sort/dedup",
         "l2": "inputs > L2: arena + frontier + PP/TP outputs ~2.9 GB per step >> 129 MB L2"}
    if extra:
        d.update(extra)
    return d


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def kernel_source_digest():
    h = hashlib.sha256()
    for f in ("enumerate.cu", "common.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_2210_16998_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the frontier kernel from the committed ncu summary,
    or None if that summary was taken on a different kernel source."""
    if not os.path.exists(PROFILE):
        return None
    kv = {}
    with open(PROFILE) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_source_digest():
        return None
    try:
        return int(float(kv["dram_bytes_per_launch"]))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def closed_form_check(pp):
    """Sampled outputs against the closed form of the diamond chain: PP j in
    canonical order takes b_i (3i+2) at diamond i iff bit (k-1-i) of j is set."""
    import torch

    P = pp.num_paths
    assert P == 2 ** K_DIAMONDS, P
    idx = torch.tensor(sorted({0, 1, 2, min(12345, P - 1), P // 3, P // 2, P - 2, P - 1}), device="cuda")
    off = pp.offsets[idx].cpu().numpy()
    assert np.all(off == idx.cpu().numpy() * (2 * K_DIAMONDS + 1))
    for j, o in zip(idx.cpu().numpy(), off):
        seq = pp.vertices[int(o):int(o) + 2 * K_DIAMONDS + 1].cpu().numpy()
        exp = [0]
        for i in range(K_DIAMONDS):
            exp += [3 * i + (2 if (int(j) >> (K_DIAMONDS - 1 - i)) & 1 else 1), 3 * i + 3]
        assert list(seq) == exp, (j, seq, exp)


def parse_tile(text):
    """'block,items[,split]' -> tuple, or None for the library default."""
    if not text:
        return None
    v = tuple(int(x) for x in text.split(","))
    if len(v) not in (2, 3):
        raise SystemExit(f"--tile wants block,items[,split], got {text!r}")
    return v


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2210_16998_gb300 import cfggen, tpg

    torch.cuda.set_device(local_rank)
    tpg.load_library(build=True)
    cfg = workload()
    rp = torch.as_tensor(cfg.row_ptr, device="cuda")
    col = torch.as_tensor(cfg.col, device="cuda")

    shape = parse_tile(args.tile)

    def step(check=False):
        h = tpg.tpg_load_cfg_device(cfg.n, cfg.m, rp, col, cfg.entry, cfg.exit)
        if shape:
            tpg.set_tile(h, shape)
        pp = tpg.tpg_prime_paths(h)
        if check:
            closed_form_check(pp)
        tp = tpg.tpg_test_paths(h)
        if check:
            assert tp.num_paths == pp.num_paths  # every PP already runs entry -> exit
            assert torch.equal(tp.vertices, pp.vertices)
        st = tpg.tpg_get_stats(h, as_dict=False)  # converted after the timed region
        P = pp.num_paths
        pp.free()
        tp.free()
        h.close()
        return P, st

    for i in range(args.warmup):
        step(check=(i == 0))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = tpg.tpg_kernel_launches()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    stats, total_pp = [], 0
    for _ in range(args.steps):
        P, st = step()
        total_pp += P
        stats.append(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = tpg.tpg_kernel_launches() - launches0
    clocks = sampler.stop() if sampler else None
    stats = [tpg.stats_dict(s) for s in stats]
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    ms = float(t.item())
    ms_per_step = ms / args.steps
    value = world * total_pp / (ms / 1000.0)

    # e2e through the C ABI with host buffers (H2D of the CSR, D2H of both
    # results), with a per-call breakdown
    e2e_steps = 0 if args.no_e2e else args.steps
    bi = int(cfg.row_ptr.nbytes + cfg.col.nbytes)

    def e2e_step():
        t0 = time.perf_counter()
        h = tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, location=tpg.TPG_RESULT_HOST)
        if shape:
            tpg.set_tile(h, shape)
        t1 = time.perf_counter()
        pp = tpg.tpg_prime_paths(h)
        t2 = time.perf_counter()
        s1 = tpg.tpg_get_stats(h, as_dict=False)
        tp = tpg.tpg_test_paths(h)
        t3 = time.perf_counter()
        s2 = tpg.tpg_get_stats(h, as_dict=False)
        # bytes read back to the host: a TP list equal to the PP list shares
        # its host copy, so count every distinct buffer once
        bufs = {}
        for r in (pp, tp):
            for arr in (r.graph_path_ptr, r.offsets, r.vertices):
                bufs[arr.ctypes.data] = max(bufs.get(arr.ctypes.data, 0), arr.nbytes)
        nbytes = sum(bufs.values())
        P = pp.num_paths
        pp.free()
        tp.free()
        h.close()
        t4 = time.perf_counter()
        ph = {"load": 1e3 * (t1 - t0), "prime_paths_call": 1e3 * (t2 - t1), "test_paths_call": 1e3 * (t3 - t2),
              "free": 1e3 * (t4 - t3), "enumerate": s1.t_enumerate_ms, "order_materialise": s1.t_order_ms,
              "test_paths_device": s2.t_test_paths_ms,
              "d2h": s1.t_result_copy_ms + s2.t_result_copy_ms,
              "d2h_bytes": s1.result_copy_bytes + s2.result_copy_bytes}
        return P, nbytes, ph

    if e2e_steps:
        e2e_step()  # warm the pinned pool
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_pp, phases, bo = 0, [], 0
    for _ in range(e2e_steps):
        P, bo, ph = e2e_step()
        e2e_pp += P
        phases.append(ph)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * e2e_pp / float(te.item()) if e2e_steps else None
    # the device-to-host link alone: the same byte count copied from device
    # memory to page-locked host memory by the copy engine
    link_gbps = None
    if e2e_steps and bo > 0:
        src = torch.empty(int(bo), dtype=torch.uint8, device="cuda")
        dst = torch.empty(int(bo), dtype=torch.uint8, pin_memory=True)
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        eb.record(stream)
        torch.cuda.synchronize()
        link_gbps = 3 * int(bo) / (ea.elapsed_time(eb) / 1e3) / 1e9
        del src, dst
    e2e_break = None
    if phases:
        e2e_break = {k: statistics.median(p[k] for p in phases) for k in phases[0]}
        e2e_break["step_ms"] = 1e3 * e2e_s / e2e_steps
        d2h = e2e_break["d2h"]
        e2e_break["d2h_gb_per_s"] = e2e_break["d2h_bytes"] / (d2h / 1e3) / 1e9 if d2h > 0 else None
        e2e_break["link_d2h_gb_per_s"] = link_gbps
        e2e_break["host_other"] = e2e_break["step_ms"] - (e2e_break["enumerate"] + e2e_break["order_materialise"]
                                                          + e2e_break["test_paths_device"] + d2h)

    extra = {}
    if args.level_trace and rank == 0:
        extra["level_trace"] = level_trace(tpg, cfg, rp, col, shape)
    if not args.no_extra and rank == 0:
        extra["config1"] = config_record(tpg, cfggen.config1_cfg(), "structured CFG, 24 vertices (4 if-else, "
                                         "2 while, nesting <= 3, seed 1)", steps=max(args.steps, 20))
        extra["config3"] = config_record(tpg, cfggen.config3_cfg(), "structured CFG, 120 vertices (10 while "
                                         "nested <= 4, 3 switch x6, if-else), cyclic", steps=max(args.steps // 2, 5))
        extra["batch4096"] = batch_record(tpg, cfggen, steps=max(args.steps // 2, 5))
        extra["touring"] = touring_record(tpg, cfggen, steps=3, with_cpu=not args.no_cpu_baseline)

    if rank != 0:
        return None
    peak, peak_kind = measured_peaks()
    t_enum = statistics.mean(s["t_enumerate_ms"] for s in stats)
    nodes = stats[-1]["simple_paths"]
    achieved = ALG_BYTES_PER_NODE * nodes / (t_enum / 1000.0) / 1e9
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded diamond-chain CFG)",
        "config": config_dict({"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
        "tile": [stats[-1]["tile_block"], stats[-1]["tile_items"], shape[2] if shape and len(shape) > 2 else 1],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": int(bo),
                "steps": e2e_steps, "phases_ms": e2e_break},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "enumerate_kernel", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "alg_bytes_per_launch": ALG_BYTES_PER_NODE * nodes,
                     "launch_ms": t_enum},
        "phases_ms": {"enumerate": t_enum, "order_materialise": statistics.mean(s["t_order_ms"] for s in stats),
                      "test_paths": statistics.mean(s["t_test_paths_ms"] for s in stats)},
        "clocks": clocks,
    }
    line.update(extra)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, budget_s=args.cpu_budget)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(cfg, budget_s=args.cpu_budget / 2)
    return line


def level_trace(tpg, cfg, rp, col, shape):
    """Per-level timing of one frontier launch (tpg_set_level_trace), after
    two untraced calls: rows [level, duration us, last warp us, mean warp us,
    warps with work]; the duration of a level runs to the next level's
    start, so it includes the grid barrier and the prefix step."""
    h = tpg.tpg_load_cfg_device(cfg.n, cfg.m, rp, col, cfg.entry, cfg.exit)
    if shape:
        tpg.set_tile(h, shape)
    for _ in range(2):
        tpg.tpg_prime_paths(h).free()
    tpg.tpg_set_level_trace(h, True)
    tpg.tpg_prime_paths(h).free()
    tr = tpg.tpg_get_level_trace(h)
    h.close()
    rows = []
    for k in range(1, len(tr)):
        if tr[k, 0] < 0:
            continue
        nxt = tr[k + 1, 0] if k + 1 < len(tr) and tr[k + 1, 0] >= 0 else tr[k, 1]
        rows.append([k, round((nxt - tr[k, 0]) / 1e3, 2), round((tr[k, 1] - tr[k, 0]) / 1e3, 2),
                     round(tr[k, 2] / max(tr[k, 3], 1) / 1e3, 2), int(tr[k, 3])])
    return rows


def config_record(tpg, cfg, what, steps):
    """One graph with device-resident inputs: load + PPs + TPs per step (CUDA
    events over `steps` steps after warm-up), with the enumeration's volumes."""
    import torch

    rp = torch.as_tensor(cfg.row_ptr, device="cuda")
    col = torch.as_tensor(cfg.col, device="cuda")

    def one():
        h = tpg.tpg_load_cfg_device(cfg.n, cfg.m, rp, col, cfg.entry, cfg.exit)
        pp = tpg.tpg_prime_paths(h)
        tp = tpg.tpg_test_paths(h)
        st = tpg.tpg_get_stats(h, as_dict=False)
        out = (pp.num_paths, tp.num_paths, st)
        pp.free()
        tp.free()
        h.close()
        return out

    for _ in range(3):
        one()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    sts = []
    for _ in range(steps):
        P, T, st = one()
        sts.append(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    st = tpg.stats_dict(sts[-1])
    rec_bytes = 8 + 2 + 4 * st["bitset_words"]  # {first, last}, count word, bitset per frontier path
    return {"workload": what, "vertices": cfg.n, "arcs": cfg.m, "prime_paths": P, "test_paths": T,
            "ms_per_step": ms, "pp_per_s": P / (ms / 1e3), "steps": steps,
            "step": "load+validate+BFS tables, PPs, TPs (inputs resident)",
            "simple_paths": st["simple_paths"], "levels": st["levels"],
            "peak_level_paths": st["peak_level_nodes"],
            "peak_frontier_bytes": st["peak_level_nodes"] * rec_bytes,
            "arena_bytes_used": st["arena_bytes_used"], "arena_bytes_alloc": st["arena_bytes_alloc"],
            "frontier_bytes_alloc": st["frontier_bytes_alloc"],
            "device_ms": {"enumerate": statistics.median(s.t_enumerate_ms for s in sts),
                          "order_materialise": statistics.median(s.t_order_ms for s in sts),
                          "test_paths": statistics.median(s.t_test_paths_ms for s in sts)}}


def batch_record(tpg, cfggen, steps, tile=(1024, 1, 1)):
    """The 4096-graph batch: host-driven batched calls and graph-mode replays
    on one handle (inputs and BFS tables resident; fixed tile shape)."""
    import torch

    cfgs = cfggen.batch_cfgs(4096)
    ns, rp, col, ent, ext = cfggen.concat_batch(cfgs)
    h = tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE)
    tpg.set_tile(h, tile)
    host_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pp = tpg.tpg_prime_paths(h)
        tp = tpg.tpg_test_paths(h)
        torch.cuda.synchronize()
        host_ms.append(1e3 * (time.perf_counter() - t0))
        P, T = pp.num_paths, tp.num_paths
        pp.free()
        tp.free()
    st = tpg.tpg_get_stats(h)
    tpg.tpg_graph_capture(h)
    for _ in range(3):
        a, b = tpg.tpg_graph_launch(h)
        a.free()
        b.free()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        a, b = tpg.tpg_graph_launch(h)
        a.free()
        b.free()
    ev1.record(stream)
    torch.cuda.synchronize()
    rep_ms = ev0.elapsed_time(ev1) / steps
    fb = tpg.tpg_get_stats(h)["graph_fallbacks"]
    h.close()
    return {"workload": "batch of 4096 seeded structured CFGs (n log-uniform 10-150, loop nesting 0-4, switch "
                        "fan-out 2-6)", "graphs": len(cfgs), "vertices": int(ns.sum()), "prime_paths": P,
            "test_paths": T, "simple_paths": st["simple_paths"], "tile": list(tile),
            "graph_replay_ms": rep_ms, "graph_replay_pp_per_s": P / (rep_ms / 1e3), "replays": steps,
            "graph_fallbacks": fb,
            "host_driven_ms": min(host_ms), "host_driven_pp_per_s": P / (min(host_ms) / 1e3),
            "host_driven_device_ms": {"enumerate": st["t_enumerate_ms"], "order_materialise": st["t_order_ms"],
                                      "test_paths": st["t_test_paths_ms"]}}


def touring_record(tpg, cfggen, steps, with_cpu, which=("batch4096", "config3")):
    """Longest-first touring (tpg_test_paths_greedy) after the one-per-PP TP
    list, on the 4096-graph batch and the 120-vertex CFG: TP counts and the
    touring's device time (hash tables, touring launch, compaction)."""
    import torch

    out = {}
    cases = [("batch4096", lambda: cfggen.batch_cfgs(4096)), ("config3", lambda: [cfggen.config3_cfg()])]
    for name, make in cases:
        if name not in which:
            continue
        cfgs = make()
        ns, rp, col, ent, ext = cfggen.concat_batch(cfgs)
        h = tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE)
        with tpg.tpg_test_paths(h) as tp:
            T = tp.num_paths
        dev, call = [], []
        for i in range(steps + 2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gt = tpg.tpg_test_paths_greedy(h)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            GT = gt.num_paths
            gt.free()
            st = tpg.tpg_get_stats(h)
            if i >= 2:
                dev.append(st["t_touring_ms"])
                call.append(1e3 * el)
        P = st["prime_paths"]
        rec = {"graphs": len(cfgs), "prime_paths": P, "one_per_pp_test_paths": T, "touring_test_paths": GT,
               "touring_device_ms": statistics.median(dev), "call_ms": statistics.median(call),
               "decision_sweeps": st["touring_sweeps"], "cover_edges": st["touring_edges"], "steps": steps,
               "call": "tpg_test_paths_greedy on a handle whose PPs are cached: one-per-PP TP pipeline, then "
                       "touring (device_ms covers the touring alone)"}
        h.close()
        if with_cpu and len(cfgs) > 1:  # (the 120-vertex CFG alone takes the oracle ~2 minutes)
            import oracle

            oracle.build()
            t0 = time.perf_counter()
            k = 0
            while k < len(cfgs) and (k == 0 or time.perf_counter() - t0 < 10.0):
                oracle.run_cfg(cfgs[k], test_paths=False, greedy=True)
                k += 1
            el = time.perf_counter() - t0
            rec["cpu_baseline"] = {"kind": "oracle", "cores": 1, "graphs": k, "s": el,
                                   "sample": f"PPs + touring of the first {k} of {len(cfgs)} graphs, "
                                             f"single-threaded C -O2"}
        out[name] = rec
    return out


def run_pervertex(args, rank, world, local_rank):
    """The paper-style per-vertex-list baseline (tpg_prime_paths_pervertex)
    beside tpg_prime_paths on out-degree-2 inputs: its device time, the
    simple paths it copies and their bytes."""
    import torch

    from paper_2210_16998_gb300 import cfggen, tpg

    torch.cuda.set_device(local_rank)
    tpg.load_library(build=True)
    cases = [("structured CFG, 24 vertices", cfggen.config1_cfg())] + \
        [(f"diamond chain k={k}", cfggen.diamond_chain(k)) for k in (6, 8, 10)] + \
        [("structured CFG of the 4096-graph batch (graph 25), switches binarised",
          cfggen.binarise_switches(cfggen.random_cfg(cfggen.BATCH_SEED0 + 25)))]
    rows = []
    for name, cfg in cases:
        h = tpg.tpg_load_cfg_device(cfg.n, cfg.m, torch.as_tensor(cfg.row_ptr, device="cuda"),
                                    torch.as_tensor(cfg.col if cfg.m else np.zeros(1, np.int32), device="cuda"),
                                    cfg.entry, cfg.exit)
        tpg.tpg_set_result_location(h, tpg.TPG_RESULT_DEVICE)
        pv, ours = [], []
        for i in range(max(args.steps, 1) + 1):
            a = tpg.tpg_prime_paths_pervertex(h)
            P = a.num_paths
            a.free()
            st = tpg.tpg_get_stats(h)
            b = tpg.tpg_prime_paths(h)
            assert b.num_paths == P
            b.free()
            st2 = tpg.tpg_get_stats(h)
            if i:
                pv.append(st["t_pervertex_ms"])
                ours.append(st2["t_enumerate_ms"] + st2["t_order_ms"])
            tpg.tpg_release_cached_memory()
        h.close()
        rows.append({"input": name, "vertices": cfg.n, "prime_paths": P, "simple_paths": st["pervertex_paths"],
                     "pervertex_ms": statistics.median(pv), "pervertex_list_bytes": st["pervertex_bytes"],
                     "frontier_ms": statistics.median(ours),
                     "speedup": statistics.median(pv) / max(statistics.median(ours), 1e-9)})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    if rank != 0:
        return None
    return {"metric": "per-vertex-list baseline vs the frontier path (device ms)", "unit": "ms",
            "n_gpus": world, "steps": args.steps, "higher_is_better": False, "dtype": "int32",
            "data": "synthetic (seeded CFGs, out-degree <= 2)",
            "config": {"workload": "paper-style baseline: one thread per vertex, copied path lists"},
            "pervertex": rows}


def run_scc(args, rank, world, local_rank):
    """The per-SCC step of the compositional route (tpg_scc_internal_pps)
    beside the direct PP enumeration, on single CFGs."""
    import torch

    from paper_2210_16998_gb300 import cfggen, tpg

    torch.cuda.set_device(local_rank)
    tpg.load_library(build=True)
    cases = [("structured CFG, 24 vertices", cfggen.config1_cfg()),
             ("structured CFG, 120 vertices", cfggen.config3_cfg())] + \
        [(f"structured CFG of the 4096-graph batch (graph {i})", cfggen.random_cfg(cfggen.BATCH_SEED0 + i))
         for i in (21, 47, 54)]
    rows = []
    for name, cfg in cases:
        h = tpg.tpg_load_cfg(cfg.n, cfg.row_ptr, cfg.col, cfg.entry, cfg.exit, location=tpg.TPG_RESULT_DEVICE)
        scc, direct, compo = [], [], []
        for i in range(max(args.steps, 1) + 1):
            a = tpg.tpg_scc_internal_pps(h)
            a.free()
            st = tpg.tpg_get_stats(h)
            c = tpg.tpg_prime_paths_compositional(h)
            Pc = c.num_paths
            c.free()
            st3 = tpg.tpg_get_stats(h)
            b = tpg.tpg_prime_paths(h)
            P = b.num_paths
            b.free()
            st2 = tpg.tpg_get_stats(h)
            assert Pc == P
            if i:
                scc.append(st["t_scc_ms"])
                compo.append(st3["t_compositional_ms"])
                direct.append(st2["t_enumerate_ms"] + st2["t_order_ms"])
        comp = tpg.tpg_scc_ids(h, cfg.n)
        h.close()
        rows.append({"input": name, "vertices": cfg.n, "sccs": int(len(set(comp.tolist()))),
                     "largest_scc": int(np.bincount(comp).max()), "prime_paths": P,
                     "scc_subgraph_pps": st["scc_pps"], "scc_internal_pps": st["scc_internal_pps"],
                     "scc_step_ms": statistics.median(scc), "direct_pp_ms": statistics.median(direct),
                     "compositional_pp_ms": statistics.median(compo),
                     "extracted_paths": {"entry_exit": st3["comp_entry_exit_paths"], "exit": st3["comp_exit_paths"],
                                         "entry": st3["comp_entry_paths"]},
                     "crossing_pps": st3["comp_crossing_pps"]})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    if rank != 0:
        return None
    return {"metric": "compositional route vs the direct enumeration (device ms)", "unit": "ms", "n_gpus": world,
            "steps": args.steps, "higher_is_better": False, "dtype": "int32", "data": "synthetic (seeded CFGs)",
            "config": {"workload": "SCC ids, SccInternalPPs through the frontier, path extraction, merge, sort"},
            "scc": rows}


def run_touring(args, rank, world, local_rank):
    """Only the touring sub-record (longest-first TP sets of the 4096-graph
    batch and the 120-vertex CFG)."""
    import torch

    from paper_2210_16998_gb300 import cfggen, tpg

    torch.cuda.set_device(local_rank)
    tpg.load_library(build=True)
    which = ("batch4096", "config3") if args.touring_case == "all" else (args.touring_case,)
    rec = touring_record(tpg, cfggen, steps=max(args.steps, 1), with_cpu=not args.no_cpu_baseline, which=which)
    if rank != 0:
        return None
    first = rec[which[0]]
    P = first["prime_paths"]
    ms = first["touring_device_ms"]
    return {"metric": "prime paths toured/sec (longest-first touring)", "value": P / (ms / 1e3), "unit": "PP/s",
            "n_gpus": world, "steps": args.steps, "higher_is_better": True, "dtype": "int32",
            "data": "synthetic (seeded structured CFGs)",
            "config": {"workload": f"longest-first touring of {which[0]}"}, "touring": rec}


def cpu_baseline_all_cores(cfg, budget_s=6.0, min_runs=2):
    """The oracle's root-parallel driver on every host core: PPs + TPs of the
    same graph (the same enumeration per root; TPs built over PP ranges)."""
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    times, P = [], 0
    t_start = time.perf_counter()
    while len(times) < min_runs or time.perf_counter() - t_start < budget_s:
        t0 = time.perf_counter()
        r = oracle.run_cfg_parallel(cfg, test_paths=True, threads=threads)
        times.append(time.perf_counter() - t0)
        P = r.num_pp
        if len(times) >= 50:
            break
    return {"value": P / statistics.mean(times), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"full workload (PPs + TPs of the k=22 diamond chain), {len(times)} runs, "
                      f"mean {statistics.mean(times):.3f} s, root-parallel C -O2 on {threads} threads",
            "host": host_cpu()}


def cpu_baseline(cfg, budget_s=12.0, min_runs=2):
    """The oracle, as it stands, on the host cores: PPs + TPs of the same graph."""
    import oracle

    oracle.build()
    times, P = [], 0
    t_start = time.perf_counter()
    while len(times) < min_runs or time.perf_counter() - t_start < budget_s:
        t0 = time.perf_counter()
        r = oracle.run_cfg(cfg, test_paths=True)
        times.append(time.perf_counter() - t0)
        P = r.num_pp
        if len(times) >= 50:
            break
    return {"value": P / statistics.mean(times), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"full workload (PPs + TPs of the k=22 diamond chain), {len(times)} runs, "
                      f"mean {statistics.mean(times):.3f} s, single-threaded C -O2",
            "host": host_cpu()}


def host_cpu():
    name = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    name = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": name, "machine": os.uname().machine}


def run_batch(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2210_16998_gb300 import autotune, cfggen, tpg

    torch.cuda.set_device(local_rank)
    tpg.load_library(build=True)
    cfgs = cfggen.batch_cfgs(4096)
    ns, rp, col, ent, ext = cfggen.concat_batch(cfgs)
    if args.tile:
        shape, tuned = parse_tile(args.tile), {"fixed": args.tile}
    else:
        shape, tuned = autotune.tune()
    h = tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE)
    tpg.set_tile(h, shape)
    # host-driven batched run: exact sizes for the capture, and its own timing
    host_ms = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pp = tpg.tpg_prime_paths(h)
        tp = tpg.tpg_test_paths(h)
        torch.cuda.synchronize()
        host_ms.append(1000 * (time.perf_counter() - t0))
        P, T = pp.num_paths, tp.num_paths
        gptr = pp.graph_path_ptr.cpu().numpy()
        pp.free()
        tp.free()
    st_host = tpg.tpg_get_stats(h)
    tpg.tpg_graph_capture(h)
    for _ in range(args.warmup):
        a, b = tpg.tpg_graph_launch(h)
        assert a.num_paths == P and b.num_paths == T
        a.free()
        b.free()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = tpg.tpg_kernel_launches()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        a, b = tpg.tpg_graph_launch(h)
        a.free()
        b.free()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = tpg.tpg_kernel_launches() - launches0
    clocks = sampler.stop() if sampler else None
    st = tpg.tpg_get_stats(h)
    assert st["graph_fallbacks"] == 0
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item()) / args.steps
    value = world * P / (ms_per_step / 1000.0)
    h.close()

    # per-graph plain launches over the same 4096 graphs (inputs resident)
    plain_s = float("nan")
    if not args.no_plain:
        dev_inputs = [(torch.as_tensor(c.row_ptr, device="cuda"), torch.as_tensor(c.col, device="cuda"))
                      for c in cfgs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain_pp = 0
        for c, (r_, c_) in zip(cfgs, dev_inputs):
            hh = tpg.tpg_load_cfg_device(c.n, c.m, r_, c_, c.entry, c.exit)
            a = tpg.tpg_prime_paths(hh)
            b = tpg.tpg_test_paths(hh)
            plain_pp += a.num_paths
            a.free()
            b.free()
            hh.close()
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t0
        assert plain_pp == P

    # e2e through the C ABI with host buffers
    t0 = time.perf_counter()
    bo = 0
    he = tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_HOST)
    tpg.set_tile(he, shape)
    if not args.no_e2e:
        a = tpg.tpg_prime_paths(he)
        b = tpg.tpg_test_paths(he)
        bo = sum(x.nbytes for r in (a, b) for x in (r.graph_path_ptr, r.offsets, r.vertices))
        a.free()
        b.free()
    he.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    bi = int(ns.nbytes + rp.nbytes + col.nbytes + ent.nbytes + ext.nbytes)
    if rank != 0:
        return None
    peak, peak_kind = measured_peaks()
    nodes = st_host["simple_paths"]
    achieved = ALG_BYTES_PER_NODE * nodes / (st_host["t_enumerate_ms"] / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (4096 seeded structured CFGs)",
        "config": {"workload": "batch of 4096 seeded structured CFGs (n log-uniform 10-150, loop nesting 0-4, "
                               "switch fan-out 2-6)", "graphs": len(cfgs), "vertices": int(ns.sum()),
                   "prime_paths": P, "test_paths": T, "simple_paths": nodes,
                   "step": "CUDA-graph replay: one persistent frontier launch over all graphs, PP order + "
                           "materialise, TP assembly + sort/dedup (inputs and BFS tables resident)",
                   "tile_shape": list(shape), "autotune": tuned,
                   "l2": "inputs > L2: arena ~1.6 GB + outputs per step >> 129 MB L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "compare": {"host_driven_batched_pp_per_s": P / (min(host_ms) / 1000.0),
                    "host_driven_batched_ms": min(host_ms),
                    "host_driven_phases_ms": {"enumerate": st_host["t_enumerate_ms"],
                                              "order_materialise": st_host["t_order_ms"],
                                              "test_paths": st_host["t_test_paths_ms"]},
                    "per_graph_plain_pp_per_s": P / plain_s, "per_graph_plain_s": plain_s},
        "e2e": {"value": (P / e2e_s) if not args.no_e2e else None, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": int(bo)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": "enumerate_kernel", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "alg_bytes_per_launch": ALG_BYTES_PER_NODE * nodes, "launch_ms": st_host["t_enumerate_ms"]},
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        k, sP = 0, 0
        while time.perf_counter() - t0 < args.cpu_budget and k < len(cfgs):
            sP += oracle.run_cfg(cfgs[k], test_paths=True).num_pp
            k += 1
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sP / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {k} of the 4096 graphs (PPs + TPs), {el:.1f} s, "
                                          f"single-threaded C -O2", "host": host_cpu()}
    return line


def run_sizer(args, rank, world, local_rank):
    import torch

    from paper_2210_16998_gb300 import cfggen, tpg

    torch.cuda.set_device(local_rank)
    tpg.load_library(build=True)
    n_train = args.train_graphs
    t0 = time.perf_counter()
    train = [cfggen.random_cfg(cfggen.TRAIN_SEED0 + i) for i in range(n_train)]
    held = cfggen.batch_cfgs(4096, cfggen.HELDOUT_SEED0)
    gen_s = time.perf_counter() - t0
    z = tpg.tpg_sizer_create(seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b0 in range(0, n_train, 4096):
        ns, rp, col, ent, ext = cfggen.concat_batch(train[b0:b0 + 4096])
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
            tpg.tpg_sizer_add_batch(z, h)
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = tpg.tpg_sizer_train(z, args.epochs, 3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    ns, rp, col, ent, ext = cfggen.concat_batch(held)
    N = int(ns.sum())

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, out

    # exact per-graph volumes of the held-out batch (exact counting mode)
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
        counts = tpg.tpg_root_counts(h, N)
    bounds = np.concatenate([[0], np.cumsum(ns)])
    truth = np.array([counts[bounds[i]:bounds[i + 1]].sum(0) for i in range(len(held))], np.float64)

    # (a) plain host-driven enumerator, cold handle
    def plain_host():
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
            tpg.set_tile(h, shape)
            a, b = tpg.tpg_prime_paths(h), tpg.tpg_test_paths(h)
            st = tpg.tpg_get_stats(h)
            P = a.num_paths
            a.free()
            b.free()
        return P, st

    # (b) graph mode sized by an exact run, cold handle
    def plain_graph():
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
            tpg.set_tile(h, shape)
            tpg.tpg_graph_capture(h)
            a, b = tpg.tpg_graph_launch(h)
            P = a.num_paths
            a.free()
            b.free()
        return P

    # (c) host-driven calls pre-sized by the sizer, cold handle: the arena,
    # frontier and PP list start at the predicted sizes (times the margin)
    def sized_host(margin=args.margin):
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
            tpg.set_tile(h, shape)
            tpg.tpg_sizer_presize(z, h, margin)
            a, b = tpg.tpg_prime_paths(h), tpg.tpg_test_paths(h)
            st = tpg.tpg_get_stats(h)
            P = a.num_paths
            a.free()
            b.free()
        return P, st

    # (d) graph mode pre-sized by the sizer, cold handle
    def sized_graph(margin=args.margin):
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext, location=tpg.TPG_RESULT_DEVICE) as h:
            tpg.set_tile(h, shape)
            caps = tpg.tpg_sizer_presize(z, h, margin)
            tpg.tpg_graph_capture(h)
            a, b = tpg.tpg_graph_launch(h)
            st = tpg.tpg_get_stats(h)
            P = a.num_paths
            a.free()
            b.free()
            torch.cuda.synchronize()
            t_first = time.perf_counter() - t_start
            # steady-state replay of the same capture
            t = time.perf_counter()
            a, b = tpg.tpg_graph_launch(h)
            torch.cuda.synchronize()
            rep = time.perf_counter() - t
            a.free()
            b.free()
        return P, st, caps, rep, t_first

    shape = (512, 1)
    plain_host()
    plain_graph()
    sized_host()
    sized_graph()  # warm-up (allocator, module loading)
    ta, (Pa, sta) = min((timed(plain_host) for _ in range(3)), key=lambda r: r[0])
    tb, Pb = timed(plain_graph)
    td, (Pd, std) = min((timed(sized_host) for _ in range(3)), key=lambda r: r[0])
    Pc, stc, caps, rep_s, tc = sized_graph()
    assert Pa == Pb == Pc == Pd
    with tpg.tpg_load_cfg_batch(ns, rp, col, ent, ext) as h:
        pred, _ = tpg.tpg_sizer_predict(z, h, N)
    vol = np.expm1(np.maximum(pred.astype(np.float64), 0))
    est = np.array([vol[bounds[i]:bounds[i + 1]].sum(0) for i in range(len(held))])
    err = np.abs(np.log1p(est) - np.log1p(truth))
    used = truth[:, 0].sum() * 8
    line = {
        "metric": METRIC, "value": Pd / td, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1,
        "ms_per_step": 1000 * td, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 (sizer: bf16 weights, fp32 accumulate)", "data": "synthetic (seeded structured CFGs)",
        "config": {"workload": "learned sizer: train on 50k seeded CFGs (10-150 vertices), evaluate on a held-out "
                               "batch of 4096", "train_graphs": n_train, "epochs": args.epochs, "margin": args.margin,
                   "held_out_graphs": len(held), "vertices": N, "prime_paths": Pc,
                   "step": "cold start of a new batch: load + predict + presize + PPs + TPs (host-driven calls)"},
        "sizer": {"generate_s": gen_s, "label_s": label_s, "train_s": train_s,
                  "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                  "per_graph_abs_log_err_mean": [float(x) for x in err.mean(0)],
                  "per_graph_abs_log_err_p90": [float(x) for x in np.percentile(err, 90, axis=0)]},
        "compare": {
            "plain_host_driven": {"pp_per_s": Pa / ta, "s": ta, "arena_alloc_bytes": sta["arena_bytes_alloc"],
                                  "arena_waste": 1 - used / max(sta["arena_bytes_alloc"], 1),
                                  "frontier_launches": sta["attempts"]},
            "plain_graph_exact_sizing": {"pp_per_s": Pb / tb, "s": tb},
            "sizer_graph": {"pp_per_s": Pc / tc, "s": tc, "arena_alloc_bytes": int(caps[0]) * 8,
                            "arena_waste": 1 - used / max(int(caps[0]) * 8, 1),
                            "fallback": bool(stc["graph_fallbacks"]), "replay_pp_per_s": Pc / rep_s},
            "sizer_host_driven": {"pp_per_s": Pd / td, "s": td, "arena_alloc_bytes": std["arena_bytes_alloc"],
                                  "arena_waste": 1 - used / max(std["arena_bytes_alloc"], 1),
                                  "frontier_launches": std["attempts"]},
        },
    }
    z.close()
    return line


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle

    oracle.build()
    cfg = workload()
    for _ in range(args.warmup):
        oracle.run_cfg(cfg, test_paths=True)
    times, P = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.run_cfg(cfg, test_paths=True)
        times.append(time.perf_counter() - t0)
        P = r.num_pp
    total = sum(times)
    value = args.steps * P / total
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded diamond-chain CFG)",
        "config": config_dict({"parallelism": "host CPU, 1 thread"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"full workload per step (PPs + TPs), {args.steps} steps", "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    global K_DIAMONDS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--level-trace", action="store_true",
                    help="chain: add a per-level trace of one frontier launch")
    ap.add_argument("--no-extra", action="store_true",
                    help="chain: skip the structured-CFG and 4096-graph sub-records")
    ap.add_argument("--k", type=int, default=K_DIAMONDS, help="diamonds in the chain (22 = the benchmark workload)")
    ap.add_argument("--workload", choices=["chain", "batch", "sizer", "touring", "pervertex", "scc"],
                    default="chain")
    ap.add_argument("--train-graphs", type=int, default=50000, help="sizer: training graphs")
    ap.add_argument("--epochs", type=int, default=40, help="sizer: training epochs")
    ap.add_argument("--margin", type=float, default=1.25, help="sizer: capacity margin over predictions")
    ap.add_argument("--no-plain", action="store_true", help="batch: skip the per-graph plain launches")
    ap.add_argument("--touring-case", choices=["all", "batch4096", "config3"], default="all",
                    help="touring: which inputs")
    ap.add_argument("--tile", default="",
                    help="fixed frontier tile 'block,items' (batch: instead of the autotuner)")
    args = ap.parse_args()
    K_DIAMONDS = args.k
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist

            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        line = {"batch": run_batch, "sizer": run_sizer, "touring": run_touring,
                "pervertex": run_pervertex, "scc": run_scc}.get(args.workload, run_ours)(
            args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
