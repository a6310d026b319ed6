#!/usr/bin/env python3
"""Benchmark of the GB300 powersort path.

Workload: n = 10^8 int32 keys with a uint32 payload (the original index), made of runs whose
lengths are uniform in [1, 2 sqrt(n)] = [1, 20000], each run filled with sorted uniform-random
int32 values and 25% of runs reversed (descending).  Seeded and synthetic.  One step = one full
stable sort of one such array (run detection, node powers, merge tree, all merges).

GB300 arm (default): every step sorts its own resident device copy (800 MB of keys + payload,
larger than the 129 MB L2), so nothing is reused across steps; K steps are timed with CUDA
events between a barrier + synchronize on both sides, max over ranks.  Also reported:
  * roofline  -- the merge-tile kernel (the dominant one): algorithmic bytes (2 x elements x 8 B
                 per merge output) over its CUDA-event time inside the timed region, against the
                 measured HBM copy bandwidth; plus the whole sort against the merge-cost
                 roofline M x 8 B x 2 / bandwidth (M = exact merge cost of the detected runs).
  * e2e       -- the same metric through the C ABI's host-buffer call ps_sort_host_ws: every step
                 copies one pinned host array in, sorts it and copies it out to pinned host
                 memory, four streams with one caller-owned device buffer set each (the package's
                 HostSortPipeline and the serial ps_sort_host are reported beside it).
  * cpu_baseline -- the CPU oracle (single-threaded plain C++ powersort) on one input of the same
                 workload on the host cores.
--impl reference: the oracle as the reference arm, each step one full n = 10^8 input of the
same workload (the headline configuration), single thread.
Multi-GPU (torchrun): independent replicas, one array per rank, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GKeys/s and % of HBM merge-cost roofline; batched/served vs plain; p50/p99 latency"
UNIT = "GKeys/s"
N_DEFAULT = 10 ** 8
SEED = 42
WORKLOAD = "plain powersort, n=1e8 int32 keys + uint32 payload, run lengths uniform in [1, 2*sqrt(n)], " \
           "sorted uniform int32 per run, 25% of runs descending"
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it): the whole job is done when the last replica is."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, n: int, steps: int, max_ms: float) -> float:
    """Whole-job GKeys/s of `world` replicas that each sorted `steps` arrays of n keys."""
    return world * n * steps / (max_ms / 1000.0) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None, period_ms: int = 50):
        import tempfile
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="ps_clocks_", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", f"-lms={period_ms}"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3][0].isdigit())}


def _gen(n: int, seed: int):
    import numpy as np
    import workloads
    max_len = max(1, int(2 * np.sqrt(N_DEFAULT if n == N_DEFAULT else n)))
    return workloads.runs_i32(n, seed, max_len=max_len)


def _cpu_baseline(keys, vals, sample_desc: str):
    import oracle
    t = time.perf_counter()
    res = oracle.powersort(keys, vals)
    dt = time.perf_counter() - t
    return {"value": keys.size / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample_desc, "seconds": dt, "merge_cost": res.cost, "runs": res.r}


def check_sorted_device(out_k, out_v, in_k) -> bool:
    """The output is the unique stable sort of the input: keys non-decreasing, every output key is
    the input key its payload (the original index) names, every index appears once, and equal
    keys keep increasing indices."""
    import torch
    n = out_k.numel()
    idx = out_v.to(torch.int64) & 0xFFFFFFFF
    if not bool((out_k[1:] >= out_k[:-1]).all()):
        return False
    if not torch.equal(in_k[idx], out_k):
        return False
    seen = torch.zeros(n, dtype=torch.int32, device=out_k.device)
    seen.index_add_(0, idx, torch.ones(n, dtype=torch.int32, device=out_k.device))
    if not bool((seen == 1).all()):
        return False
    eq = out_k[1:] == out_k[:-1]
    return bool(((idx[1:] > idx[:-1]) | ~eq).all())


def measure_variant(ps, dev, name: str, keys, vals, kt: int, steps: int = 5, tree: int = 0, min_run: int = 1):
    """Sort throughput of one more workload (resident inputs, fresh copy per step); tree 1 uses
    peeksort's merge tree (Alg. 1) instead of powersort's; min_run > 1 extends short runs to that
    length first (Sec. 5.1)."""
    import numpy as np
    import torch
    eb = keys.dtype.itemsize + 4
    k0 = torch.from_numpy(keys.view({4: np.int32, 8: np.int64}[keys.dtype.itemsize])).to(dev)
    v0 = torch.from_numpy(vals.view(np.int32)).to(dev)
    an = ps.ps_analyze(k0, key_type=kt, tree=tree, min_run=min_run)
    n = keys.size
    ws = torch.empty(ps.ps_workspace_size(kt, True, n, False, tree), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    copies = [(k0.clone(), v0.clone()) for _ in range(steps + 2)]

    def one(i):
        if min_run > 1:
            ps.ps_sort_minrun_ws(copies[i][0], copies[i][1], ws, min_run, key_type=kt, stream=stream)
        elif tree:
            ps.ps_sort_tree_ws(copies[i][0], copies[i][1], ws, tree, key_type=kt, stream=stream)
        else:
            ps.ps_sort_ws(copies[i][0], copies[i][1], ws, key_type=kt, stream=stream)

    for i in range(2):
        one(i)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(2, steps + 2):
        one(i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    # per-stage device time of one more sort (the library's stage events, outside the timed loop)
    copies[0][0].copy_(k0)
    copies[0][1].copy_(v0)
    torch.cuda.synchronize(dev)
    ps.ps_profile_enable(True)
    one(0)
    torch.cuda.synchronize(dev)
    stages = {k2: round(v2["ms"], 4) for k2, v2 in ps.ps_profile_read().items() if v2["launches"]}
    ps.ps_profile_enable(False)
    peak, _ = _peaks()
    ideal = an["cost"] * eb * 2 / (peak * 1e9) * 1e3
    del copies, ws, k0, v0
    return {"workload": name, "n": int(n), "min_run": int(min_run), "runs": int(an["runs"]), "merge_cost": int(an["cost"]),
            "ms_per_sort": ms, "gkeys_s": n / (ms / 1e3) / 1e9, "merge_cost_roofline_frac": ideal / ms,
            "stages_ms": stages}


def measure_batched(ps, dev, count: int, reps: int = 3):
    """10,000 uneven int32 arrays (sizes floor(2^U(8,20)), runs uniform in [1, 2 sqrt(size)])
    sorted in one segmented call vs one plain call per array, same device-resident inputs."""
    import numpy as np
    import torch
    import workloads
    keys, vals, off = workloads.segmented_i32(count, seed=SEED)
    n = keys.size
    k0 = torch.from_numpy(keys).to(dev)
    v0 = torch.from_numpy(vals.view(np.int32)).to(dev)
    doff = torch.from_numpy(off).to(dev)
    an = ps.ps_analyze(k0, offsets=doff, key_type=ps.PS_KEY_I32)  # merge cost of all segments' trees
    # the batched mode's own tuned entry (segmented sorts of this size bucket), outside the timing
    tune = ps.ps_autotune_segmented(k0, v0, doff, key_type=ps.PS_KEY_I32)
    M = int(an["cost"])
    peak, peak_kind = _peaks()
    ideal_ms = M * 8 * 2 / (peak * 1e9) * 1e3
    dk, dv = k0.clone(), v0.clone()
    ws = torch.empty(ps.ps_workspace_size(ps.PS_KEY_I32, True, n, True), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    best = None
    for rep in range(reps + 1):
        dk.copy_(k0)
        dv.copy_(v0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ps.ps_sort_segmented_ws(dk, dv, doff, ws, key_type=ps.PS_KEY_I32, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rep > 0:
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    batched_ms = best
    out_k, out_v = dk.clone(), dv.clone()
    # the same batch as one captured CUDA graph of the device-driven entry, replayed
    gk, gv = k0.clone(), v0.clone()
    wsg = torch.empty(ps.ps_workspace_size(ps.PS_KEY_I32, True, n, True), dtype=torch.uint8, device=dev)
    longest = int(np.diff(off).max())  # the batch's longest array, known to the caller
    ps.ps_sort_async_bounded_ws(gk, gv, wsg, longest, offsets=doff, key_type=ps.PS_KEY_I32, stream=stream)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ps.ps_sort_async_bounded_ws(gk, gv, wsg, longest, offsets=doff, key_type=ps.PS_KEY_I32)
    gbest = None
    for rep in range(reps + 1):
        gk.copy_(k0)
        gv.copy_(v0)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rep > 0:
            ms = e0.elapsed_time(e1)
            gbest = ms if gbest is None else min(gbest, ms)
    graph_identical = bool(torch.equal(out_k, gk)) and bool(torch.equal(out_v, gv)) and ps.ps_stream_status() == 0
    del graph, gk, gv, wsg
    # one plain ps_sort_ws per array on the same data (workspace sized for the largest array)
    dk.copy_(k0)
    dv.copy_(v0)
    sizes = np.diff(off)
    wsp = torch.empty(ps.ps_workspace_size(ps.PS_KEY_I32, True, int(sizes.max()), False), dtype=torch.uint8,
                      device=dev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for a, b in zip(off[:-1], off[1:]):
        ps.ps_sort_ws(dk[a:b], dv[a:b], wsp, key_type=ps.PS_KEY_I32, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = e0.elapsed_time(e1)
    identical = bool(torch.equal(out_k, dk)) and bool(torch.equal(out_v, dv))
    del ws, wsp, k0, v0, out_k, out_v
    return {"workload": f"{count} int32 arrays, sizes floor(2^U(8,20)), runs uniform in [1, 2*sqrt(size)], "
                        "uint32 payload", "keys": int(n), "segments": count,
            "batched_ms": batched_ms, "batched_gkeys_s": n / (batched_ms / 1e3) / 1e9,
            "plain_loop_ms": plain_ms, "plain_gkeys_s": n / (plain_ms / 1e3) / 1e9,
            "speedup": plain_ms / batched_ms, "identical_results": identical,
            "graph_ms": gbest, "graph_gkeys_s": n / (gbest / 1e3) / 1e9, "graph_identical_results": graph_identical,
            "merge_cost_roofline": {"M": M, "runs": int(an["runs"]), "bytes": M * 16, "ideal_ms": ideal_ms,
                                    "frac": ideal_ms / batched_ms, "graph_frac": ideal_ms / gbest,
                                    "peak_gbs": peak, "peak_kind": peak_kind},
            "level_pass_config": {"autotune": tune,
                                  "in_use": list(ps.ps_tune_get_for(ps.PS_KEY_I32, True, n, True))},
            "batched_entry": "ps_sort_segmented_ws (one call)",
            "graph_entry": "ps_sort_async_bounded_ws (device-driven, the batch's longest array as the bound) "
                           "captured once in a CUDA graph, replayed",
            "plain_entry": "ps_sort_ws per array"}


def measure_serving(ps, dev, nreq: int, loads=(0.5, 0.8, 1.0, 2.0)):
    """Poisson arrivals of float32 sort requests (sizes floor(2^U(10,24)), ~1% NaN/+-0, Pareto(1.5)
    runs, uint32 payload): continuous batching (SortServer, 64 GB budget) vs one request at a time
    through ps_sort_host, both from pinned host memory to pinned host memory."""
    import numpy as np
    import torch
    import workloads
    from paper_1805_04154_gb300.serve import SortServer, latency_stats
    rng = np.random.default_rng(SEED)
    reqs = []
    for i in range(nreq):
        m = int(2 ** rng.uniform(10, 24))
        k, v = workloads.pareto_f32(m, seed=SEED * 7919 + i, alpha=1.5, special_frac=0.01)
        reqs.append((torch.from_numpy(k.view(np.int32)).pin_memory(), torch.from_numpy(v.view(np.int32)).pin_memory()))
    total = sum(k.numel() for k, _ in reqs)
    # merge cost of every request's own tree (the work the served batches must do)
    M = 0
    for k, _ in reqs:
        M += int(ps.ps_analyze(k.to(dev), key_type=ps.PS_KEY_F32)["cost"])
    peak, peak_kind = _peaks()
    ideal_s = M * 8 * 2 / (peak * 1e9)
    outs = [(torch.empty_like(k, pin_memory=True), torch.empty_like(v, pin_memory=True)) for k, v in reqs]
    stream = torch.cuda.current_stream(dev)

    def plain_one(i):
        k, v = reqs[i]
        ok, ov = outs[i]
        ps.ps_sort_host_ptr(ps.PS_KEY_F32, k.data_ptr(), v.data_ptr(), ok.data_ptr(), ov.data_ptr(), k.numel(),
                            stream=stream)

    for i in range(min(3, nreq)):
        plain_one(i)
    t0 = time.perf_counter()
    for i in range(nreq):
        plain_one(i)
    plain_busy = time.perf_counter() - t0
    capacity = nreq / plain_busy  # requests per second of back-to-back plain launches
    # the served mode's own tuned entry: segmented sorts of a batch of the first requests packed
    # as the server packs them (outside the timing)
    pk = torch.cat([k for k, _ in reqs[:12]]).to(dev)
    pv = torch.cat([v for _, v in reqs[:12]]).to(dev)
    poff = torch.tensor(np.concatenate([[0], np.cumsum([k.numel() for k, _ in reqs[:12]])]), dtype=torch.int64,
                        device=dev)
    serve_tune = ps.ps_autotune_segmented(pk, pv, poff, key_type=ps.PS_KEY_F32)
    del pk, pv, poff
    srv_cfg = dict(budget_bytes=64 << 30, max_batch_keys=1 << 25, slots=3)
    warm = SortServer(ps.PS_KEY_F32, **srv_cfg)
    for i in range(min(4, nreq)):
        warm.submit(reqs[i][0], reqs[i][1], outs[i][0], outs[i][1])
    warm.drain(120)
    warm.close()
    out = {"workload": f"{nreq} float32 requests, sizes floor(2^U(10,24)), ~1% NaN/+-0 (totalOrder), "
                       "Pareto(1.5) runs, uint32 payload, Poisson arrivals", "keys": int(total),
           "plain_capacity_req_s": capacity, "plain_back_to_back_gkeys_s": total / plain_busy / 1e9,
           "level_pass_config": {"autotune": serve_tune, "batch_keys": int(sum(k.numel() for k, _ in reqs[:12]))},
           "merge_cost_roofline": {"M": M, "bytes": M * 16, "ideal_ms": ideal_s * 1e3, "peak_gbs": peak,
                                   "peak_kind": peak_kind, "plain_back_to_back_frac": ideal_s / plain_busy,
                                   "note": "frac = ideal device time of all merges / wall time of the whole "
                                           "trace; every request also crosses the host link twice"},
           "loads": {}}
    for load in loads:
        lam = load * capacity
        gaps = rng.exponential(1.0 / lam, size=nreq)
        arrivals = np.cumsum(gaps)
        # continuous batching
        srv = SortServer(ps.PS_KEY_F32, **srv_cfg)
        handles = []
        start = time.perf_counter()
        for i in range(nreq):
            wait = arrivals[i] - (time.perf_counter() - start)
            if wait > 0:
                time.sleep(wait)  # sleeping releases the GIL to the server's threads
            h = srv.submit(reqs[i][0], reqs[i][1], outs[i][0], outs[i][1])
            h.t_submit = start + arrivals[i]  # latency counts from the scheduled arrival
            handles.append(h)
        srv.drain(600)
        srv.close()
        sb = latency_stats(handles)
        sb["batches"] = srv.batches
        sb["merge_cost_roofline_frac"] = ideal_s / sb["wall_s"] if sb.get("wall_s") else None
        sb["server"] = {"slots": len(srv._free), "max_batch_keys": srv.cap, "held_bytes": srv.held_bytes}
        # sequential plain launches on the same arrival trace
        lat = []
        start = time.perf_counter()
        t_free = 0.0
        for i in range(nreq):
            wait = arrivals[i] - (time.perf_counter() - start)
            if wait > 0:
                time.sleep(wait)
            plain_one(i)
            lat.append(time.perf_counter() - start - arrivals[i])
        wall = time.perf_counter() - start
        lat = np.array(lat) * 1e3
        sp = {"keys_per_s": total / wall, "p50_ms": float(np.percentile(lat, 50)),
              "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "wall_s": wall,
              "merge_cost_roofline_frac": ideal_s / wall}
        out["loads"][str(load)] = {"arrival_rate_req_s": lam, "batched": sb, "plain": sp}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import workloads
    oracle.build()
    workloads.build()
    n_s = args.n
    keys, vals = _gen(n_s, SEED)
    for _ in range(args.warmup):
        oracle.powersort(keys, vals)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.powersort(keys, vals)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = n_s * args.steps / total / 1e9
    sample = f"one full n={n_s} input of the headline workload per step (the GPU arm's seed), oracle powersort (Alg. 2)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "sample_n": n_s, "same_config": n_s == args.n,
                       "parallelism": "replicas (reference runs on rank 0 only)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_1805_04154_gb300 import _build
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    import paper_1805_04154_gb300 as ps
    ps.load()
    import oracle

    n = args.n
    keys, vals = _gen(n, SEED + rank)
    eb = 8
    dk0 = torch.from_numpy(keys).to(dev)
    dv0 = torch.from_numpy(vals.view(np.int32)).to(dev)
    an = ps.ps_analyze(dk0, key_type=ps.PS_KEY_I32)
    # the library's autotuner picks the level-pass configuration on this input (outside the
    # timed region; the input is left unchanged)
    tune = None if args.no_tune else ps.ps_autotune(dk0, dv0, key_type=ps.PS_KEY_I32)
    M = an["cost"]
    lengths = np.diff(an["starts"]).astype(np.float64)
    H = float(-(lengths / n * np.log2(lengths / n)).sum())

    # one resident copy per step (each step sorts fresh data; inputs > L2)
    free, _ = torch.cuda.mem_get_info(dev)
    per_copy = n * eb
    wsb = ps.ps_workspace_size(ps.PS_KEY_I32, True, n)
    fit = max(1, int((free - wsb - (4 << 30)) // per_copy))
    ncopies = min(args.steps + args.warmup, fit)
    copies = [(dk0.clone(), dv0.clone()) for _ in range(ncopies)]
    workspace = torch.empty(wsb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(i):
        k, v = copies[i]
        ps.ps_sort_ws(k, v, workspace, key_type=ps.PS_KEY_I32, stream=stream)

    def restore(lo, hi):
        for i in range(lo, hi):
            copies[i][0].copy_(dk0)
            copies[i][1].copy_(dv0)

    # warm-up
    for w in range(args.warmup):
        step(w % ncopies)
    torch.cuda.synchronize(dev)
    restore(0, ncopies)
    torch.cuda.synchronize(dev)

    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if gpu_id and not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    time.sleep(0.15)

    # timed region: chunks of at most ncopies steps; restores happen between chunks, outside
    ps.ps_profile_enable(True)
    launches0 = ps.ps_launch_count()
    total_ms = 0.0
    done = 0
    while done < args.steps:
        chunk = min(ncopies, args.steps - done)
        if done > 0:
            restore(0, chunk)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(chunk):
            step(i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        total_ms += e0.elapsed_time(e1)
        done += chunk
    launches = ps.ps_launch_count() - launches0
    prof = ps.ps_profile_read()
    ps.ps_profile_enable(False)
    clocks = sampler.stop()
    assert ps.ps_stream_status() == 0, "device reported an error"

    # correctness of the timed outputs: the last copy is the unique stable sort of the input
    k, v = copies[(args.steps - 1) % ncopies]
    ok = check_sorted_device(k, v, dk0)
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(ws, n, args.steps, total_ms)

    peak, peak_kind = _peaks()
    mt = prof["level_pass"]
    achieved = (mt["bytes"] / (mt["ms"] / 1000.0) / 1e9) if mt["ms"] > 0 else None
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "level_pass_traffic.json")
    if os.path.exists(tpath):
        try:
            import hashlib
            with open(tpath) as f:
                tr = json.load(f)
            csrc = os.path.join(ROOT, "paper_1805_04154_gb300", "csrc")
            src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in tr.get("sources", []))
            cfg = ps.ps_tune_get_for(ps.PS_KEY_I32, True, n)
            same_cfg = list(tr.get("config", [])) == [int(cfg[0]), int(cfg[1])]
            if (src and same_cfg and tr.get("source_sha256") == hashlib.sha256(src).hexdigest()
                    and mt["launches"]):
                elems_per_launch = mt["bytes"] / (2 * eb) / mt["launches"]
                traffic = tr["dram_bytes_per_output_elem"] * elems_per_launch
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "kernel": "level_pass_kernel", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_kind": peak_kind,
                "launches": mt["launches"], "ms_total": mt["ms"], "algorithmic_bytes_total": mt["bytes"]}
    ideal_ms = M * eb * 2 / (peak * 1e9) * 1000.0
    merge_cost_roofline = {"M": int(M), "bytes_per_step": int(M * eb * 2), "ideal_ms": ideal_ms,
                           "frac": ideal_ms / ms_per_step, "nH": H * n, "peak_gbs": peak}
    stages_ms = {k2: round(v2["ms"] / args.steps, 4) for k2, v2 in prof.items()}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "key": "int32", "payload": "uint32",
                       "run_lengths": f"uniform [1, {int(2 * N_DEFAULT ** 0.5) if n == N_DEFAULT else int(2 * n ** 0.5)}]",
                       "desc_frac": 0.25, "seed": SEED,
                       "l2": "no flush: every step sorts its own resident 800 MB copy (> 129 MB L2)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roofline, "merge_cost_roofline": merge_cost_roofline,
            "plan": {"runs": int(an["runs"]), "merge_cost": int(M), "entropy_bits": H,
                     "max_leaf_depth": int(an["leaf_depth"].max())},
            "stages_ms_per_step": stages_ms, "gpu_launches": int(launches), "clocks": clocks,
            "level_pass_config": {"items_per_thread": ps.ps_tune_get_for(ps.PS_KEY_I32, True, n)[0],
                                  "stages": ps.ps_tune_get_for(ps.PS_KEY_I32, True, n)[1],
                                  "autotune": tune,
                                  "entries": {"plain, 2^24 <= n < 2^28 (headline)": tune}},
            "sorted_check": ok}

    # end to end through the C ABI with host buffers (pinned), every step H2D + sort + D2H:
    # ps_sort_host_ws on four streams with one caller-owned device buffer set each, so the
    # copy-in of one step, the sort of another and the copy-out of a third overlap (the way a
    # caller sorting a stream of host arrays uses it); HostSortPipeline (the package's wrapper
    # with copies in submission order) and the serial single-stream ps_sort_host are kept too
    if not args.no_e2e:
        del copies
        torch.cuda.empty_cache()
        copies = None
        hk_in = torch.from_numpy(keys).pin_memory()
        hv_in = torch.from_numpy(vals.view(np.int32)).pin_memory()
        depth = 4
        outs = [(torch.empty_like(hk_in).pin_memory(), torch.empty_like(hv_in).pin_memory()) for _ in range(depth)]
        e2e_steps = max(4 * depth, min(args.steps, 24))
        sets = [(torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
                 torch.empty(wsb, dtype=torch.uint8, device=dev), torch.cuda.Stream(dev)) for _ in range(depth)]

        def abi_step(i):
            q = i % depth
            kd, vd, wd, st_ = sets[q]
            ps.ps_sort_host_ws(ps.PS_KEY_I32, hk_in.data_ptr(), hv_in.data_ptr(), outs[q][0].data_ptr(),
                               outs[q][1].data_ptr(), n, kd, vd, wd, stream=st_)

        def timed_loop(submit, streams, count):
            """Median of three repetitions (the host link is shared with the machine's other GPUs,
            so single runs vary); events on the first stream, the others joined to it."""
            reps_ms = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(streams[0])
                for st_ in streams[1:]:
                    st_.wait_event(e0)
                for i in range(count):
                    submit(i)
                for st_ in streams[1:]:
                    ev = torch.cuda.Event()
                    ev.record(st_)
                    streams[0].wait_event(ev)
                e1.record(streams[0])
                torch.cuda.synchronize(dev)
                reps_ms.append(max_over_ranks(e0.elapsed_time(e1), dist, dev))
            return sorted(reps_ms)[1], reps_ms

        for i in range(depth):
            abi_step(i)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        launches_e2e0 = ps.ps_launch_count()
        e2e_ms, reps_ms = timed_loop(abi_step, [st_ for (_, _, _, st_) in sets], e2e_steps)
        e2e_launches = (ps.ps_launch_count() - launches_e2e0) // (3 * e2e_steps)
        assert ps.ps_stream_status() == 0, "device reported an error"
        ok_e2e = all(check_sorted_device(o[0].to(dev), o[1].to(dev), dk0) for o in outs)
        del sets
        torch.cuda.empty_cache()
        # the package's HostSortPipeline over the same C-ABI sort
        from paper_1805_04154_gb300.pipeline import HostSortPipeline
        pipe = HostSortPipeline(n, torch.int32, True, depth=depth, device=dev)

        def pipe_step(i):
            q = i % depth
            pipe.submit(hk_in, hv_in, outs[q][0], outs[q][1])

        for i in range(depth):
            pipe_step(i)
        pipe.synchronize()
        torch.cuda.synchronize(dev)
        pipe_ms, pipe_reps = timed_loop(pipe_step, [st_ for (_, _, _, st_) in pipe._sets], e2e_steps)
        pipe.synchronize()
        del pipe
        torch.cuda.empty_cache()
        # serial: one ps_sort_host call at a time (synchronous, pool workspace)
        hk_out, hv_out = outs[0]
        ps.ps_sort_host_ptr(ps.PS_KEY_I32, hk_in.data_ptr(), hv_in.data_ptr(), hk_out.data_ptr(),
                            hv_out.data_ptr(), n, stream=stream)
        torch.cuda.synchronize(dev)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        serial_steps = 3
        for _ in range(serial_steps):
            ps.ps_sort_host_ptr(ps.PS_KEY_I32, hk_in.data_ptr(), hv_in.data_ptr(), hk_out.data_ptr(),
                                hv_out.data_ptr(), n, stream=stream)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        serial_ms = s0.elapsed_time(s1) / serial_steps
        line["e2e"] = {"value": replica_throughput(ws, n, e2e_steps, e2e_ms), "unit": UNIT,
                       "h2d_bytes_per_step": n * eb, "d2h_bytes_per_step": n * eb, "steps": e2e_steps,
                       "ms_per_step": e2e_ms / e2e_steps,
                       "repetitions_ms_per_step": [x / e2e_steps for x in reps_ms],
                       "entry": "ps_sort_host_ws (C ABI; pinned host buffers, 4 streams with one caller-owned "
                                "device buffer set each; copy-in, device-driven sort and copy-out per call)",
                       "gpu_launches_per_step": int(e2e_launches),
                       "pipeline": {"entry": "HostSortPipeline (4 arrays in flight, copies in each direction in "
                                             "submission order)", "ms_per_step": pipe_ms / e2e_steps,
                                    "value": replica_throughput(ws, n, e2e_steps, pipe_ms),
                                    "repetitions_ms_per_step": [x / e2e_steps for x in pipe_reps]},
                       "serial": {"entry": "ps_sort_host (one call at a time)", "ms_per_step": serial_ms,
                                  "value": n / (serial_ms / 1000.0) / 1e9},
                       "sorted_check": ok_e2e}
        del outs
        torch.cuda.empty_cache()

    if rank == 0 and ws == 1 and not args.no_variants:
        import workloads
        copies = None
        torch.cuda.empty_cache()
        var = []
        hk, hv = _gen(n, SEED)
        var.append(measure_variant(ps, dev, "peeksort merge tree (Alg. 1) on the headline workload", hk, hv, 0,
                                   tree=1))
        del hk, hv
        pk, pv = workloads.perm_i32(n, seed=SEED)
        var.append(measure_variant(ps, dev, f"random permutation, n={n} int32 + uint32 (runs ~2.4)", pk, pv, 0))
        var.append(measure_variant(ps, dev, f"random permutation, n={n}, runs extended to 24 (Sec. 5.1)", pk, pv, 0,
                                   min_run=24))
        del pk, pv
        rk, rv = workloads.random_runs_i32(10 ** 7, seed=SEED, mean_len=3000)
        var.append(measure_variant(ps, dev, "paper random-runs: n=1e7, geometric run lengths, mean 3000", rk, rv, 0))
        var.append(measure_variant(ps, dev, "paper random-runs: n=1e7, mean 3000, runs extended to 24 (Sec. 5.1)",
                                   rk, rv, 0, min_run=24))
        uk, uv = workloads.pareto_u64(n, seed=SEED, alpha=1.2, distinct=1000, max_len=n // 10)
        var.append(measure_variant(ps, dev, f"uint64 keys from 1000 values, Pareto(1.2) runs, n={n} + uint32", uk, uv, 2))
        del uk, uv
        line["variants"] = var
        torch.cuda.empty_cache()
        copies = None
    if rank == 0 and ws == 1 and not args.no_batched:
        copies = None
        torch.cuda.empty_cache()
        line["batched"] = measure_batched(ps, dev, args.batched_segments)
        torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_serving:
        line["serving"] = measure_serving(ps, dev, args.serving_requests)
        torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(keys, vals, f"one full n={n} input of the same workload, "
                                                         "oracle powersort (Alg. 2), single thread")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--n", type=int, default=N_DEFAULT, help="array size (default 1e8)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default level-pass configuration")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 10,000-array batched measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the other single-array workloads")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--batched-segments", type=int, default=10000)
    ap.add_argument("--serving-requests", type=int, default=300)
    ap.add_argument("--once", choices=["runs", "perm", "runs_minrun24", "perm_minrun24", "u64"], default=None,
                    help="profiling driver: exactly one sort of the headline (runs), permutation or uint64 "
                         "Pareto(1.2) workload (*_minrun24: runs extended to 24) at --n, no warm-up, no JSON line")
    ap.add_argument("--l2-sweep", action="store_true",
                    help="measurement of the L2 against HBM: a streaming copy kernel over buffer pairs of "
                         "4 MB .. 2 GB, and the level passes of sorts of 2^20 .. 2^24 headline-like keys; "
                         "one JSON line, nothing else")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.once:
        return run_once(args)
    if args.l2_sweep:
        return run_l2_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


# Streaming copy for the L2 sweep: every thread copies its own fixed 16-byte words from one
# buffer to the other and back, `iters` times, with L2-only (.cg) loads and stores and no
# dependence between threads, so the rate is the memory system's, not a synchronisation's.
_PINGPONG_CU = r"""
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ uint4 ldcg(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ void stcg(uint4* p, uint4 v) {
  asm volatile("st.global.cg.v4.u32 [%0], {%1,%2,%3,%4};" :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}
__global__ void pingpong(uint4* a, uint4* b, long long n16, int iters) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
    const uint4* src = (it & 1) ? b : a;
    uint4* dst = (it & 1) ? a : b;
    for (long long i = t0; i < n16; i += stride) {
      uint4 v = ldcg(src + i);
      v.x += 1u;
      stcg(dst + i, v);
    }
  }
}
extern "C" int pingpong_launch(void* a, void* b, long long n16, int iters, int grid, void* stream) {
  pingpong<<<grid, 256, 0, (cudaStream_t)stream>>>((uint4*)a, (uint4*)b, n16, iters);
  return (int)cudaGetLastError();
}
"""


def run_l2_sweep(args):
    """L2 against HBM on this GPU: the streaming rate for buffer pairs that fit the 129 MB L2 or
    not, and what the level passes reach on arrays whose two buffers fit it."""
    import ctypes
    import tempfile
    import numpy as np
    import torch
    import workloads
    from paper_1805_04154_gb300 import _build
    _build.build()
    import paper_1805_04154_gb300 as ps
    ps.load()
    tmp = tempfile.mkdtemp()
    src, so = os.path.join(tmp, "pingpong.cu"), os.path.join(tmp, "pingpong.so")
    with open(src, "w") as f:
        f.write(_PINGPONG_CU)
    subprocess.check_call([_build._nvcc(), *_build.ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC", src, "-o", so])
    lib = ctypes.CDLL(so)
    lib.pingpong_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p]
    s = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    copy = []
    for mb in (4, 8, 16, 32, 48, 64, 96, 128, 512, 2048):
        nb = mb << 20
        a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        iters = max(2, min(4000, int(0.02 * 6e12 / (2 * nb))))  # about 20 ms of copying
        best = 0.0
        for grid in (sms * 4, sms * 8):
            assert lib.pingpong_launch(a.data_ptr(), b.data_ptr(), nb // 16, 2, grid, s.cuda_stream) == 0
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            assert lib.pingpong_launch(a.data_ptr(), b.data_ptr(), nb // 16, iters, grid, s.cuda_stream) == 0
            e1.record(s)
            torch.cuda.synchronize()
            best = max(best, 2 * nb * iters / e0.elapsed_time(e1) / 1e6)
        copy.append({"mb_per_buffer": mb, "gbs": round(best, 1)})
        del a, b
    sorts = []
    for n in (1 << 20, 1 << 22, 1 << 24, N_DEFAULT):
        keys, vals = workloads.runs_i32(n, SEED, max_len=2 * int(N_DEFAULT ** 0.5))
        dk0 = torch.from_numpy(keys).cuda()
        dv0 = torch.from_numpy(vals.view(np.int32)).cuda()
        ws = torch.empty(ps.ps_workspace_size(ps.PS_KEY_I32, True, n), dtype=torch.uint8, device="cuda")
        dk, dv = dk0.clone(), dv0.clone()
        reps = 10
        for i in range(reps + 3):
            if i == 3:
                torch.cuda.synchronize()
                ps.ps_profile_enable(True)
            dk.copy_(dk0)
            dv.copy_(dv0)
            ps.ps_sort_ws(dk, dv, ws, key_type=ps.PS_KEY_I32)
        torch.cuda.synchronize()
        prof = ps.ps_profile_read()["level_pass"]
        ps.ps_profile_enable(False)
        sorts.append({"n": n, "working_set_mb": round(2 * n * 8 / 2 ** 20, 1), "level_passes": prof["launches"] // reps,
                      "level_ms": round(prof["ms"] / reps, 4), "gbs": round(prof["bytes"] / prof["ms"] / 1e6, 1)})
        del dk0, dv0, dk, dv, ws
        torch.cuda.empty_cache()
    print(json.dumps({"l2_sweep": {"copy": copy, "level_pass": sorts, "peak_hbm_gbs": _peaks()[0],
                                   "note": "copy: best of grids 4 and 8 CTAs per SM, read + write bytes; "
                                           "level_pass: algorithmic bytes of all level passes / their CUDA-event time"}}))
    return 0


def run_once(args):
    """One sort and nothing else, so that a profiler's launch list is exactly one pipeline."""
    import numpy as np
    import torch
    import workloads
    from paper_1805_04154_gb300 import _build
    _build.build()
    import paper_1805_04154_gb300 as ps
    ps.load()
    n = args.n
    kt = ps.PS_KEY_I32
    if args.once == "u64":
        keys, vals = workloads.pareto_u64(n, seed=SEED, alpha=1.2, distinct=1000, max_len=n // 10)
        kt = ps.PS_KEY_U64
        dk = torch.from_numpy(keys.view(np.int64)).cuda()
    else:
        keys, vals = _gen(n, SEED) if args.once.startswith("runs") else workloads.perm_i32(n, seed=SEED)
        dk = torch.from_numpy(keys).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    orig = dk.clone()
    ws = torch.empty(ps.ps_workspace_size(kt, True, n), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    ps.ps_profile_enable(True)
    if args.once.endswith("_minrun24"):
        ps.ps_sort_minrun_ws(dk, dv, ws, 24, key_type=kt)
    else:
        ps.ps_sort_ws(dk, dv, ws, key_type=kt)
    torch.cuda.synchronize()
    prof = ps.ps_profile_read()
    ps.ps_profile_enable(False)
    if kt == ps.PS_KEY_U64:  # signed tensor view of unsigned keys: compare in the key order
        dk, orig = dk ^ (-(1 << 63)), orig ^ (-(1 << 63))
    ok = ps.ps_stream_status() == 0 and check_sorted_device(dk, dv, orig)
    lp = prof["level_pass"]
    stages = {k2: round(v2["ms"], 4) for k2, v2 in prof.items() if v2["launches"]}
    print(f"once {args.once} n={n} sorted={ok} level_pass_launches={lp['launches']} "
          f"level_pass_outputs={lp['bytes'] // (2 * (keys.dtype.itemsize + 4))} "
          f"config={ps.ps_tune_get(kt, True)} stages_ms={stages}")
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
