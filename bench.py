#!/usr/bin/env python3
"""Benchmark of the trace-analysis hot path on B300.

One step = one pass of the whole path over one trace set resident in HBM:
ingest (validate, durations, iteration cut, the rank x iteration x context
tensor, exclusive and inclusive per-rank CSR), cross-rank statistics with
outliers over every context, the rack rollup of a communication context, and
the potential-speedup estimate over the iteration program's contexts.

Prints one JSON line (see --help).  ``--impl reference`` times the CPU oracle
(the plain single-threaded definition) on a bounded sample of the same
workload instead.
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trace records/s & HBM GB/s vs peak (batched vs plain); query p50/p99 latency"
WORKLOADS = {
    1: "plain: R=64 ranks x 20k samples, C=200, I=10, 2 ranks slowed 1.5x",
    2: "plain: R=4096 ranks, C=5000 (depth<=24), lognormal lengths mean 100k sigma 0.5, I=50, "
       "jitter 5%, 1% of ranks 1.2-2x on random iterations",
    3: "plain at scale: R=100,000 ranks, C=20,000, lognormal lengths mean 20k sigma 0.7 "
       "(~2e9 records), I=100, 12 ranks/node, 22 racks, 3 racks 1.3x slower in communication "
       "contexts",
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------- workload --
def make_workload(preset: int, seed: int = 1, pinned: bool = True, ranks: int = 0):
    """Generate the synthetic trace set on the host (pinned memory)."""
    import torch
    from paper_2605_03561_b300 import synth
    cfg = synth.preset(preset, seed=seed)
    if ranks:
        cfg.n_ranks = ranks
    rank_off, parent, info = synth.plan(cfg)
    N = int(rank_off[-1])
    t0 = time.time()
    ts = torch.empty(N, dtype=torch.uint64, pin_memory=pinned)
    cx = torch.empty(N, dtype=torch.uint32, pin_memory=pinned)
    synth.fill(cfg, rank_off, 0, cfg.n_ranks, ts.data_ptr(), cx.data_ptr(), 0)
    log(f"generated {N} records in {time.time() - t0:.1f} s")
    truth = synth.truth(cfg, info)
    topo = synth.topology(cfg, info)
    return dict(cfg=cfg, info=info, rank_off=rank_off, parent=parent, ts=ts, ctx=cx, N=N,
                marker=cfg.marker_ctx, truth=truth, topo=topo)


BATCHED = ("batched: 256 independent trace sets, ranks per set lognormal (median 362, sigma "
           "1.04) in 16..8192, C log-uniform in 100..10,000, trace lengths lognormal (mean 30k, "
           "sigma 1.0), I=50, jitter 5%, 1% of ranks 1.2-2x on random iterations; per set: "
           "tensor, exclusive, inclusive, statistics, potential speedup over its iteration "
           "program, rack rollup of a communication context")
SET_ALIGN = 32  # samples; every set of the input arena starts 16-byte aligned


def batch_shapes(n_sets: int, seed: int):
    """Per-set rank and context counts of the batched workload."""
    rng = np.random.default_rng(seed)
    R = np.clip(np.rint(np.exp(np.log(362.0) + 1.04 * rng.standard_normal(n_sets))), 16, 8192)
    Cn = np.rint(np.exp(rng.uniform(np.log(100.0), np.log(10000.0), n_sets)))
    return R.astype(np.int64), Cn.astype(np.int64)


def make_batch_workload(n_sets: int, seed: int, device: str, scale: float = 1.0):
    """Generate every set into one device arena (aligned per set) through a
    pinned staging buffer; returns per-set host metadata and device views."""
    import torch
    from paper_2605_03561_b300 import synth
    R, Cn = batch_shapes(n_sets, seed)
    sets, starts, total = [], [], 0
    for k in range(n_sets):
        cfg = synth.preset(2, seed=seed * 1000 + k, n_ranks=int(max(16, R[k] * scale)),
                           n_ctx=int(Cn[k]), len_mean=30000.0, len_sigma=1.0,
                           n_segments=int(min(64, Cn[k] - 2)))
        rank_off, parent, info = synth.plan(cfg)
        truth = synth.truth(cfg, info)
        segs = np.unique(truth["segment_ctx"]).astype(np.uint32)
        comm = truth["segment_ctx"][truth["comm_segment"].astype(bool)]
        sets.append(dict(cfg=cfg, rank_off=rank_off, parent=parent, marker=cfg.marker_ctx,
                         N=int(rank_off[-1]), kset=segs, topo=synth.topology(cfg, info),
                         topo_ctx=int(comm[0]) if len(comm) else int(segs[0])))
        starts.append(total)
        total += (int(rank_off[-1]) + SET_ALIGN - 1) // SET_ALIGN * SET_ALIGN
    t0 = time.time()
    d_ts = torch.empty(max(total, 1), dtype=torch.uint64, device=device)
    d_cx = torch.empty(max(total, 1), dtype=torch.uint32, device=device)
    big = max(x["N"] for x in sets)
    h_ts = torch.empty(max(big, 1), dtype=torch.uint64, pin_memory=True)
    h_cx = torch.empty(max(big, 1), dtype=torch.uint32, pin_memory=True)
    for x, a in zip(sets, starts):
        n = x["N"]
        synth.fill(x["cfg"], x["rank_off"], 0, x["cfg"].n_ranks, h_ts.data_ptr(), h_cx.data_ptr(), 0)
        d_ts[a:a + n].copy_(h_ts[:n])
        d_cx[a:a + n].copy_(h_cx[:n])
        torch.cuda.synchronize()
        x["ts"], x["ctx"] = d_ts[a:a + n], d_cx[a:a + n]
        x["d_rank_off"] = torch.from_numpy(x["rank_off"]).to(device)
        x["d_parent"] = torch.from_numpy(x["parent"]).to(device)
    log(f"generated {len(sets)} sets, {sum(x['N'] for x in sets)} records in "
        f"{time.time() - t0:.1f} s")
    return sets, (d_ts, d_cx)


def analysis_args(w):
    segs = np.unique(w["truth"]["segment_ctx"]).astype(np.uint32)
    comm = w["truth"]["segment_ctx"][w["truth"]["comm_segment"].astype(bool)]
    return dict(kset=segs, topo_ctx=int(comm[0]) if len(comm) else int(segs[0]))


# ------------------------------------------------------- device-side calls --
class DeviceCalls:
    """ta_context_stats / ta_topology_rollup / ta_potential_speedup with every
    output in preallocated device buffers (no host copies inside the step)."""

    def __init__(self, ta, w, args, device=0):
        import torch
        self.ta, self.torch = ta, torch
        dev = f"cuda:{device}"
        C_ = len(w["parent"])
        topo = w["topo"]
        self.nn, self.nc, self.nr = int(topo["n_nodes"]), int(topo["n_chassis"]), int(topo["n_racks"])
        self.stats = torch.empty(C_ * C.sizeof(ta.CtxStats), dtype=torch.uint8, device=dev)
        self.outlier_cap = 1 << 20
        self.outliers = torch.empty(self.outlier_cap * C.sizeof(ta.Outlier), dtype=torch.uint8,
                                    device=dev)
        self.node = torch.from_numpy(topo["node_of_rank"]).to(dev)
        self.rack = torch.from_numpy(topo["rack_of_node"]).to(dev)
        self.chassis = torch.from_numpy(topo["chassis_of_node"]).to(dev)
        u32, u64 = torch.uint32, torch.uint64
        self.o = {k: torch.empty(n, dtype=t, device=dev) for k, n, t in [
            ("node_outliers", self.nn, u32), ("node_sum", self.nn, u64), ("node_ranks", self.nn, u32),
            ("node_flag", self.nn, torch.uint8), ("chassis_flagged", self.nc, u32),
            ("chassis_nodes", self.nc, u32), ("chassis_sum", self.nc, u64),
            ("rack_flagged", self.nr, u32), ("rack_nodes", self.nr, u32),
            ("rack_sum", self.nr, u64), ("flagged_racks", self.nr, u32)]}
        self.kset = torch.from_numpy(args["kset"]).to(dev)
        self.nk = len(args["kset"])
        self.per = torch.empty(self.nk * C.sizeof(ta.SpeedupCtx), dtype=torch.uint8, device=dev)
        self.tot = torch.empty(C.sizeof(ta.SpeedupTotal), dtype=torch.uint8, device=dev)
        self.topo_ctx = args["topo_ctx"]

    def run(self, e):
        ta = self.ta
        a = ta.StatsArgs()
        a.metric, a.mem_kind, a.tau_num, a.tau_den = ta.EXCLUSIVE, ta.MEM_DEVICE, 3, 1
        o = ta.StatsOut()
        o.stats, o.outliers, o.outlier_cap = self.stats.data_ptr(), self.outliers.data_ptr(), self.outlier_cap
        ta._check(ta.lib().ta_context_stats(e.h, C.byref(a), C.byref(o)))
        t = ta.Topology()
        t.n_nodes, t.n_chassis, t.n_racks, t.mem_kind = self.nn, self.nc, self.nr, ta.MEM_DEVICE
        t.node_of_rank, t.rack_of_node, t.chassis_of_node = (
            self.node.data_ptr(), self.rack.data_ptr(), self.chassis.data_ptr())
        ta_ = ta.TopoArgs()
        ta_.metric, ta_.ctx, ta_.tau_num, ta_.tau_den, ta_.min_ranks = ta.EXCLUSIVE, self.topo_ctx, 2, 1, 1
        to = ta.TopoOut()
        to.mem_kind = ta.MEM_DEVICE
        for k, v in self.o.items():
            setattr(to, k, v.data_ptr())
        ta._check(ta.lib().ta_topology_rollup(e.h, C.byref(t), C.byref(ta_), C.byref(to)))
        sa = ta.SpeedupArgs()
        sa.mem_kind, sa.n_ctxs, sa.ctxs = ta.MEM_DEVICE, self.nk, self.kset.data_ptr()
        so = ta.SpeedupOut()
        so.per_ctx, so.total = self.per.data_ptr(), self.tot.data_ptr()
        ta._check(ta.lib().ta_potential_speedup(e.h, C.byref(sa), C.byref(so)))
        return int(o.n_outliers)


def host_calls(e, w, args):
    """The same three calls with host outputs (the user-facing e2e form)."""
    topo = w["topo"]
    st, outl, n_out, _ = e.stats(0, tau=(3, 1))
    tp = e.topology(args["topo_ctx"], topo["node_of_rank"], topo["rack_of_node"],
                    topo["chassis_of_node"], topo["n_racks"], topo["n_chassis"], tau=(2, 1))
    sp = e.speedup(args["kset"])
    C_ = len(w["parent"])
    nn, nc, nr = topo["n_nodes"], topo["n_chassis"], topo["n_racks"]
    d2h = (C_ * C.sizeof(__import__("paper_2605_03561_b300").CtxStats) + n_out * 16 +
           nn * (4 + 8 + 4 + 1) + nc * 16 + nr * 20 + len(args["kset"]) * 88 + 48)
    return d2h


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.lines = []  # (arrival time, csv line)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=5.0):
        """Block until nvidia-smi has produced its first sample."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.02)

    def mark(self):
        return time.perf_counter()

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken between t0 and t1 (perf_counter)."""
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if (t0 is not None and ts < t0) or (t1 is not None and ts > t1 + 0.25):
                continue
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- replicas --
def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's time: N independent replicas (weak scaling) finish
    when the slowest does.  Needs an initialised process group when world > 1."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def aggregate_rate(world: int, units_per_rank: int, steps: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank * steps / (ms / 1000.0)


# --------------------------------------------------------------- baselines --
def oracle_sample(w, n_ranks, args):
    """Run the oracle on ranks [0, n_ranks) of the workload; returns (records, s)."""
    import oracle
    ro = w["rank_off"][: n_ranks + 1].copy()
    n = int(ro[-1])
    ts = w["ts"][:n].numpy()
    cx = w["ctx"][:n].numpy()
    tr = oracle.Traces(ro, ts, cx, w["parent"], w["marker"])
    topo = w["topo"]
    node = topo["node_of_rank"][:n_ranks]
    nn = int(node.max()) + 1
    t0 = time.perf_counter()
    a = oracle.Analysis(tr)
    a.stats(0, tau=(3, 1))
    a.topology(args["topo_ctx"], node, topo["rack_of_node"][:nn], topo["chassis_of_node"][:nn],
               topo["n_racks"], topo["n_chassis"], tau=(2, 1))
    a.speedup(args["kset"])
    return n, time.perf_counter() - t0


def oracle_sample_threads(w, n_ranks, args, n_threads):
    """The same oracle path split over ranks: n_threads contiguous rank ranges
    of [0, n_ranks), each analysed whole (tensor, exclusive, inclusive,
    statistics, rack rollup, speedup over its own ranks) in its own thread
    (the oracle's calls release the GIL); returns (records, wall s)."""
    import threading
    import oracle
    ro_all = w["rank_off"][: n_ranks + 1]
    n = int(ro_all[-1])
    bounds = [int(np.searchsorted(ro_all, n * i // n_threads)) for i in range(n_threads)]
    bounds = sorted(set([0] + bounds[1:] + [n_ranks]))
    topo = w["topo"]
    jobs = []
    for r0, r1 in zip(bounds[:-1], bounds[1:]):
        if r1 <= r0:
            continue
        a, b = int(ro_all[r0]), int(ro_all[r1])
        ro = (ro_all[r0:r1 + 1] - ro_all[r0]).astype(np.uint64)
        tr = oracle.Traces(ro, w["ts"][a:b].numpy(), w["ctx"][a:b].numpy(), w["parent"], w["marker"])
        node = topo["node_of_rank"][r0:r1].astype(np.int64)
        n_lo = int(node.min())
        nn = int(node.max()) - n_lo + 1
        jobs.append((tr, (node - n_lo).astype(np.uint32), topo["rack_of_node"][n_lo:n_lo + nn],
                     topo["chassis_of_node"][n_lo:n_lo + nn]))

    def work(tr, node, rack, chassis):
        a = oracle.Analysis(tr)
        a.stats(0, tau=(3, 1))
        a.topology(args["topo_ctx"], node, rack, chassis, topo["n_racks"], topo["n_chassis"],
                   tau=(2, 1))
        a.speedup(args["kset"])

    threads = [threading.Thread(target=work, args=j) for j in jobs]
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    return n, time.perf_counter() - t0, len(jobs)


def host_info():
    """The host's thread count and CPU model (for the CPU baselines)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


# Both CPU legs (the reference arm and the bench line's cpu_baseline) time the
# oracle on the same sample: the ranks holding the first SAMPLE_RECORDS records.
SAMPLE_RECORDS = 2e7


def pick_sample(w, target_records):
    ro = w["rank_off"]
    k = int(np.searchsorted(ro, target_records))
    return max(1, min(k, len(ro) - 1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0}, "fallback"


def committed_traffic(preset):
    """Per-launch DRAM traffic of the tensor kernel from a committed ncu
    summary, if the kernel source is unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "k_tensor_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except OSError:
        return None
    src = os.path.join(ROOT, "paper_2605_03561_b300", "csrc", "tensor.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if d.get("tensor_cu_sha256_16") != h:
        return None
    return d.get("per_record_bytes")


# ------------------------------------------ more plain workloads, timed --
def device_workload(preset, seed=1, ranks=0, **overrides):
    """A generated trace set resident on the device (host copy dropped)."""
    import torch
    from paper_2605_03561_b300 import synth
    cfg = synth.preset(preset, seed=seed, **overrides)
    if ranks:
        cfg.n_ranks = ranks
    rank_off, parent, info = synth.plan(cfg)
    N = int(rank_off[-1])
    ts = torch.empty(N, dtype=torch.uint64, pin_memory=True)
    cx = torch.empty(N, dtype=torch.uint32, pin_memory=True)
    synth.fill(cfg, rank_off, 0, cfg.n_ranks, ts.data_ptr(), cx.data_ptr(), 0)
    w = dict(cfg=cfg, info=info, rank_off=rank_off, parent=parent, N=N, marker=cfg.marker_ctx,
             truth=synth.truth(cfg, info), topo=synth.topology(cfg, info))
    w["d_ro"] = torch.from_numpy(rank_off).cuda()
    w["d_par"] = torch.from_numpy(parent).cuda()
    w["d_ts"] = ts.cuda()
    w["d_cx"] = cx.cuda()
    torch.cuda.synchronize()
    return w


def tensor_roofline(prof, R, peak):
    """The write pass's algorithmic bytes per launch over its event time."""
    n_l = max(1, prof["tensor_launches"])
    t = prof["tensor_ms"] / n_l / 1000.0
    alg = (12 * prof["tensor_records"] + 16 * prof["tensor_entries"] + 8 * prof["tensor_rows"]
           + 8 * (R + 1) * prof["tensor_launches"]) / n_l
    return {"ms_per_launch": t * 1e3, "achieved_gbs": alg / t / 1e9,
            "frac": alg / t / 1e9 / peak, "alg_bytes_per_launch": alg}


def run_plain_config(ctx, w, steps, warmup, peak, stream, device=0):
    """The whole step (ingest + statistics + rack rollup + speedup) on a
    device-resident workload, timed with CUDA events on the library stream."""
    import torch
    import paper_2605_03561_b300 as ta
    aa = analysis_args(w)
    calls = DeviceCalls(ta, w, aa, device)
    R = len(w["rank_off"]) - 1

    def step():
        e = ctx.load(w["d_ro"], w["d_ts"], w["d_cx"], w["d_par"], w["marker"], borrow=True)
        calls.run(e)
        e.free()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ctx.profile(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    prof = ctx.profile(reset=True)
    out = {"records": w["N"], "ranks": R, "ms_per_step": ms,
           "records_per_s": w["N"] / (ms / 1e3), "steps": steps,
           "phase_ms_per_step": {k: prof[k] / steps for k in
                                 ("tensor_count_ms", "tensor_ms", "exclusive_ms",
                                  "inclusive_ms", "stats_ms", "topology_ms", "speedup_ms")},
           "tensor_write": tensor_roofline(prof, R, peak)}
    del calls
    return out


def run_shuffled(ctx, ranks, steps, peak):
    """The tensor passes on the plain-at-scale generator cut to `ranks` ranks,
    as generated (consecutive iterations repeat their run sequence) and with
    every iteration's segments in a fresh random order (no row repeats the
    previous row's runs, so the write pass's template path never applies):
    load time and the write pass's roofline for both."""
    import torch
    out = {"ranks": ranks}
    for name, shuffle in (("repeating", 0), ("shuffled", 1)):
        w = device_workload(3, ranks=ranks, shuffle_segments=shuffle)
        R = len(w["rank_off"]) - 1
        for _ in range(2):
            ctx.load(w["d_ro"], w["d_ts"], w["d_cx"], w["d_par"], w["marker"], borrow=True).free()
        torch.cuda.synchronize()
        ctx.profile(reset=True)
        t0 = time.perf_counter()
        for _ in range(steps):
            ctx.load(w["d_ro"], w["d_ts"], w["d_cx"], w["d_par"], w["marker"], borrow=True).free()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / steps
        prof = ctx.profile(reset=True)
        out[name] = {"records": w["N"], "load_ms": wall * 1e3,
                     "records_per_s_load": w["N"] / wall,
                     "tensor_count_ms": prof["tensor_count_ms"] / steps,
                     "tensor_write": tensor_roofline(prof, R, peak)}
        del w
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------ batched vs plain --
def run_batched(args, ctx, local):
    """The batched form (one graph replay over every set) against plain
    per-experiment calls on the same device-resident sets, same products:
    tensor, exclusive, inclusive, statistics of the exclusive metric over all
    ranks and contexts (tau = 3) with outliers, the potential speedup over
    each set's iteration-program contexts and the rack rollup of one of its
    communication contexts (tau = 2)."""
    import torch
    import paper_2605_03561_b300 as ta
    dev = f"cuda:{local}"
    sets, arena = make_batch_workload(args.batch_sets, 7, dev, args.batch_scale)
    N = sum(x["N"] for x in sets)
    R = sum(len(x["rank_off"]) - 1 for x in sets)
    stream = ctx.stream
    cmax = max(len(x["parent"]) for x in sets)
    st = torch.empty(cmax * C.sizeof(ta.CtxStats), dtype=torch.uint8, device=dev)
    cap = 1 << 20
    ol = torch.empty(cap * C.sizeof(ta.Outlier), dtype=torch.uint8, device=dev)

    nkmax = max(len(x["kset"]) for x in sets)
    per = torch.empty(nkmax * C.sizeof(ta.SpeedupCtx), dtype=torch.uint8, device=dev)
    tot = torch.empty(C.sizeof(ta.SpeedupTotal), dtype=torch.uint8, device=dev)
    nnmax = max(int(x["topo"]["n_nodes"]) for x in sets)
    ncmax = max(int(x["topo"]["n_chassis"]) for x in sets)
    nrmax = max(int(x["topo"]["n_racks"]) for x in sets)
    tout = {k: torch.empty(n * w, dtype=torch.uint8, device=dev) for k, n, w in [
        ("node_outliers", nnmax, 4), ("node_sum", nnmax, 8), ("node_ranks", nnmax, 4),
        ("node_flag", nnmax, 1), ("chassis_flagged", ncmax, 4), ("chassis_nodes", ncmax, 4),
        ("chassis_sum", ncmax, 8), ("rack_flagged", nrmax, 4), ("rack_nodes", nrmax, 4),
        ("rack_sum", nrmax, 8), ("flagged_racks", nrmax, 4)]}
    for x in sets:
        x["d_kset"] = torch.from_numpy(x["kset"]).to(dev)
        x["d_topo"] = [torch.from_numpy(x["topo"][k]).to(dev)
                       for k in ("node_of_rank", "rack_of_node", "chassis_of_node")]

    def plain_step():
        for x in sets:
            e = ctx.load(x["d_rank_off"], x["ts"], x["ctx"], x["d_parent"], x["marker"],
                         borrow=True)
            a = ta.StatsArgs()
            a.metric, a.mem_kind, a.tau_num, a.tau_den = ta.EXCLUSIVE, ta.MEM_DEVICE, 3, 1
            o = ta.StatsOut()
            o.stats, o.outliers, o.outlier_cap = st.data_ptr(), ol.data_ptr(), cap
            ta._check(ta.lib().ta_context_stats(e.h, C.byref(a), C.byref(o)))
            sa = ta.SpeedupArgs()
            sa.mem_kind, sa.n_ctxs, sa.ctxs = ta.MEM_DEVICE, len(x["kset"]), x["d_kset"].data_ptr()
            so = ta.SpeedupOut()
            so.per_ctx, so.total = per.data_ptr(), tot.data_ptr()
            ta._check(ta.lib().ta_potential_speedup(e.h, C.byref(sa), C.byref(so)))
            t = ta.Topology()
            t.n_nodes, t.n_chassis = int(x["topo"]["n_nodes"]), int(x["topo"]["n_chassis"])
            t.n_racks, t.mem_kind = int(x["topo"]["n_racks"]), ta.MEM_DEVICE
            t.node_of_rank, t.rack_of_node, t.chassis_of_node = (z.data_ptr() for z in x["d_topo"])
            ta_ = ta.TopoArgs()
            ta_.metric, ta_.ctx, ta_.tau_num, ta_.tau_den, ta_.min_ranks = (
                ta.EXCLUSIVE, x["topo_ctx"], 2, 1, 1)
            to = ta.TopoOut()
            to.mem_kind = ta.MEM_DEVICE
            for k, v in tout.items():
                setattr(to, k, v.data_ptr())
            ta._check(ta.lib().ta_topology_rollup(e.h, C.byref(t), C.byref(ta_), C.byref(to)))
            e.free()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        clocks = ClockSampler(local)
        clocks.start()
        clocks.wait_first()
        torch.cuda.synchronize()
        l0 = ctx.launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tc0 = clocks.mark()
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        tc1 = clocks.mark()
        return (ev0.elapsed_time(ev1) / steps, (ctx.launches() - l0) / steps,
                clocks.stop(tc0, tc1))

    steps = max(1, min(args.steps, 3))
    plain_ms, plain_l, plain_clk = timed(plain_step, steps, 1)
    t0 = time.perf_counter()
    set_args = [dict(speedup_ctxs=x["kset"], topology=x["topo"], topo_ctx=x["topo_ctx"],
                     topo_tau=(2, 1), min_ranks=1) for x in sets]
    b = ta.Batch(ctx, [(x["d_rank_off"], x["ts"], x["ctx"], x["d_parent"], x["marker"])
                       for x in sets], tau=(3, 1), outlier_cap=cap, set_args=set_args)
    plan_s = time.perf_counter() - t0
    info = b.info()
    torch.cuda.nvtx.range_push("batched")  # lets a profiler take the replays alone
    batch_ms, batch_l, batch_clk = timed(b.run, args.steps, max(3, args.warmup))
    torch.cuda.nvtx.range_pop()
    alg = 12 * N + 16 * info["tensor_nnz"] + 8 * info["n_rows"] + 8 * (R + len(sets))
    out = {"workload": BATCHED + (f" (rank scale {args.batch_scale})" if args.batch_scale != 1 else ""),
           "sets": len(sets), "records": N, "ranks": R, "tensor_entries": info["tensor_nnz"],
           "outliers": info["n_outliers"],
           "plain": {"value": N / (plain_ms / 1e3), "unit": "records/s", "ms_per_step": plain_ms,
                     "gpu_launches_per_step": plain_l, "steps": steps, "clocks": plain_clk,
                     "hbm_gbs_tensor_floor": alg / (plain_ms / 1e3) / 1e9},
           "batched": {"value": N / (batch_ms / 1e3), "unit": "records/s",
                       "ms_per_step": batch_ms, "gpu_launches_per_step": batch_l,
                       "graph_kernels": info["graph_kernels"], "steps": args.steps,
                       "clocks": batch_clk,
                       "plan_s": plan_s, "hbm_gbs_tensor_floor": alg / (batch_ms / 1e3) / 1e9},
           "speedup_batched_over_plain": plain_ms / batch_ms,
           "device_bytes_batch": info["device_bytes"],
           "tuned": {"tile_width": info["tile_width"], "count_warps": info["count_warps"],
                     "count_grid": info["count_grid"], "write_warps": info["write_warps"],
                     "write_grid": info["write_grid"], "trials": info["tune_trials"]}}
    out["batched"]["hbm_frac_tensor_floor"] = (out["batched"]["hbm_gbs_tensor_floor"]
                                               / measured_peaks()[0]["hbm_gbs"])
    b.free()
    del arena, sets
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ serving --
SERVING = ("serving: 8 resident experiments, R uniform in 1k..50k, C=5000 (depth<=24), I=50, "
           "jitter 5%, 1% of ranks 1.2-2x (trace lengths mean 20k, sigma 0.5: the resident "
           "products, R x 51 rows x ~64 contexts, do not depend on trace length), Poisson stream "
           "of queries: 40% context stats over a rank subset (size log-uniform 16..R), 30% "
           "rank x iteration slices (area log-uniform up to 1e6 cells), 20% top-k (k in 1, 10, "
           "100), 10% rack rollups")


def make_serving(args, ctx, device):
    """Load the serving experiments one by one (raw traces generated into
    device memory in chunks, ingested, then dropped: only products stay)."""
    import torch
    from paper_2605_03561_b300 import synth
    rng = np.random.default_rng(17)
    exps = []
    t0 = time.time()
    for k in range(args.serve_exps):
        R = int(rng.integers(1000, 50001) * args.serve_scale)
        cfg = synth.preset(2, seed=500 + k, n_ranks=max(R, 16), len_mean=20000.0)
        rank_off, parent, info = synth.plan(cfg)
        N = int(rank_off[-1])
        d_ts = torch.empty(N, dtype=torch.uint64, device=device)
        d_cx = torch.empty(N, dtype=torch.uint32, device=device)
        step = max(1, cfg.n_ranks // 16)
        big = int(max(rank_off[min(r + step, cfg.n_ranks)] - rank_off[r]
                      for r in range(0, cfg.n_ranks, step)))
        h_ts = torch.empty(big, dtype=torch.uint64, pin_memory=True)
        h_cx = torch.empty(big, dtype=torch.uint32, pin_memory=True)
        for r0 in range(0, cfg.n_ranks, step):
            r1 = min(r0 + step, cfg.n_ranks)
            a, b = int(rank_off[r0]), int(rank_off[r1])
            sub = (rank_off[r0: r1 + 1] - rank_off[r0]).astype(np.uint64)
            synth.fill(cfg, rank_off, r0, r1, h_ts.data_ptr(), h_cx.data_ptr(), 0)
            d_ts[a:b].copy_(h_ts[: b - a])
            d_cx[a:b].copy_(h_cx[: b - a])
            torch.cuda.synchronize()
        e = ctx.load(torch.from_numpy(rank_off).to(device), d_ts, d_cx,
                     torch.from_numpy(parent).to(device), cfg.marker_ctx)
        del d_ts, d_cx
        torch.cuda.empty_cache()
        topo = synth.topology(cfg, info)
        truth = synth.truth(cfg, info)
        exps.append(dict(e=e, R=cfg.n_ranks, C=cfg.n_ctx, N=N, topo=topo,
                         ctxs=np.unique(truth["segment_ctx"]).astype(np.uint32),
                         iters=cfg.n_iter))
    log(f"serving: {len(exps)} experiments, {sum(x['R'] for x in exps)} ranks, "
        f"{sum(x['N'] for x in exps)} records ingested in {time.time() - t0:.1f} s")
    return exps


def serving_queries(ta, exps, n, seed):
    rng = np.random.default_rng(seed)
    qs = []
    kinds = rng.choice([1, 2, 3, 4], size=n, p=[0.4, 0.3, 0.2, 0.1])
    for kind in kinds:
        x = int(rng.integers(0, len(exps)))
        E = exps[x]
        R = E["R"]
        c = int(rng.choice(E["ctxs"]))
        if kind == 1:
            m = int(np.exp(rng.uniform(np.log(16), np.log(R))))
            ranks = np.unique(rng.integers(0, R, size=m)).astype(np.uint32)  # ~m distinct
            qs.append(ta.make_query(1, x, c, ranks=ranks))
        elif kind == 2:
            area = int(np.exp(rng.uniform(0, np.log(1e6))))
            w = int(rng.integers(1, E["iters"] + 1))
            h = max(1, min(R, area // w))
            r0 = int(rng.integers(0, R - h + 1))
            i0 = int(rng.integers(0, E["iters"] - w + 1))
            qs.append(ta.make_query(2, x, c, r0=r0, r1=r0 + h, i0=i0, i1=i0 + w))
        elif kind == 3:
            qs.append(ta.make_query(3, x, c, k=int(rng.choice([1, 10, 100]))))
        else:
            qs.append(ta.make_query(4, x, c, tau=(2, 1), min_ranks=1))
    return qs


def run_serving(args, ctx, local):
    """Plain (one query per launch, one at a time) against continuous
    batching on the same open-loop Poisson stream, at the arrival rate where
    the plain path is 50% busy."""
    import paper_2605_03561_b300 as ta
    dev = f"cuda:{local}"
    exps = make_serving(args, ctx, dev)
    queries = serving_queries(ta, exps, args.serve_queries, 23)

    def server(plain):
        s = ta.Server(ctx, max_batch=1 if plain else 256, n_streams=1 if plain else 3,
                      result_bytes=2 << 30, scratch_bytes=1 << 30)
        for E in exps:
            s.add(E["e"], E["topo"])
        return s

    # plain service time: back-to-back stream (every query queued at t = 0)
    probe = queries[: min(len(queries), 3000)]
    sp = server(True)
    sp.replay(probe[:200], np.zeros(200, np.uint64))  # warm-up
    _, wall = sp.replay(probe, np.zeros(len(probe), np.uint64))
    service = wall / len(probe)
    rate = 0.5 / (service * 1e-9)  # queries/s at 50% utilisation of the plain path
    rng = np.random.default_rng(29)
    arrival = np.cumsum(rng.exponential(1e9 / rate, size=len(queries))).astype(np.uint64)
    out = {"workload": SERVING + (f" (rank scale {args.serve_scale})" if args.serve_scale != 1 else ""),
           "experiments": len(exps), "ranks": sum(E["R"] for E in exps),
           "queries": len(queries), "plain_service_us": service / 1e3,
           "arrival_rate_qps": rate}
    for name, plain in (("plain", True), ("serving", False)):
        s = sp if plain else server(False)
        if not plain:
            s.replay(probe[:200], np.zeros(200, np.uint64))
        l0 = ctx.launches()
        lat, wall = s.replay(queries, arrival)
        launches = ctx.launches() - l0
        lat = lat.astype(np.float64) / 1e3
        out[name] = {"p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                     "mean_us": float(lat.mean()), "qps": len(queries) / (wall * 1e-9),
                     "gpu_launches": launches}
        # saturated throughput: the whole stream queued at once
        _, wall_sat = s.replay(queries, np.zeros(len(queries), np.uint64))
        out[name]["saturated_qps"] = len(queries) / (wall_sat * 1e-9)
        s.close()
    out["p99_plain_over_serving"] = out["plain"]["p99_us"] / out["serving"]["p99_us"]
    out["saturated_serving_over_plain"] = (out["serving"]["saturated_qps"]
                                           / out["plain"]["saturated_qps"])
    for E in exps:
        E["e"].free()
    return out


# --------------------------------------------------------------------- arms --
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.config, pinned=False, ranks=args.ranks)
    aa = analysis_args(w)
    k = pick_sample(w, SAMPLE_RECORDS)
    recs = 0
    secs = 0.0
    for i in range(args.warmup + args.steps):
        n, s = oracle_sample(w, k, aa)
        if i >= args.warmup:
            recs += n
            secs += s
    v = recs / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "records/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config] + (f" (ranks={args.ranks})" if args.ranks else ""), "sample_ranks": k,
                       "sample_records": recs // args.steps},
            "cpu_baseline": {"value": v, "unit": "records/s", "cores": 1, "kind": "oracle",
                             "sample": f"ranks [0, {k}) of the workload per step "
                                       f"({recs // args.steps} records; the same sample as the "
                                       f"GPU line's cpu_baseline)", **host_info()},
            "e2e": {"value": v, "unit": "records/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# cuDF on an A100 (Polaris), seconds, Table I of the paper (context only:
# other data, other machine)
PAPER_CUDF_S = {
    10: dict(grouping=0.000982, sorting=0.000581, filtering=0.003548, merging=0.001739),
    100: dict(grouping=0.001980, sorting=0.000520, filtering=0.001278, merging=0.002199),
    1000: dict(grouping=0.002260, sorting=0.002224, filtering=0.002433, merging=0.005326),
    10000: dict(grouping=0.003993, sorting=0.003165, filtering=0.003908, merging=0.007574),
    100000: dict(grouping=0.024470, sorting=0.023193, filtering=0.008901, merging=0.046568),
}


def run_columns(ta, ctx, e, w, R, stream, peaks):
    import torch
    cols = ta.Columns(ctx)
    node = torch.from_numpy(w["topo"]["node_of_rank"]).cuda()
    out = {"rows": "trace events of ranks [0, T) of the workload: rank, ts, ctx, dur columns",
           "ops": {"grouping": "group-by (rank, ctx): sum of dur and count",
                   "sorting": "stable sort of dur with its permutation",
                   "filtering": "row ids with dur >= 20 us",
                   "merging": "join rank -> node (gather)",
                   "scalar_compare": "dur > 10 us", "vector_add": "ts + dur",
                   "inplace_multiply": "dur *= 3 (on a copy)", "reduction_sum": "sum of dur",
                   "cumulative_sum": "inclusive prefix sum of dur"},
           "paper_cudf_a100_s": PAPER_CUDF_S, "by_traces": {}}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=10):
        fn()
        ms = []
        for _ in range(reps):
            torch.cuda.synchronize()
            ev0.record(stream)
            r = fn()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            del r
        ms.sort()
        return 0.5 * (ms[len(ms) // 2 - 1] + ms[len(ms) // 2])

    for T in (10, 100, 1000, 10000, 100000):
        if T > R:
            break
        t = cols.events(e, 0, T)
        n = int(t["dur"].numel())
        seg = torch.from_numpy(w["rank_off"][:T + 1] - w["rank_off"][0]).cuda()
        dcopy = t["dur"].clone()
        C = len(w["parent"])
        res = {"events": n}
        res["grouping"] = timed(lambda: cols.group(seg, t["ctx"], C, t["dur"]))
        res["sorting"] = timed(lambda: cols.sort(t["dur"]))
        res["filtering"] = timed(lambda: cols.filter(t["dur"], 20000, (1 << 64) - 1))
        res["merging"] = timed(lambda: cols.gather(t["rank"], node))
        res["scalar_compare"] = timed(lambda: cols.compare(t["dur"], 10000))
        res["vector_add"] = timed(lambda: cols.add(t["ts"], t["dur"]))
        res["inplace_multiply"] = timed(lambda: cols.scale(dcopy, 3))
        res["reduction_sum"] = timed(lambda: cols.sum(t["dur"]))
        res["cumulative_sum"] = timed(lambda: cols.cumsum(t["dur"]))
        # sort bytes: per pass 3 key reads, a value read and a key+value write
        mx = int(t["dur"].view(torch.int64).max().item()) if n else 0
        passes = (max(mx, 1).bit_length() + 7) // 8
        res["sort_passes"] = passes
        res["sorting_gbs"] = (40 * n * passes) / (res["sorting"] / 1e3) / 1e9 if n else 0.0
        res["cumulative_sum_gbs"] = (16 * n) / (res["cumulative_sum"] / 1e3) / 1e9 if n else 0.0
        out["by_traces"][str(T)] = res
        del t, seg, dcopy
        torch.cuda.empty_cache()
    out["unit"] = "ms per call (median of 10)"
    out["hbm_peak_gbs"] = peaks["hbm_gbs"]
    return out


def rounded(x, sig=5):
    """Floats to `sig` significant digits (keeps the JSON line short)."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}")
    if isinstance(x, dict):
        return {k: rounded(v, sig) for k, v in x.items()}
    if isinstance(x, list):
        return [rounded(v, sig) for v in x]
    return x


def cpu_summary(cpu):
    if not cpu:
        return cpu
    out = {k: v for k, v in cpu.items() if k != "all_cores"}
    if cpu.get("all_cores"):
        a = cpu["all_cores"]
        out["all_cores"] = {"value": a["value"], "cores": a["cores"], "kind": a["kind"]}
    return out


def block_summaries(d):
    """The headline numbers of every extra block (the full blocks go to
    stderr as 'bench detail')."""
    out = {}
    c2 = d.get("config2")
    if c2:
        out["config2"] = {"records_per_s": c2["records_per_s"], "ms_per_step": c2["ms_per_step"],
                          "records": c2["records"],
                          "tensor_write_frac": c2["tensor_write"]["frac"]}
    sh = d.get("shuffled")
    if sh:
        out["shuffled_rows"] = {
            "ranks": sh["ranks"],
            **{k: {"records": sh[k]["records"], "write_ms": sh[k]["tensor_write"]["ms_per_launch"],
                   "write_frac": sh[k]["tensor_write"]["frac"],
                   "records_per_s_load": sh[k]["records_per_s_load"]}
               for k in ("repeating", "shuffled")}}
    b = d.get("batched_vs_plain")
    if b:
        out["batched"] = {"records_per_s": b["batched"]["value"],
                          "ms_per_step": b["batched"]["ms_per_step"],
                          "plain_ms_per_step": b["plain"]["ms_per_step"],
                          "speedup_over_plain": b["speedup_batched_over_plain"],
                          "launches_per_step": b["batched"]["gpu_launches_per_step"],
                          "plain_launches_per_step": b["plain"]["gpu_launches_per_step"],
                          "hbm_gbs_tensor_floor": b["batched"]["hbm_gbs_tensor_floor"],
                          "hbm_frac_tensor_floor": b["batched"].get("hbm_frac_tensor_floor"),
                          "tuned": b.get("tuned")}
    sv = d.get("serving")
    if sv:
        out["serving"] = {"p50_us": sv["serving"]["p50_us"], "p99_us": sv["serving"]["p99_us"],
                          "plain_p50_us": sv["plain"]["p50_us"],
                          "plain_p99_us": sv["plain"]["p99_us"],
                          "saturated_qps": sv["serving"]["saturated_qps"],
                          "plain_saturated_qps": sv["plain"]["saturated_qps"],
                          "arrival_rate_qps": sv["arrival_rate_qps"]}
    pr = d.get("prune")
    if pr:
        out["prune"] = {"ms": pr["ms"], "kept": pr["kept"], "contexts": pr["contexts"]}
    iv = d.get("interval")
    if iv:
        out["interval"] = {k: {"ms": iv[k]["ms"], "frac": iv[k].get("frac_of_measured_hbm")}
                           for k in iv if isinstance(iv[k], dict)}
    sw = d.get("serve_window")
    if sw:
        out["serve_window"] = {"qps": sw["serving"]["saturated_qps"],
                               "plain_qps": sw["plain"]["saturated_qps"]}
    cl = d.get("cluster")
    if cl:
        out["cluster_ms"] = {k: cl[k]["ms"] for k in cl if isinstance(cl[k], dict)}
    co = d.get("columns")
    if co and co.get("by_traces"):
        last = max(co["by_traces"], key=int)
        out["columns_ms"] = {"traces": int(last),
                             **{k: v for k, v in co["by_traces"][last].items()
                                if k not in ("events", "sort_passes")}}
    return out


def run_gpu(args):
    import torch
    import paper_2605_03561_b300 as ta
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    w = make_workload(args.config, seed=1 + rank, ranks=args.ranks)
    aa = analysis_args(w)
    N, R = w["N"], len(w["rank_off"]) - 1
    dev = f"cuda:{local}"
    d_ro = torch.from_numpy(w["rank_off"]).to(dev)
    d_par = torch.from_numpy(w["parent"]).to(dev)
    d_ts = w["ts"].to(dev, non_blocking=True)
    d_cx = w["ctx"].to(dev, non_blocking=True)
    torch.cuda.synchronize()
    ctx = ta.Context(local)
    calls = DeviceCalls(ta, w, aa, local)
    stream = ctx.stream

    def step():
        e = ctx.load(d_ro, d_ts, d_cx, d_par, w["marker"], borrow=True)
        n_out = calls.run(e)
        info = e.info()
        e.free()
        return info, n_out

    for _ in range(args.warmup):
        info, n_out = step()
    torch.cuda.synchronize()
    ctx.profile(reset=True)
    launches0 = ctx.launches()
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps - 1)]
    tc0 = clocks.mark()
    ev0.record(stream)
    for i in range(args.steps):
        info, n_out = step()
        if i + 1 < args.steps:
            evs[i].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    tc1 = clocks.mark()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    marks = [ev0] + evs + [ev1]
    step_ms = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))
    ms_median = step_ms[len(step_ms) // 2] if len(step_ms) % 2 else \
        0.5 * (step_ms[len(step_ms) // 2 - 1] + step_ms[len(step_ms) // 2])
    clk = clocks.stop(tc0, tc1)
    prof = ctx.profile(reset=True)
    launches = ctx.launches() - launches0
    ms_step = ms / args.steps
    value = aggregate_rate(world, N, args.steps, ms)

    # dominant kernel: the iteration-tensor kernel, timed with events on its stream
    peaks, peak_kind = measured_peaks()
    n_l = max(1, prof["tensor_launches"])
    t_launch = prof["tensor_ms"] / n_l / 1000.0
    alg_bytes = (12 * prof["tensor_records"] + 16 * prof["tensor_entries"]
                 + 8 * prof["tensor_rows"] + 8 * (R + 1) * prof["tensor_launches"]) / n_l
    achieved = alg_bytes / t_launch / 1e9
    per_rec = committed_traffic(args.config)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": (per_rec * prof["tensor_records"] / n_l) if per_rec else None,
                "kernel": "k_tensor", "peak_kind": peak_kind,
                "frac_of_8TBs_nominal": achieved / 8000.0,
                "alg_bytes_per_launch": alg_bytes, "ms_per_launch": t_launch * 1e3}
    step_bytes = alg_bytes  # the step's HBM floor is dominated by the tensor pass
    roofline["step_hbm_gbs"] = step_bytes / (ms_step / 1000.0) / 1e9
    roofline["step_frac"] = roofline["step_hbm_gbs"] / peaks["hbm_gbs"]
    roofline["step_note"] = ("the write pass's algorithmic bytes (the step's HBM floor) over "
                             "the whole step's time")

    # the 4,096-rank workload at its stated size, and the write pass on
    # traces whose rows never repeat their predecessor's run sequence
    config2 = shuffled = None
    if world == 1 and args.config == 3 and not args.no_config2:
        w2 = device_workload(2)
        config2 = run_plain_config(ctx, w2, max(3, args.steps // 2), 2, peaks["hbm_gbs"],
                                   stream, local)
        config2["workload"] = WORKLOADS[2]
        del w2
        torch.cuda.empty_cache()
    if world == 1 and args.config == 3 and not args.no_shuffled:
        shuffled = run_shuffled(ctx, 10000, 5, peaks["hbm_gbs"])

    # next row N1: pruning on the summary profile (the paper's 1 % rule) of one
    # freshly loaded experiment, timed alone around the call (not in the step)
    prune = None
    if not args.no_prune:
        e = ctx.load(d_ro, d_ts, d_cx, d_par, w["marker"], borrow=True)
        before = e.info()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pr = e.prune(keep=(1, 100))
        el = time.perf_counter() - t0
        e.free()
        prune = {"keep": "1/100 of the summary total", "ms": el * 1e3, "kept": pr["n_kept"],
                 "contexts": len(w["parent"]),
                 "exclusive_entries": [before["excl_nnz"], pr["excl_nnz"]],
                 "inclusive_entries": [before["incl_nnz"], pr["incl_nnz"]],
                 "timing": "host clock around ta_prune_profiles (it synchronises)"}

    # next row N2: per-rank profiles of a time window (borrowed traces stay on
    # the device), all ranks; device time of the window kernels from the
    # library's stream events.  Algorithmic bytes: the edge samples and inner
    # tensor entries the kernels must read (counted by the library), the
    # output entries and per-rank offsets.  Each timed call has new bounds
    # (t1 moved by 1 ns) so that none reuses the previous result.
    interval = None
    if not args.no_interval:
        e = ctx.load(d_ro, d_ts, d_cx, d_par, w["marker"], borrow=True)
        ro = w["rank_off"].astype(np.int64)
        ne = ro[1:] > ro[:-1]
        ts_np = w["ts"].numpy()
        first = ts_np[ro[:-1][ne]].astype(np.int64)
        last = ts_np[ro[1:][ne] - 1].astype(np.int64)
        med = int(np.median(last - first)) + int(np.median(first))
        interval = {"timing": "CUDA events on the library stream around the window kernels "
                              "(count pass, scan, write pass; inclusive adds the rollup); "
                              "median of 5 calls after 1 warm-up, one computation per call",
                    "window_10pct": "[45%, 55%) of the median rank's end time",
                    "whole_range": "[0, 2^64 - 1)"}
        big = (1 << 64) - 1
        for name, (t0, t1, step) in (("window_10pct", (med * 45 // 100, med * 55 // 100, 1)),
                                     ("whole_range", (0, big, -1))):
            for metric, mname in ((ta.EXCLUSIVE, "exclusive"), (ta.INCLUSIVE, "inclusive")):
                e.interval(t0, t1, metric=metric, device=True)
                recs = []
                for i in range(5):
                    ctx.profile(reset=True)
                    out = e.interval(t0, t1 + step * (i + 1), metric=metric, device=True)
                    p = ctx.profile(reset=True)
                    recs.append((p["interval_ms"], p["interval_samples"], p["interval_entries"]))
                    nnz = int(out["ctx"].numel())
                    samples = int(out["cnt"].to(torch.int64).sum().item()) \
                        if metric == ta.EXCLUSIVE else None
                    del out
                recs.sort()
                ms, es, ee = recs[2]
                rec = {"ms": ms, "entries_out": nnz, "edge_samples_read": es,
                       "inner_entries_read": ee}
                if metric == ta.EXCLUSIVE:
                    alg = 12 * es + 16 * ee + 16 * nnz + 40 * R
                    gbs = alg / (ms / 1e3) / 1e9
                    rec.update({"samples_in_window": samples, "alg_bytes": alg,
                                "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peaks["hbm_gbs"],
                                "samples_per_s": samples / (ms / 1e3)})
                interval[f"{name}_{mname}"] = rec
        e.free()
        del ts_np

    # the serving form's window query (N2) on this experiment: 2,000 queries,
    # each the time of one segment context in a window of 10 % of the median
    # rank's time on 1,000 consecutive ranks; all queued at once (saturated)
    serve_window = None
    if not args.no_serve_window:
        e = ctx.load(d_ro, d_ts, d_cx, d_par, w["marker"], borrow=True)
        rng = np.random.default_rng(31)
        ro = w["rank_off"].astype(np.int64)
        ne = ro[1:] > ro[:-1]
        ts_np = w["ts"].numpy()
        med = int(np.median(ts_np[ro[1:][ne] - 1].astype(np.int64)
                            - ts_np[ro[:-1][ne]].astype(np.int64)))
        span_r = min(1000, R)
        qs = []
        for _ in range(2000):
            t0 = int(rng.integers(0, max(1, med * 9 // 10)))
            r0 = int(rng.integers(0, R - span_r + 1))
            qs.append(ta.make_query(ta.Q_WINDOW, 0, int(rng.choice(aa["kset"])), r0=r0,
                                    r1=r0 + span_r, t0=t0, t1=t0 + med // 10))
        serve_window = {"queries": len(qs), "ranks_per_query": span_r,
                        "window": "10 % of the median rank's time at a random start"}
        for name, mb, ns in (("plain", 1, 1), ("serving", 256, 3)):
            srv = ta.Server(ctx, max_batch=mb, n_streams=ns, result_bytes=1 << 30,
                            scratch_bytes=1 << 28)
            srv.add(e, None)
            srv.replay(qs[:100], np.zeros(100, np.uint64))
            _, wall = srv.replay(qs, np.zeros(len(qs), np.uint64))
            serve_window[name] = {"saturated_qps": len(qs) / (wall * 1e-9),
                                  "us_per_query": wall / len(qs) / 1e3}
            srv.close()
        serve_window["saturated_serving_over_plain"] = (
            serve_window["serving"]["saturated_qps"] / serve_window["plain"]["saturated_qps"])
        e.free()
        del ts_np

    # next row N3: DBSCAN and K-Means (k = 2..5, the paper's stability check)
    # over every rank's exclusive time of a communication context, with the
    # node view; host clock around each call (it synchronises), median of 5
    cluster = None
    if not args.no_cluster:
        e = ctx.load(d_ro, d_ts, d_cx, d_par, w["marker"], borrow=True)
        c = aa["topo_ctx"]
        node = w["topo"]["node_of_rank"]
        nn = int(w["topo"]["n_nodes"])
        x = e.csr(ta.EXCLUSIVE)
        vals = x["time"][x["ctx"] == c]
        med = int(np.median(vals)) if len(vals) else 1
        cluster = {"ctx": c, "ranks": R, "nodes": nn,
                   "timing": "host clock around ta_cluster_ranks (host outputs, node view), "
                             "median of 5 calls after 1 warm-up"}
        runs = [("dbscan", dict(eps=max(1, med // 100), min_pts=10))] + \
               [(f"kmeans_k{k}", dict(k=k)) for k in (2, 3, 4, 5)]
        for name, kw in runs:
            meth = "dbscan" if name == "dbscan" else "kmeans"
            e.cluster(c, meth, node_of_rank=node, n_nodes=nn, **kw)
            el = []
            for _ in range(5):
                t0 = time.perf_counter()
                got = e.cluster(c, meth, node_of_rank=node, n_nodes=nn, **kw)
                el.append(time.perf_counter() - t0)
            el.sort()
            rec = {"ms": el[2] * 1e3, "clusters": got["n_clusters"], "noise": got["n_noise"],
                   "iterations": got["iterations"],
                   "cluster_sizes": got["clusters"]["n"].tolist()[:8]}
            if "pair_nodes" in got:
                pn = got["pair_nodes"]
                rec["cluster_nodes"] = got["cluster_nodes"].tolist()[:8]
                rec["nodes_in_two_clusters"] = int(np.triu(pn, 1).sum())
            cluster[name] = rec
        e.free()

    # next row N4: the DataFrame operation classes of Tables I-III as column
    # kernels over the events of the first T traces (T = 10 .. 100,000),
    # device time from CUDA events on the library stream, median of 10 runs
    # (the paper averages 10)
    columns = None
    if not args.no_columns:
        e = ctx.load(d_ro, d_ts, d_cx, d_par, w["marker"], borrow=True)
        columns = run_columns(ta, ctx, e, w, R, stream, peaks)
        e.free()
        torch.cuda.empty_cache()

    # e2e: the user-facing call with host (pinned) inputs and host outputs
    e2e = None
    if not args.no_e2e:
        del d_ts, d_cx
        torch.cuda.empty_cache()
        h_ro, h_par = w["rank_off"], w["parent"]
        h_ts, h_cx = w["ts"].numpy(), w["ctx"].numpy()
        k_e2e = max(1, min(args.steps, 3))
        for _ in range(1):
            e = ctx.load(h_ro, h_ts, h_cx, h_par, w["marker"])
            host_calls(e, w, aa)
            e.free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(k_e2e):
            e = ctx.load(h_ro, h_ts, h_cx, h_par, w["marker"])
            d2h = host_calls(e, w, aa)
            e.free()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        h2d = 8 * (R + 1) + 12 * N + 4 * len(h_par) + 4 * (R + 2 * len(w["topo"]["rack_of_node"])) + 4 * len(aa["kset"])
        e2e = {"value": world * N * k_e2e / el, "unit": "records/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k_e2e, "s_per_step": el / k_e2e}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        k = pick_sample(w, SAMPLE_RECORDS)
        n, s, reps = 0, 0.0, 0
        while reps < 3 or (s < args.cpu_seconds and reps < 20):
            n1, s1 = oracle_sample(w, k, aa)
            n, s, reps = n + n1, s + s1, reps + 1
        cpu = {"value": n / s, "unit": "records/s", "cores": 1, "kind": "oracle",
               "sample": f"ranks [0, {k}) = {n // reps} records of the same workload (the "
                         f"reference arm's sample), whole path (analysis, stats over all "
                         f"contexts, rack rollup, speedup), {reps} runs, {s:.1f} s",
               **host_info()}
        if not args.no_cpu_threads:
            n_thr = max(1, os.cpu_count() or 1)
            kt = pick_sample(w, args.cpu_records * min(n_thr, 8))
            n2, s2, used = oracle_sample_threads(w, kt, aa, n_thr)
            cpu["all_cores"] = {
                "value": n2 / s2, "unit": "records/s", "cores": used,
                "kind": "oracle split over ranks (threads)",
                "sample": f"ranks [0, {kt}) = {n2} records in {used} contiguous rank ranges, "
                          f"each analysed whole (statistics, rollup and speedup over its own "
                          f"ranks); {s2:.1f} s"}

    batched = None
    if not args.no_batched:
        for k in ("ts", "ctx"):
            w[k] = None
        d_ro = d_par = d_ts = d_cx = calls = None
        torch.cuda.empty_cache()
        batched = run_batched(args, ctx, local)
    serving = None
    if not args.no_serving:
        serving = run_serving(args, ctx, local)

    if rank == 0:
        detail = {"batched_vs_plain": batched, "serving": serving, "prune": prune,
                  "interval": interval, "serve_window": serve_window, "cluster": cluster,
                  "columns": columns, "config2": config2, "shuffled": shuffled,
                  "cpu_baseline": cpu}
        log("bench detail " + json.dumps(detail))
        line = {"metric": METRIC, "value": value, "unit": "records/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "ms_per_step_median": ms_median,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config] + (f" (ranks={args.ranks})" if args.ranks else ""),
                           "records": N, "ranks": R,
                           "contexts": len(w["parent"]), "tensor_rows": info["n_rows"],
                           "tensor_entries": info["tensor_nnz"],
                           "exclusive_entries": info["excl_nnz"],
                           "inclusive_entries": info["incl_nnz"], "outliers": n_out,
                           "l2": "inputs (12 B x records) far exceed the 126 MB L2; no flush",
                           "step": "ingest + tensor + exclusive + inclusive + stats(all ctx) + "
                                   "rack rollup + speedup",
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                "hbm_gbs_step": step_bytes / (ms_step / 1000.0) / 1e9 * 1.0,
                "phase_ms_per_step": {k: prof[k] / args.steps for k in
                                      ("validate_ms", "tensor_count_ms", "tensor_ms", "exclusive_ms", "inclusive_ms",
                                       "stats_ms", "topology_ms", "speedup_ms")},
                "roofline": roofline, "cpu_baseline": cpu_summary(cpu), "e2e": e2e,
                "blocks": block_summaries(detail),
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(rounded(line)), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=3, choices=[1, 2, 3])
    p.add_argument("--ranks", type=int, default=0,
                   help="override the rank count (smaller cases for profiling)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-records", type=float, default=1.5e8,
                   help="records per thread of the all-cores oracle baseline")
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="CPU time the single-core oracle baseline repeats its sample for")
    p.add_argument("--no-cpu-threads", action="store_true",
                   help="skip the oracle split over all host cores")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-prune", action="store_true")
    p.add_argument("--no-interval", action="store_true")
    p.add_argument("--no-cluster", action="store_true")
    p.add_argument("--no-serve-window", action="store_true")
    p.add_argument("--no-columns", action="store_true")
    p.add_argument("--no-config2", action="store_true",
                   help="skip the 4,096-rank workload at its stated size")
    p.add_argument("--no-shuffled", action="store_true",
                   help="skip the write pass on traces whose rows never repeat")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serve-exps", type=int, default=8)
    p.add_argument("--serve-queries", type=int, default=100000)
    p.add_argument("--serve-scale", type=float, default=1.0,
                   help="scale the rank count of every served experiment")
    p.add_argument("--batch-sets", type=int, default=256)
    p.add_argument("--batch-scale", type=float, default=1.0,
                   help="scale the rank count of every batched set (smaller runs)")
    args = p.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
