#!/usr/bin/env python3
"""Throughput of the global Curveball super step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload n2^25|n2^20|n2^21|n4096|ensemble|serving|uniform|swaps|autocorr]

One "step" is one global super step (Def. "Undirected Global Trade",
Section 3.3) over the whole graph.  The metric is edge-trades/s = m * steps /
device time, the reciprocal of the paper's "walltime per edge and super step"
(Section 5.2).  The default workload is n=2^25 nodes with PLD([10,10000),2)
degrees realised by Havel-Hakimi (about 1.1e9 undirected edges, adjacency far
larger than L2).  With N>1 processes (torchrun) every rank randomises its own
replica of the graph with its own chain seed: the chain itself does not shard.

--impl reference times the sequential CPU oracle (the reference this project
is checked against) on a bounded sample of the same workload family.

The line also carries "batched": the ensemble workload (256 independent
graphs, n log-uniform in [2^10, 2^16], 50 super steps each) run as one batch
handle (one CUDA-graph launch per super step, autotuned work split) against
256 sequential plain runs on the same GPU.  --workload ensemble makes that
the headline of the line.

--workload uniform times uniform single trades instead (Simple Undirected
Curveball, Section 3.2): one step is n/2 trades on the --uniform-graph graph,
run as the successor-list dataflow.  --workload autocorr runs Section 5.1's
mixing experiment (fraction of edges still correlated against the thinning
k, n = 2000).  --workload swaps prints the appendix's
swap-fraction series (uniform trades against global trades as n grows).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge-trades/s per global super step"
UNIT = "edge-trades/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n2^25")
    ap.add_argument("--batched", type=int, default=1, help="1: add the batched-ensemble comparison to the line")
    ap.add_argument("--generate", type=int, default=0,
                    help="1: time the workload's input graph generated on the device against the host generator")
    ap.add_argument("--requests", type=int, default=200, help="serving workload: number of requests replayed")
    ap.add_argument("--plain-compare", type=int, default=1,
                    help="ensemble workload: 0 skips the 256 sequential plain runs it is compared with")
    ap.add_argument("--uniform-graph", default="n2^25",
                    help="uniform workload: the plain graph the uniform single trades run on")
    ap.add_argument("--perm", default="sort", choices=["sort", "relaxed"],
                    help="relaxed: permutations from linear congruential maps (Def. 'Relaxed global trade')")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Replicas: one chain does not shard, so every rank randomises its own replica
# of the workload; the job's time is its slowest rank's, and its throughput
# counts the work of all ranks.

def replica_seed(seed, rank):
    """The chain seed of rank `rank`'s replica."""
    return seed + rank


def ensemble_replica_seeds(seeds, rank):
    """Every graph's chain seed in rank `rank`'s replica of an ensemble."""
    return [s + 1000003 * rank for s in seeds]


def max_over_ranks(x, world, device="cuda"):
    """The largest x over all ranks (a collective when world > 1)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, t_max_s):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / t_max_s


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- workloads

def workload(name):
    from paper_1804_08487_gb300 import synth
    if name not in synth.PLAIN:
        raise SystemExit(f"unknown workload {name}; choose from {sorted(synth.PLAIN)}")
    return synth.PLAIN[name]


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass,
# every launch of the unit in one super step) of the dominant unit of a
# workload, and the sha256 of csrc/trade.cu the capture ran on; a unit whose
# code changed since reports no traffic.  profiles/ holds the captures.
MEASURED_TRAFFIC = {
    # profiles/rebuild_traffic_n2p25.md: mean of four super steps
    ("rebuild phase (k_far_pack, k_chunk_rows, k_fixup passes)", "n2^25"): {
        "bytes": 92497908608,
        "trade_cu_sha256": "048fcb563ef234b9ff0c1de074ee5f6ff6650e8c2293f61419123590ebc5da4b",
    },
}


def measured_traffic(unit, workload):
    """DRAM bytes per launch of `unit` on `workload` from the committed ncu
    capture, or None."""
    import hashlib
    rec = MEASURED_TRAFFIC.get((unit, workload))
    if rec is None:
        return None
    src = os.path.join(ROOT, "paper_1804_08487_gb300", "csrc", "trade.cu")
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["trade_cu_sha256"]:
        return None
    return rec["bytes"]


# the threshold phase's kernel of each size class (cb_timings ms[4 + k])
CLASS_KERNELS = ["k_phase_a_lanes<8>", "k_phase_a_lanes<16>", "k_phase_a_warp", "k_phase_a_team<256,64>",
                 "k_phase_a_team<256,128>", "k_phase_a_team<256,256>", "k_phase_a_team<1024,512>",
                 "k_phase_a_team<1024,1024>", "k_phase_a_block<1024>"]
# algorithmic bytes: a threshold kernel reads each directed entry of its
# trades (4 B) and writes it into the new row with its side word (4 + 2 B),
# plus per trade its two rows' offsets, positions, threshold and done flag
# (48 B); the fix-up reads each placeholder and side word (4 + 2 B) and
# writes the final entry (4 B), plus the 8-byte far-trade record written and
# read once per trade
THRESHOLD_BYTES_PER_ENTRY = 10
THRESHOLD_BYTES_PER_TRADE = 48
FIXUP_BYTES_PER_ENTRY = 10
FIXUP_BYTES_PER_TRADE = 16


# the rebuild is timed as one unit per super step: the far-trade records,
# each chunk's first row, and the fix-up passes over slices of the far trades
REBUILD_UNIT = "rebuild phase (k_far_pack, k_chunk_rows, k_fixup passes)"


def dominant_kernel(stats, phases, m, ntasks, K):
    """The kernel (or, for the rebuild, the fix-up launches of one step) with
    the largest event-timed device time per super step, its algorithmic bytes
    per launch and average launch duration.  The first threshold pass's class
    kernels are bracketed by events; the retry passes and the in-order pass
    run only the few deferred trades; the rebuild counts as one launch per
    super step."""
    cands = []
    for k, name in enumerate(CLASS_KERNELS):
        ms = phases.get(f"class{k}_ms", 0.0) / K
        if ms > 0:
            b = (THRESHOLD_BYTES_PER_ENTRY * stats.get(f"class{k}_entries", 0)
                 + THRESHOLD_BYTES_PER_TRADE * stats.get(f"class{k}_trades", 0))
            cands.append((ms, name, b, stats.get(f"class{k}_entries", 0)))
    cands.append((phases["rebuild_ms"] / K, REBUILD_UNIT,
                  FIXUP_BYTES_PER_ENTRY * 2 * m + FIXUP_BYTES_PER_TRADE * ntasks, 2 * m))
    ms, name, b, entries = max(cands)
    return name, b, ms, entries


def verify_step1(name, c, m):
    """{"step1": bool, "against": ...}: the handle's edge list after its first
    super step compared with the oracle's sha256 stored in tests/golden for
    this workload (None when no digest is stored)."""
    import hashlib
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"plain_{name.replace('^', 'p')}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        want = json.load(f)["edge_sha256_after_step"].get("1")
    if want is None:
        return None
    out = np.empty((m, 2), dtype=np.int32)
    c.edges(out)
    got = hashlib.sha256(memoryview(out).cast("B")).hexdigest()
    return {"step1": got == want, "against": os.path.relpath(path, ROOT) + " (oracle digest)"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_sample(w, steps=1, log2n=19, perm="sort"):
    """Oracle on a bounded sample of the workload family: the same degree law
    at n=2^log2n, `steps` super steps, one host core (the chain is sequential)."""
    from oracle import Oracle
    from paper_1804_08487_gb300 import synth
    g = synth.powerlaw_graph(1 << log2n, w.a, w.b, w.gamma, w.degree_seed)
    o = Oracle(g.row_ptr, g.col, w.chain_seed)
    if perm == "relaxed":
        o.set_relaxed(True)
    t0 = time.perf_counter()
    o.superstep(steps)
    dt = time.perf_counter() - t0
    desc = (f"oracle, n=2^{log2n} PLD([{w.a},{w.b}),{w.gamma:g}) Havel-Hakimi graph (m={g.m}), "
            f"{steps} super step(s), sequential")
    return g.m * steps / dt, desc, g.m, dt


def config_of(w, g, world, perm="sort"):
    return {"workload": w.name + (" relaxed (linear congruential maps)" if perm == "relaxed" else ""),
            "n": g.n, "m": g.m, "degree_seed": g.degree_seed, "chain_seed": w.chain_seed,
            "l2": "inputs larger than L2 (adjacency %.1f GB vs 129 MB L2)" % (g.m * 8 / 1e9),
            "parallelism": "replicas" if world > 1 else "single"}


# -------------------------------------------------------------- ensemble

ENSEMBLE_GRAPHS = 256
ENSEMBLE_STEPS = 50
ENSEMBLE_TUNE_STEPS = 60     # autotuning super steps before the timed ones (untimed warm-up)
ENSEMBLE_NAME = ("ensemble of 256 graphs: n log-uniform in [2^10, 2^16], PLD([4, n/16), gamma in [2, 3]), "
                 "Havel-Hakimi, seed 1000+i, 50 super steps each")


def ensemble_graphs(count=ENSEMBLE_GRAPHS):
    from paper_1804_08487_gb300 import synth
    members = [synth.ensemble_member(i) for i in range(count)]
    graphs = []
    for w in members:
        g = w.graph()
        graphs.append((g.row_ptr, g.col))
    return graphs, [w.chain_seed for w in members]


def measure_ensemble(graphs, seeds, stream, steps=ENSEMBLE_STEPS, tune_steps=ENSEMBLE_TUNE_STEPS, clocks=None,
                     plain_compare=True):
    """Batched: one handle, autotuned (its tuning steps are untimed warm-up),
    CUDA-graph replay, `steps` timed super steps.  Plain (unless
    plain_compare is off): each graph in its own handle, `steps` super steps
    each, timed one after another (device time summed), with direct launches
    and with CUDA-graph replay."""
    import torch
    from paper_1804_08487_gb300 import cb

    total_m = sum(int(rp[-1]) // 2 for rp, _ in graphs)
    total_n = sum(len(rp) - 1 for rp, _ in graphs)
    ens = cb.Ensemble(graphs, seeds, stream=stream)
    tuned = ens.autotune(tune_steps)
    ens.set_option("cuda_graph", 1)
    ens.global_trades(2)
    ens.sync()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
    e0.record(stream)
    ens.global_trades(steps)
    e1.record(stream)
    e1.synchronize()
    clk = clocks.stop() if clocks else None
    batched_ms = e0.elapsed_time(e1)
    launches = int(ens.stats().get("launches", 0))
    ens.close()

    def plain(use_graph):
        total = 0.0
        for (rp, col), sd in zip(graphs, seeds):
            c = cb.Curveball(rp, col, sd, stream=stream)
            c.set_option("cuda_graph", use_graph)
            c.sync()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.global_trades(steps)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b)
            c.close()
        return total

    et = total_m * steps
    r = {"workload": ENSEMBLE_NAME, "graphs": len(graphs), "n_total": total_n, "m_total": total_m,
         "steps": steps, "batched_ms": batched_ms, "batched_edge_trades_s": et / (batched_ms / 1e3),
         "autotuned": tuned, "batched_launches": launches, "clocks": clk}
    if plain_compare:
        plain_ms = plain(0)
        plain_graph_ms = plain(1)
        r.update({"plain_ms": plain_ms, "plain_edge_trades_s": et / (plain_ms / 1e3),
                  "plain_cuda_graph_ms": plain_graph_ms,
                  "plain_cuda_graph_edge_trades_s": et / (plain_graph_ms / 1e3),
                  "speedup_vs_plain": plain_ms / batched_ms, "speedup_vs_plain_cuda_graph": plain_graph_ms / batched_ms})
    return r


def _oracle_member_rate(args):
    """Oracle edge-trades/s on one graph of the ensemble (a worker process)."""
    i, steps = args
    from oracle import Oracle
    from paper_1804_08487_gb300 import synth
    w = synth.ensemble_member(i)
    g = w.graph()
    o = Oracle(g.row_ptr, g.col, w.chain_seed)
    t0 = time.perf_counter()
    o.superstep(steps)
    return g.m * steps, time.perf_counter() - t0


def ensemble_cpu_sample(graphs_sampled=32, steps=5):
    """The oracle on a bounded sample of the ensemble: the first 32 graphs,
    5 super steps each, the graphs spread over every host core."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_member_rate, [(i, steps) for i in range(graphs_sampled)], chunksize=1)
    wall = time.perf_counter() - t0
    work = sum(r[0] for r in res)
    return work / wall, cores, (f"oracle on graphs 0..{graphs_sampled - 1} of the ensemble, {steps} super steps "
                                f"each, {cores} worker processes (wall time incl. graph generation)")


def run_ensemble(args):
    import torch
    from paper_1804_08487_gb300 import cb

    rank, world, local = dist_env()
    # the oracle pool starts before this process touches the GPU
    cpu_v, cpu_cores, cpu_desc = ensemble_cpu_sample() if rank == 0 else (None, None, None)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    graphs, seeds = ensemble_graphs()
    seeds = ensemble_replica_seeds(seeds, rank)   # each replica its own chains
    stream = torch.cuda.Stream()
    r = measure_ensemble(graphs, seeds, stream, steps=ENSEMBLE_STEPS, clocks=ClockSampler(local),
                         plain_compare=bool(args.plain_compare))
    t_ms = max_over_ranks(r["batched_ms"], world)
    # end to end: create from pinned host buffers, the super steps, every
    # graph's edge list back to pinned host memory
    rp_all = torch.from_numpy(__import__("numpy").concatenate([g[0] for g in graphs])).pin_memory()
    col_all = torch.from_numpy(__import__("numpy").concatenate([g[1] for g in graphs])).pin_memory()
    ns = [len(g[0]) - 1 for g in graphs]
    out_h = torch.empty(2 * r["m_total"], dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = cb.cb_create_batch(ns, rp_all, col_all, seeds, 0, stream)
    cb.cb_set_option(h, "cuda_graph", 1)
    cb.cb_global_trades(h, ENSEMBLE_STEPS)
    cb.cb_export_edges(h, out_h)
    cb.cb_sync(h)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    cb.cb_destroy(h)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    K = ENSEMBLE_STEPS
    b_min = 16 * r["m_total"] + 24 * r["n_total"]
    gbs = b_min / (t_ms / K / 1e3) / 1e9
    value = job_rate(world, r["m_total"] * K, t_ms / 1e3)
    line = {
        "metric": METRIC + " (batched ensemble)", "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": ENSEMBLE_TUNE_STEPS + 2, "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": ENSEMBLE_NAME, "graphs": r["graphs"], "n_total": r["n_total"],
                   "m_total": r["m_total"], "l2": "inputs smaller than L2 are re-read every step (no flush)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "kernel": "whole super step", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs"},
        "batched_vs_plain": r.get("speedup_vs_plain"),
        "batched": r,
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cpu_cores, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": job_rate(world, r["m_total"] * K, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": (rp_all.numel() * 8 + col_all.numel() * 4) / K,
                "d2h_bytes_per_step": out_h.numel() * 4 / K},
        "gpu_launches": r["batched_launches"],
        "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------- serving

SERVING_REQUESTS = 200
SERVING_BUDGET = 120 * 10**9
SERVING_NAME = ("serving: Poisson arrivals (mean 200 req/s), n log-uniform in [2^12, 2^22], PLD([4, n/16], "
                "gamma in [2, 3]), Havel-Hakimi, 5..50 super steps, seed = request index, 120 GB budget")


def _serving_graph(i):
    from paper_1804_08487_gb300 import synth
    w = synth.serving_request(i)
    g = w.graph()
    return i, g.row_ptr, g.col, w.chain_seed, w.supersteps


def serving_requests(count):
    """Every request's graph, generated on all host cores (spawn pool, before
    any GPU work of this process)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        out = pool.map(_serving_graph, range(count), chunksize=1)
    return sorted(out)


def measure_serving(reqs, arrivals, budget=SERVING_BUDGET, max_active=64, depth=2, clocks=None):
    """Replay the arrivals into the serving loop: a thread submits request i
    at arrival time i; latency = finished - submitted (the server's clock)."""
    import threading
    import numpy as np
    from paper_1804_08487_gb300 import cb

    srv = cb.Server(budget, max_active=max_active, depth=depth)
    t0 = time.perf_counter()
    ids = {}

    def submitter():
        for (i, rp, col, seed, steps), at in zip(reqs, arrivals):
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids[srv.submit(rp, col, seed, steps)] = i

    if clocks:
        clocks.start()
    th = threading.Thread(target=submitter)
    th.start()
    results = {}
    while len(results) < len(reqs):
        for rid in srv.poll(timeout_ms=200):
            edges, times = srv.result(rid)
            results[rid] = (times, edges)
    th.join()
    clk = clocks.stop() if clocks else None
    st = srv.stats()
    srv.close()
    lat = np.array([results[r][0][3] - results[r][0][0] for r in sorted(results)])
    first = min(results[r][0][0] for r in results)
    last = max(results[r][0][3] for r in results)
    work = sum(int(rp[-1]) // 2 * steps for _, rp, _, _, steps in reqs)
    by_index = {ids[r]: results[r][1] for r in results}
    return {
        "requests": len(reqs), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()), "max_s": float(lat.max()), "makespan_s": last - first,
        "edge_trades": work, "edge_trades_s": work / (last - first),
        "reserved_peak_bytes": st.get("reserved_peak_bytes"), "steps_issued": st.get("steps_issued"),
        "failed": st.get("failed"), "clocks": clk,
    }, by_index


def measure_plain_sequential(reqs, results=None):
    """The same requests one at a time through plain handles (create, super
    steps, export), wall time; optionally checks each edge list against the
    served one."""
    import numpy as np
    from paper_1804_08487_gb300 import cb
    total = 0.0
    same = True
    for i, rp, col, seed, steps in reqs:
        t = time.perf_counter()
        c = cb.Curveball(rp, col, seed)
        c.global_trades(steps)
        e = c.edges()
        c.close()
        total += time.perf_counter() - t
        if results is not None:
            same &= bool(np.array_equal(e, results[i]))
    work = sum(int(rp[-1]) // 2 * steps for _, rp, _, _, steps in reqs)
    return {"seconds": total, "edge_trades_s": work / total, "served_equal_alone": same if results else None}


def run_serving(args):
    import torch
    from paper_1804_08487_gb300 import synth

    rank, world, local = dist_env()
    count = args.requests
    reqs = serving_requests(count)
    arrivals = synth.serving_arrivals(count)
    torch.cuda.set_device(local)
    if rank != 0:
        return
    served, by_index = measure_serving(reqs, arrivals, clocks=ClockSampler(local))
    plain = measure_plain_sequential(reqs, by_index)
    line = {
        "metric": METRIC + " (serving)", "value": served["edge_trades_s"], "unit": UNIT, "n_gpus": 1,
        "steps": sum(r[4] for r in reqs), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": SERVING_NAME, "requests": count, "budget_bytes": SERVING_BUDGET,
                   "max_active": 64, "depth": 2, "parallelism": "single"},
        "latency": {"p50_s": served["p50_s"], "p99_s": served["p99_s"], "mean_s": served["mean_s"],
                    "max_s": served["max_s"]},
        "serving": served, "plain_sequential": plain,
        "served_vs_plain": served["edge_trades_s"] / plain["edge_trades_s"],
        "e2e": {"value": served["edge_trades_s"], "unit": UNIT,
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
        "clocks": served["clocks"],
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- uniform single trades

UNIFORM_METRIC = "edge-trades/s per n/2 uniform single trades"


def uniform_cpu_sample(w, log2n=19):
    """Oracle's uniform single trades on a bounded sample: the same degree law
    at n=2^log2n, n/2 trades, one host core (the sequence is sequential)."""
    from oracle import Oracle
    from paper_1804_08487_gb300 import synth
    g = synth.powerlaw_graph(1 << log2n, w.a, w.b, w.gamma, w.degree_seed)
    o = Oracle(g.row_ptr, g.col, w.chain_seed)
    t0 = time.perf_counter()
    o.uniform_trades(g.n // 2)
    dt = time.perf_counter() - t0
    desc = (f"oracle, n=2^{log2n} PLD([{w.a},{w.b}),{w.gamma:g}) Havel-Hakimi graph (m={g.m}), "
            f"n/2 uniform single trades, sequential")
    return g.m / dt, desc


def run_uniform(args):
    """One step = n/2 uniform single trades (Section 3.2; as many trades as one
    global trade) on the plain workload graph, run as the Suc dataflow."""
    import torch
    from paper_1804_08487_gb300 import cb
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args.uniform_graph)
    g = w.graph()
    seed = replica_seed(w.chain_seed, rank)
    stream = torch.cuda.Stream()
    half = g.n // 2
    c = cb.Curveball(g.row_ptr, g.col, seed, stream=stream)
    c.uniform_trades(half * args.warmup)
    c.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        c.uniform_trades(half)
        launches += int(c.stats().get("launches", 0))
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(t_ms, world)
    K = args.steps
    value = job_rate(world, g.m * K, t_max / 1e3)
    c.set_option("swap_stats", 1)   # one more, untimed step for the swap fraction
    c.uniform_trades(half)
    sw_done, sw_all = c.swap_counts()
    # end to end through the C ABI with host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    out_h = torch.empty(2 * g.m, dtype=torch.int32).pin_memory()
    c.close()
    barrier()
    t0 = time.perf_counter()
    c2 = cb.Curveball(rp_h, col_h, seed, stream=stream)
    c2.uniform_trades(half * K)
    c2.edges(out_h)
    c2.sync()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    c2.close()
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    b_min = 16 * g.m + 24 * g.n
    gbs = b_min / (t_max / K / 1e3) / 1e9
    cpu_v, cpu_desc = uniform_cpu_sample(w)
    line = {
        "metric": UNIFORM_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(config_of(w, g, world), workload=w.name + ", n/2 uniform single trades per step"),
        "roofline": {"bound": "hbm", "kernel": "uniform trades (whole step)", "achieved": gbs, "peak": peak,
                     "unit": "GB/s", "frac": gbs / peak, "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "note": "B_min = 16m + 24n per step; the dataflow is bound by its chain of dependent trades"},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": job_rate(world, g.m * K, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": (g.row_ptr.nbytes + g.col.nbytes) / K, "d2h_bytes_per_step": 2 * g.m * 4 / K},
        "gpu_launches": launches,
        "clocks": clk,
        "swap_fraction": {"performed": sw_done, "possible": sw_all,
                          "fraction": sw_done / sw_all if sw_all else None, "of": "n/2 uniform single trades"},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------- swap fraction

def run_swaps(args):
    """The appendix experiment "Swaps performed by Curveball and Global
    Curveball": the fraction of performed to possible neighbourhood swaps of
    n/2 uniform trades and of one global trade, on 10-regular graphs and on
    PLD([10, n/20), 2) graphs (Havel-Hakimi) for growing n.  Each graph first
    takes 10 global super steps away from its structured start; both kinds of
    step then run from that same state (two handles, same seed)."""
    import torch
    from paper_1804_08487_gb300 import cb, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    series = []
    t0 = time.perf_counter()
    for log2n in range(10, 21, 2):
        n = 1 << log2n
        for kind, (a, b) in (("10-regular", (10, 11)), ("PLD([10,n/20),2)", (10, max(n // 20, 11)))):
            g = synth.powerlaw_graph(n, a, b, 2.0, 100 + log2n)
            row = {"graph": kind, "n": n, "m": g.m}
            for how in ("global", "uniform"):
                c = cb.Curveball(g.row_ptr, g.col, 7 + log2n)
                c.global_trades(10)
                c.set_option("swap_stats", 1)
                if how == "global":
                    c.global_trades(1)
                else:
                    c.uniform_trades(n // 2)
                done, possible = c.swap_counts()
                row[how] = done / possible if possible else None
                c.close()
            series.append(row)
    dt = time.perf_counter() - t0
    reg = [r for r in series if r["graph"] == "10-regular"]
    line = {
        "metric": "fraction of performed neighbourhood swaps", "value": reg[-1]["global"], "unit": "fraction",
        "n_gpus": 1, "steps": 1, "warmup": 10, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "swap fractions: 10-regular and PLD([10,n/20),2) graphs, n = 2^10..2^20, "
                               "one global trade vs n/2 uniform trades after 10 global super steps",
                   "parallelism": "single"},
        "series": series, "seconds": dt,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ input generation

def run_generate(args):
    """The workload's input graph generated on the device (include/cb_gen.h)
    against the host generator: wall time of each, and the device graph's
    sha256 against the stored digest of the host graph."""
    import hashlib
    import numpy as np
    import torch
    from paper_1804_08487_gb300 import cb
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    w = workload(args.workload if args.workload in ("n2^25", "n2^20", "n2^21", "n4096") else "n2^25")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rp, col, dseed = cb.generate_powerlaw(w.n, w.a, w.b, w.gamma, w.degree_seed)
    torch.cuda.synchronize()
    t_dev = time.perf_counter() - t0
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(rp.cpu().numpy(), dtype="<i8")).cast("B"))
    h.update(memoryview(np.ascontiguousarray(col.cpu().numpy(), dtype="<i4")).cast("B"))
    m = col.numel() // 2
    del rp, col
    torch.cuda.empty_cache()
    t1 = time.perf_counter()
    g = w.graph()
    t_host = time.perf_counter() - t1
    path = os.path.join(ROOT, "tests", "golden", f"plain_{args.workload.replace('^', 'p')}.json")
    want = json.load(open(path)).get("graph_sha256") if os.path.exists(path) else None
    line = {
        "metric": "input generation time (PLD degrees + Havel-Hakimi)", "value": t_dev, "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": t_dev * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "m": m, "degree_seed": dseed, "parallelism": "single"},
        "host_seconds": t_host, "host_cores": os.cpu_count(), "same_degree_seed": dseed == g.degree_seed,
        "graph_sha256_matches_stored": (h.hexdigest() == want) if want else None,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ edge autocorrelation

AUTOCORR_N = 2000            # Section 5.1: n = 2 10^3, PLD(a = 5, b, gamma = 2)
AUTOCORR_BS = (25, 750)
AUTOCORR_CHAINS = 8          # independent chains per b
AUTOCORR_STEPS = 6000        # super steps of each (not thinned) chain
AUTOCORR_KMAX = 64


def autocorr_graphs():
    """The chains of the autocorrelation workload: for each b, AUTOCORR_CHAINS
    PLD([5, b), 2) graphs on 2000 nodes (Havel-Hakimi), seeds 5000 + 100 b + i."""
    from paper_1804_08487_gb300 import synth
    graphs, seeds, groups = [], [], []
    for b in AUTOCORR_BS:
        for i in range(AUTOCORR_CHAINS):
            s = 5000 + 100 * b + i
            g = synth.powerlaw_graph(AUTOCORR_N, 5, b, 2.0, s)
            graphs.append((g.row_ptr, g.col))
            seeds.append(s)
            groups.append(b)
    return graphs, seeds, groups


def run_autocorr(args):
    """Section 5.1's mixing experiment with global trades: the fraction of
    edges still correlated with the start (BIC on the k-thinned presence
    series) as a function of the thinning k, for PLD([5, b), 2) graphs with
    n = 2000 and b in {25, 750}, 6000 super steps per chain; all chains of
    both b in one batch handle."""
    import numpy as np
    import torch
    from paper_1804_08487_gb300 import cb
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    graphs, seeds, groups = autocorr_graphs()
    stream = torch.cuda.Stream()
    e = cb.Ensemble(graphs, seeds, stream=stream)
    e.set_option("presence", AUTOCORR_STEPS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e.global_trades(AUTOCORR_STEPS)
    e.sync()
    t_chain = time.perf_counter() - t0
    series = {}
    t1 = time.perf_counter()
    for b in AUTOCORR_BS:
        corr = np.zeros(AUTOCORR_KMAX, dtype=np.int64)
        occ = 0
        for i, gb in enumerate(groups):
            if gb != b:
                continue
            c_i, _, o_i, _ = e.autocorr(AUTOCORR_KMAX, graph=i)
            corr += np.asarray(c_i, dtype=np.int64)
            occ += o_i
        series[f"b={b}"] = [round(float(x) / occ, 5) for x in corr]
    t_class = time.perf_counter() - t1
    e.close()
    frac25 = series["b=25"]
    k1 = next((k + 1 for k, f in enumerate(frac25) if f <= 0.01), None)
    line = {
        "metric": "fraction of edges still correlated (k-thinned presence series, BIC)", "value": k1,
        "unit": "smallest k with at most 1 % of edges correlated (b=25)", "n_gpus": 1, "steps": AUTOCORR_STEPS,
        "warmup": 0, "ms_per_step": t_chain / AUTOCORR_STEPS * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"edge autocorrelation: n={AUTOCORR_N}, PLD([5,b),2), b in {list(AUTOCORR_BS)}, "
                               f"{AUTOCORR_CHAINS} chains per b, {AUTOCORR_STEPS} global super steps, k = 1.."
                               f"{AUTOCORR_KMAX}", "parallelism": "batch handle"},
        "series": series, "seconds": {"chains_with_record": t_chain, "classification": t_class},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours

def run_ours(args):
    import numpy as np
    import torch
    from paper_1804_08487_gb300 import cb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args.workload)
    g = w.graph()
    seed = replica_seed(w.chain_seed, rank)          # each replica its own chain
    stream = torch.cuda.Stream()
    c = cb.Curveball(g.row_ptr, g.col, seed, stream=stream)
    if args.perm == "relaxed":
        c.set_option("relaxed", 1)
    c.set_option("timing", 1)
    # verify leg (untimed, inside the warm-up): the edge list after super step 1
    # of this chain against the oracle's stored digest for the workload
    parity = None
    if args.warmup >= 1 and rank == 0 and args.perm == "sort":
        c.global_trades(1)
        parity = verify_step1(args.workload, c, g.m)
        c.global_trades(args.warmup - 1)
    else:
        c.global_trades(args.warmup)
    c.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    c.global_trades(args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    stats = c.stats()
    phases = c.timings()
    # swap fraction of one more (untimed) super step (Appendix "Swaps performed
    # by Curveball and Global Curveball")
    c.set_option("swap_stats", 1)
    c.global_trades(1)
    sw_done, sw_all = c.swap_counts()
    t_max = max_over_ranks(t_ms, world)
    value = job_rate(world, g.m * args.steps, t_max / 1e3)

    # end to end through the C ABI with host buffers: create from pinned host
    # CSR (H2D inside), the same super steps, export to a pinned host buffer (D2H)
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    out_h = torch.empty(2 * g.m, dtype=torch.int32).pin_memory()
    c.close()
    barrier()
    t0 = time.perf_counter()
    c2 = cb.Curveball(rp_h, col_h, seed, stream=stream)
    if args.perm == "relaxed":
        c2.set_option("relaxed", 1)
    c2.global_trades(args.steps)
    c2.edges(out_h)
    c2.sync()
    e2e_s = time.perf_counter() - t0
    c2.close()
    e2e_max = max_over_ranks(e2e_s, world)
    h2d = (g.row_ptr.nbytes + g.col.nbytes) / args.steps
    d2h = (2 * g.m * 4) / args.steps
    batched = None
    if args.batched:
        graphs, seeds = ensemble_graphs()
        batched = measure_ensemble(graphs, seeds, stream, clocks=ClockSampler(local))

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    K = args.steps
    # roofline of the dominant kernel (algorithmic bytes per launch over its
    # event-timed launch duration); the whole step moves 16m + 24n bytes at
    # minimum (every directed entry read and written once, per node its key,
    # position and order)
    ntasks = (g.n + 1) // 2
    dom, dom_bytes, dom_ms, dom_entries = dominant_kernel(stats, phases, g.m, ntasks, K)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    phase_ms = {"threshold": phases["threshold_ms"] / K, "rebuild": phases["rebuild_ms"] / K}
    b_min = 16 * g.m + 24 * g.n
    step_gbs = b_min / (t_max / K / 1e3) / 1e9
    cpu_v, cpu_desc, _, _ = cpu_sample(w, perm=args.perm)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic", "config": config_of(w, g, world, args.perm),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": measured_traffic(dom, args.workload),
                     "traffic_unit": "DRAM bytes per launch (ncu, one pass, same workload)",
                     "algorithmic_bytes": dom_bytes, "launch_ms": dom_ms,
                     "peak_source": f"{peak_kind} hbm_gbs (burst copy)"},
        "roofline_step": {"bytes_min": b_min, "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                          "frac": step_gbs / peak},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": job_rate(world, g.m * K, e2e_max), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(stats.get("launches", 0)),
        "clocks": clk,
        "phase_ms_per_step": {"permutation": phases["permutation_ms"] / K, "threshold": phase_ms["threshold"],
                              "rebuild": phase_ms["rebuild"], "step": phases["step_ms"] / K},
        "class_ms_per_step": {CLASS_KERNELS[k]: phases.get(f"class{k}_ms", 0.0) / K for k in range(len(CLASS_KERNELS))},
        "dependency_passes_last_step": stats.get("passes"),
        "deferred_last_step": {"first_pass": stats.get("deferred"), "in_order": stats.get("inorder_trades")},
        "parity": parity,
        "swap_fraction": {"performed": sw_done, "possible": sw_all,
                          "fraction": sw_done / sw_all if sw_all else None, "of": "one global trade"},
    }
    if batched is not None:
        line["batched"] = batched
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------- reference

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "ensemble":
        value, cores, sample = ensemble_cpu_sample()
        line = {
            "impl": "reference", "metric": METRIC + " (batched ensemble)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": 5, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": ENSEMBLE_NAME, "sample": "graphs 0..31", "parallelism": "host processes"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    if args.workload == "autocorr":
        from oracle import Oracle
        from oracle import autocorr as ac
        from paper_1804_08487_gb300 import synth
        steps, kmax = 400, 16
        g = synth.powerlaw_graph(AUTOCORR_N, 5, 25, 2.0, 5000 + 100 * 25)
        t0 = time.perf_counter()
        o = Oracle(g.row_ptr, g.col, 5000 + 100 * 25)
        lists = [o.edges()]
        for _ in range(steps):
            o.superstep(1)
            lists.append(o.edges())
        corr, occ, _ = ac.fraction_correlated(lists, AUTOCORR_N, kmax)
        dt = time.perf_counter() - t0
        sample = f"oracle: one chain, n={AUTOCORR_N} PLD([5,25),2), {steps} super steps, k = 1..{kmax}"
        line = {
            "impl": "reference", "metric": "fraction of edges still correlated (k-thinned presence series, BIC)",
            "value": None, "unit": "fraction", "n_gpus": world, "steps": steps, "warmup": 0,
            "ms_per_step": dt / steps * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": "edge autocorrelation (oracle sample)", "parallelism": "single"},
            "series": {"b=25": [round(float(x) / occ, 5) for x in corr]},
            "cpu_baseline": {"value": dt, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": dt, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    if args.workload == "swaps":
        from oracle import Oracle
        from paper_1804_08487_gb300 import synth
        series = []
        t0 = time.perf_counter()
        for log2n in range(10, 15, 2):
            n = 1 << log2n
            for kind, (a, b) in (("10-regular", (10, 11)), ("PLD([10,n/20),2)", (10, max(n // 20, 11)))):
                g = synth.powerlaw_graph(n, a, b, 2.0, 100 + log2n)
                row = {"graph": kind, "n": n, "m": g.m}
                for how in ("global", "uniform"):
                    o = Oracle(g.row_ptr, g.col, 7 + log2n)
                    o.superstep(10)
                    o.swap_counts(reset=True)
                    if how == "global":
                        o.superstep(1)
                    else:
                        o.uniform_trades(n // 2)
                    done, possible = o.swap_counts()
                    row[how] = done / possible if possible else None
                series.append(row)
        dt = time.perf_counter() - t0
        reg = [r for r in series if r["graph"] == "10-regular"]
        line = {
            "impl": "reference", "metric": "fraction of performed neighbourhood swaps", "value": reg[-1]["global"],
            "unit": "fraction", "n_gpus": world, "steps": 1, "warmup": 10, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "swap fractions (oracle sample: n = 2^10..2^14)", "parallelism": "single"},
            "series": series,
            "cpu_baseline": {"value": reg[-1]["global"], "unit": "fraction", "cores": 1, "kind": "oracle",
                             "sample": f"n = 2^10..2^14, {dt:.1f} s"},
            "e2e": {"value": reg[-1]["global"], "unit": "fraction", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    if args.workload == "serving":
        from oracle import Oracle
        from paper_1804_08487_gb300 import synth
        work, t0, used = 0, time.perf_counter(), 0
        for i in range(10000):
            if used >= 16 or time.perf_counter() - t0 > 10.0:
                break
            w = synth.serving_request(i)
            if w.n > (1 << 16):
                continue
            g = w.graph()
            o = Oracle(g.row_ptr, g.col, w.chain_seed)
            o.superstep(w.supersteps)
            work += g.m * w.supersteps
            used += 1
        dt = time.perf_counter() - t0
        value = work / dt
        sample = f"oracle, serving requests with n <= 2^16 among the first ones ({used} requests), sequential"
        line = {
            "impl": "reference", "metric": METRIC + " (serving)", "value": value, "unit": UNIT, "n_gpus": world,
            "steps": used, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": SERVING_NAME, "sample": sample, "parallelism": "single"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    if args.workload == "uniform":
        w = workload(args.uniform_graph)
        vals = []
        for _ in range(max(args.steps, 1)):
            v, sample = uniform_cpu_sample(w, log2n=17)
            vals.append(v)
        value = statistics.median(vals)
        line = {
            "impl": "reference", "metric": UNIFORM_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w.name + ", n/2 uniform single trades per step", "parallelism": "single"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    w = workload(args.workload)
    from paper_1804_08487_gb300 import synth
    from oracle import Oracle
    log2n = 18
    g = synth.powerlaw_graph(1 << log2n, w.a, w.b, w.gamma, w.degree_seed)
    o = Oracle(g.row_ptr, g.col, w.chain_seed)
    o.superstep(args.warmup)
    t0 = time.perf_counter()
    o.superstep(args.steps)
    dt = time.perf_counter() - t0
    value = g.m * args.steps / dt
    sample = (f"oracle, n=2^{log2n} PLD([{w.a},{w.b}),{w.gamma:g}) Havel-Hakimi graph (m={g.m}) standing in "
              f"for {w.name}, {args.steps} super steps, sequential")
    full = workload(args.workload)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": full.name, "sample_n": g.n, "sample_m": g.m, "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "uniform":
        run_uniform(args)
    elif args.workload == "swaps":
        run_swaps(args)
    elif args.workload == "autocorr":
        run_autocorr(args)
    elif args.generate:
        run_generate(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
