#!/usr/bin/env python3
"""Throughput of the global Curveball super step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload n2^25|n2^20|n4096]

One "step" is one global super step (Def. "Undirected Global Trade",
Section 3.3) over the whole graph.  The metric is edge-trades/s = m * steps /
device time, the reciprocal of the paper's "walltime per edge and super step"
(Section 5.2).  The default workload is n=2^25 nodes with PLD([10,10000),2)
degrees realised by Havel-Hakimi (about 1.1e9 undirected edges, adjacency far
larger than L2).  With N>1 processes (torchrun) every rank randomises its own
replica of the graph with its own chain seed: the chain itself does not shard.

--impl reference times the sequential CPU oracle (the reference this project
is checked against) on a bounded sample of the same workload family.
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
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_sample(w, steps=1, log2n=19):
    """Oracle on a bounded sample of the workload family: the same degree law
    at n=2^log2n, `steps` super steps, one host core (the chain is sequential)."""
    from oracle import Oracle
    from paper_1804_08487_gb300 import synth
    g = synth.powerlaw_graph(1 << log2n, w.a, w.b, w.gamma, w.degree_seed)
    o = Oracle(g.row_ptr, g.col, w.chain_seed)
    t0 = time.perf_counter()
    o.superstep(steps)
    dt = time.perf_counter() - t0
    desc = (f"oracle, n=2^{log2n} PLD([{w.a},{w.b}),{w.gamma:g}) Havel-Hakimi graph (m={g.m}), "
            f"{steps} super step(s), sequential")
    return g.m * steps / dt, desc, g.m, dt


def config_of(w, g, world):
    return {"workload": w.name, "n": g.n, "m": g.m, "degree_seed": g.degree_seed, "chain_seed": w.chain_seed,
            "l2": "inputs larger than L2 (adjacency %.1f GB vs 129 MB L2)" % (g.m * 8 / 1e9),
            "parallelism": "replicas" if world > 1 else "single"}


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
    seed = w.chain_seed + rank          # each replica its own chain
    stream = torch.cuda.Stream()
    c = cb.Curveball(g.row_ptr, g.col, seed, stream=stream)
    c.set_option("timing", 1)
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
    t_max = t_ms
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    value = world * g.m * args.steps / (t_max / 1e3)

    # end to end through the C ABI with host buffers: create from pinned host
    # CSR (H2D inside), the same super steps, export to a pinned host buffer (D2H)
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    out_h = torch.empty(2 * g.m, dtype=torch.int32).pin_memory()
    c.close()
    barrier()
    t0 = time.perf_counter()
    c2 = cb.Curveball(rp_h, col_h, seed, stream=stream)
    c2.global_trades(args.steps)
    c2.edges(out_h)
    c2.sync()
    e2e_s = time.perf_counter() - t0
    c2.close()
    e2e_max = e2e_s
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_max = float(tt.item())
    h2d = (g.row_ptr.nbytes + g.col.nbytes) / args.steps
    d2h = (2 * g.m * 4) / args.steps

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    K = args.steps
    # algorithmic bytes: threshold phase reads every adjacency entry (4 B);
    # rebuild reads and writes every entry (8 B); the whole step moves
    # 16m + 24n bytes at minimum.
    phase_bytes = {"threshold": 2 * g.m * 4, "rebuild": 2 * g.m * 8}
    phase_ms = {"threshold": phases["threshold_ms"] / K, "rebuild": phases["rebuild_ms"] / K}
    dom = max(phase_ms, key=phase_ms.get)
    achieved = phase_bytes[dom] / (phase_ms[dom] / 1e3) / 1e9
    b_min = 16 * g.m + 24 * g.n
    step_gbs = b_min / (t_max / K / 1e3) / 1e9
    cpu_v, cpu_desc, _, _ = cpu_sample(w)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic", "config": config_of(w, g, world),
        "roofline": {"bound": "hbm", "kernel": f"{dom} phase", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "roofline_step": {"bytes_min": b_min, "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                          "frac": step_gbs / peak},
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": world * g.m * K / e2e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(stats.get("launches", 0)),
        "clocks": clk,
        "phase_ms_per_step": {"permutation": phases["permutation_ms"] / K, "threshold": phase_ms["threshold"],
                              "rebuild": phase_ms["rebuild"], "step": phases["step_ms"] / K},
        "dependency_passes_last_step": stats.get("passes"),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------- reference

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
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
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
