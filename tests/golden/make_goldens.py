"""Write the stored expected values for the plain workloads.

Runs only the CPU oracle (oracle/) on the seeded synthetic inputs
(paper_1804_08487_gb300.synth) and records, per super step, the sha256 of the
canonical edge list (int32 pairs a<b, lexicographic, little endian).

    python tests/golden/make_goldens.py n4096 n2^20        # minutes
    python tests/golden/make_goldens.py n2^25 --steps 1,10 # hours, ~45 GB RAM
    python tests/golden/make_goldens.py ensemble256        # a few minutes, all cores

ensemble256 is the batched-ensemble workload: 256 independent graphs
(synth.ensemble_member), 50 super steps each; per graph the hashes after
super steps 1, 10 and 50.
"""
import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import Oracle  # noqa: E402
from paper_1804_08487_gb300 import synth  # noqa: E402


def edge_hash(edges):
    return hashlib.sha256(np.ascontiguousarray(edges, dtype="<i4").tobytes()).hexdigest()


ENSEMBLE_STEPS = (1, 10, 50)


def _ensemble_member(i):
    w = synth.ensemble_member(i)
    g = w.graph()
    graph_hash = hashlib.sha256(g.row_ptr.astype("<i8").tobytes() + g.col.astype("<i4").tobytes()).hexdigest()
    o = Oracle(g.row_ptr, g.col, w.chain_seed)
    hashes = {}
    done = 0
    for s in ENSEMBLE_STEPS:
        o.superstep(s - done)
        done = s
        hashes[str(s)] = edge_hash(o.edges())
    return {"index": i, "n": g.n, "m": o.m, "chain_seed": w.chain_seed, "gamma": w.gamma, "b": w.b,
            "graph_sha256": graph_hash, "edge_sha256_after_step": hashes}


def make_ensemble():
    import multiprocessing as mp

    t0 = time.time()
    with mp.get_context("spawn").Pool(max(1, os.cpu_count() - 1)) as pool:
        members = pool.map(_ensemble_member, range(256), chunksize=1)
    out = {
        "workload": "ensemble of 256 graphs: n log-uniform in [2^10, 2^16], PLD([4, n/16), gamma in [2, 3]), "
                    "seed 1000+i, 50 super steps",
        "graphs": members,
        "source": "tests/golden/make_goldens.py ensemble256 (CPU oracle only)",
    }
    path = os.path.join(HERE, "ensemble_256.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(f"wrote {path} ({time.time() - t0:.0f}s)", flush=True)


def main():
    if sys.argv[1:] == ["ensemble256"]:
        make_ensemble()
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="+", choices=sorted(synth.PLAIN))
    ap.add_argument("--steps", default="", help="comma-separated steps to record (default: every step)")
    args = ap.parse_args()
    for name in args.workloads:
        w = synth.PLAIN[name]
        t0 = time.time()
        g = w.graph()
        graph_hash = hashlib.sha256(g.row_ptr.astype("<i8").tobytes() + g.col.astype("<i4").tobytes()).hexdigest()
        print(f"{name}: n={g.n} m={g.m} degree_seed={g.degree_seed} ({time.time() - t0:.1f}s)", flush=True)
        want = set(int(s) for s in args.steps.split(",")) if args.steps else set(range(1, w.supersteps + 1))
        o = Oracle(g.row_ptr, g.col, w.chain_seed)
        del g
        hashes = {}
        for step in range(1, w.supersteps + 1):
            t1 = time.time()
            o.superstep(1)
            if step in want:
                hashes[str(step)] = edge_hash(o.edges())
            print(f"  step {step}: {time.time() - t1:.1f}s", flush=True)
        out = {
            "workload": w.name, "n": w.n, "m": o.m, "chain_seed": w.chain_seed,
            "degree_seed_used": int(w.degree_seed), "graph_sha256": graph_hash,
            "edge_sha256_after_step": hashes,
            "source": "tests/golden/make_goldens.py (CPU oracle only)",
        }
        path = os.path.join(HERE, f"plain_{name.replace('^', 'p')}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print("wrote", path, flush=True)


if __name__ == "__main__":
    main()
