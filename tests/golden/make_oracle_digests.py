#!/usr/bin/env python3
"""Write the oracle's result digests for the full-size benchmark graphs.

Calls only the CPU oracle (``oracle/``) and the seeded input generator
(``paper_1210_0748_gb300.synth``, which holds none of the method's
arithmetic).  For each workload it stores, in ``oracle_digests.json`` beside
this script: the workload's generator arguments, a SHA-256 of the generated
input arrays (so a test can tell a different input from a different result),
and the oracle's rounds, block counts and a SHA-256 of every level's
identifiers (uint32, original node order).  The GPU parity test compares the
CUDA path's levels with these digests, which pins every identifier of the
full-size result without storing 700 MB of expected values.

    python tests/golden/make_oracle_digests.py [--only NAME]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_digests.json")

# name -> (generator in synth, keyword arguments, k)
WORKLOADS = {
    "powerlaw_16m_256m": ("config_single_large", {}, 10),
}


def input_digest(g) -> str:
    h = hashlib.sha256()
    for a in (np.asarray(g.offsets, np.uint64), np.asarray(g.dst, np.uint32),
              np.asarray(g.edge_label), np.asarray(g.node_label, np.uint32)):
        h.update(str(a.dtype).encode())
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def level_digest(p) -> str:
    return hashlib.sha256(np.ascontiguousarray(p, dtype=np.uint32).tobytes()).hexdigest()


def make(name):
    import oracle
    from paper_1210_0748_gb300 import synth
    gen, kw, k = WORKLOADS[name]
    t0 = time.time()
    g = getattr(synth, gen)(**kw)
    t1 = time.time()
    r = oracle.kbisim_graph(g, k)
    t2 = time.time()
    rec = {"generator": gen, "kwargs": kw, "k": k, "nodes": g.num_nodes, "edges": g.num_edges,
           "input_sha256": input_digest(g), "rounds_run": r.rounds_run,
           "counts": [int(c) for c in r.counts],
           "level_sha256": [level_digest(r.pids[i]) for i in range(k + 1)],
           "oracle_seconds": round(t2 - t1, 1)}
    print("%s: generated in %.1f s, oracle %.1f s, rounds %d, counts %s"
          % (name, t1 - t0, t2 - t1, r.rounds_run, rec["counts"]), file=sys.stderr)
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only")
    args = ap.parse_args()
    try:
        with open(OUT) as f:
            table = json.load(f)
    except (OSError, ValueError):
        table = {}
    for name in WORKLOADS:
        if args.only and name != args.only:
            continue
        table[name] = make(name)
    with open(OUT, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
