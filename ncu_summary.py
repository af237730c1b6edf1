"""Benchmark helper: summaries of an ncu launch list of one refinement
(``python ncu_summary.py CSV ...``).

The CSV comes from ``ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,
dram__bytes_write.sum --csv`` over ``bench.py --steps 1 --warmup 2``: every
launch of the graph load and of three refinements (level 0 and each round).
Only the last refinement is summarised (from its level-0 kernel on):
the warm-up refinements have already grown any hub bucket that overflows, as
in the timed steps.  Two outputs:

* a Markdown table per kernel (launches, total time, share, DRAM bytes);
* a JSON record of DRAM bytes per call of each kernel class (per round for the
  signature classes, per level for grouping, verification and renumbering),
  stamped with a digest of the kernel sources, which ``bench.py`` reports as
  the measured traffic of the dominant class while the sources are unchanged.

Per-launch times under ncu are cold-cache and serialised: compare shares, not
absolute times.
"""
from __future__ import annotations

import argparse
import collections
import csv
import hashlib
import json
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1210_0748_gb300", "csrc")

# kernel name -> class of the library's timing (kbisim_kernel_times)
CLASS_OF = [
    (r"k_label_hash|k_l0_collect", "label_group"),
    (r"k_sig_small|k_sig_chunk<128, 33,", "sig_small"),  # the library times out-degree 33..64 with <= 32
    (r"k_sig_chunk", "sig_medium"),
    (r"k_hub_sample|k_hub_chunk|k_hub_scatter|k_hub_bucket|k_hub_finish", "sig_hub"),
    (r"k_group_insert", "group"),
    (r"k_group_verify|k_verify_long", "verify"),
    (r"k_word_counts|k_tile_sum64|k_scan_tiles|k_tile_scan64|k_pid_fill|k_l0_fill", "renumber"),
]

UNITS = {"ns": 1e-9, "nsecond": 1e-9, "us": 1e-6, "usecond": 1e-6, "ms": 1e-3, "msecond": 1e-3,
         "s": 1.0, "second": 1.0, "byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9,
         "KB": 1e3, "MB": 1e6, "GB": 1e9}


# Sources of the kernels a refinement round runs (the timed classes).
ROUND_SOURCES = ("kbisim_round.cu", "kbisim_internal.cuh")


def source_digest() -> str:
    """sha256 over the sources of the round kernels (file names and contents)."""
    h = hashlib.sha256()
    for name in ROUND_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def short_name(name: str) -> str:
    """Kernel name with its template arguments, without namespaces and parameters."""
    m = re.search(r"(k_[A-Za-z_0-9]+)(<[^(]*>)?\(", name)
    return (m.group(1) + (m.group(2) or "")) if m else name[:60]


def load(path: str):
    """Launches in order: list of (id, name, {metric: value in s or bytes})."""
    rows = list(csv.reader(open(path)))
    hdr = None
    out = collections.OrderedDict()
    for r in rows:
        if r and r[0] == "ID":
            hdr = r
            continue
        if not hdr or len(r) != len(hdr):
            continue
        d = dict(zip(hdr, r))
        key = int(d["ID"])
        v = float(d["Metric Value"].replace(",", "")) * UNITS.get(d["Metric Unit"], 1.0)
        ent = out.setdefault(key, [short_name(d["Kernel Name"]), {}])
        ent[1][d["Metric Name"]] = v
    return [(k, v[0], v[1]) for k, v in out.items()]


def class_of(name: str):
    for pat, cls in CLASS_OF:
        if re.match(pat, name):
            return cls
    return None


def summarise(launches, rounds: int):
    first = max((i for i, (_, n, _) in enumerate(launches) if n.startswith(("k_label_hash", "k_l0_collect"))),
                default=0)
    refine = launches[first:]
    per_kernel = collections.OrderedDict()
    per_class = collections.defaultdict(float)
    total_t = 0.0
    for _, name, m in refine:
        t = m.get("gpu__time_duration.sum", 0.0)
        b = m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        k = per_kernel.setdefault(name, [0, 0.0, 0.0])
        k[0] += 1
        k[1] += t
        k[2] += b
        total_t += t
        cls = class_of(name)
        if cls:
            per_class[cls] += b
    calls = {c: (rounds if c.startswith("sig") else rounds + 1) for c in per_class}
    calls["label_group"] = 1
    per_call = {c: per_class[c] / max(calls[c], 1) for c in per_class}
    return per_kernel, total_t, per_call


def per_round(launches):
    """Time of each kernel class per level of the last refinement: level 0,
    then one column per round.  A round starts at its first signature kernel
    after the previous level's renumbering."""
    first = max((i for i, (_, n, _) in enumerate(launches) if n.startswith(("k_label_hash", "k_l0_collect"))),
                default=0)
    cols = [collections.defaultdict(float)]
    in_sig = False
    for _, name, m in launches[first:]:
        cls = class_of(name) or "other"
        if cls.startswith("sig") and not in_sig:
            cols.append(collections.defaultdict(float))
        in_sig = cls.startswith("sig")
        cols[-1][cls] += m.get("gpu__time_duration.sum", 0.0)
    return cols


def round_table(cols):
    """Markdown table of per_round's columns (ms)."""
    order = ["label_group", "sig_small", "sig_medium", "sig_hub", "group", "verify", "renumber", "other"]
    names = ["level 0"] + ["round %d" % i for i in range(1, len(cols))]
    lines = ["| class | " + " | ".join(names) + " |", "|---|" + "---:|" * len(cols)]
    for c in order:
        if any(c in col for col in cols):
            lines.append("| %s | " % c + " | ".join("%.3f" % (col.get(c, 0.0) * 1e3) for col in cols) + " |")
    lines.append("| total | " + " | ".join("%.3f" % (sum(col.values()) * 1e3) for col in cols) + " |")
    return lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("csv")
    ap.add_argument("--rounds", type=int, required=True, help="rounds the profiled refinement ran")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--workload", default="")
    ap.add_argument("--command", default="")
    ap.add_argument("--md", help="write the per-kernel table here")
    ap.add_argument("--traffic", help="write the per-class DRAM bytes record here")
    ap.add_argument("--units", action="store_true",
                    help="store the (edges, nodes) each class processes on the profiled workload (the bench's "
                         "single-graph generator at --scale) in the traffic record, for scaling to other sizes")
    a = ap.parse_args()
    launches = load(a.csv)
    per_kernel, total_t, per_call = summarise(launches, a.rounds)
    dram = any("dram__bytes_read.sum" in m for _, _, m in launches)
    lines = ["# Launch list: one refinement, %s" % a.workload, "",
             "Command: `%s`" % a.command, "",
             "%d rounds; per-launch times are cold-cache and serialised (compare shares)." % a.rounds, "",
             "| kernel | launches | total ms | share |" + (" DRAM MB |" if dram else ""),
             "|---|---:|---:|---:|" + ("---:|" if dram else "")]
    for name, (n, t, b) in sorted(per_kernel.items(), key=lambda kv: -kv[1][1]):
        lines.append("| `%s` | %d | %.3f | %.1f%% |" % (name, n, t * 1e3, 100 * t / total_t) +
                     (" %.1f |" % (b / 1e6) if dram else ""))
    lines += ["", "Per level (ms, same launches; a round is its signatures, grouping, verification and renumbering):",
              ""] + round_table(per_round(launches))
    if dram:
        lines += ["", "DRAM bytes per call of each kernel class (per round for signatures, per level otherwise):",
                  ""]
        for c, b in sorted(per_call.items()):
            lines.append("* %s: %.1f MB" % (c, b / 1e6))
    text = "\n".join(lines) + "\n"
    if a.md:
        with open(a.md, "w") as f:
            f.write(text)
    else:
        print(text)
    if a.traffic:
        rec = {"source_sha256": source_digest(), "scale": a.scale, "workload": a.workload,
               "command": a.command, "rounds": a.rounds,
               "dram_bytes_per_round": {c: round(b) for c, b in per_call.items()}}
        if a.units:
            import bench
            g, _ = bench.workload(a.scale)
            rec["class_units"] = {c: {"edges": e, "nodes": n} for c, (e, n) in bench.class_units(g).items()}
        with open(a.traffic, "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
