"""The ncu launch-list summariser: only the last refinement of the list is
summarised, kernels map to the library's timing classes, and DRAM bytes per
call divide by rounds (signature classes) or levels (the others)."""
import csv
import json

import ncu_summary

HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _write(path, launches):
    """launches: list of (kernel name, ns, dram read bytes, dram write bytes)."""
    with open(path, "w", newline="") as f:
        f.write("==PROF== Connected to process 1\n")
        w = csv.writer(f, quoting=csv.QUOTE_ALL)
        w.writerow(HDR)
        for i, (name, ns, rd, wr) in enumerate(launches):
            base = [str(i), "1", "python", "h", "unnamed>::%s(int)" % name, "1", "13", "(256, 1, 1)", "(1, 1, 1)",
                    "0", "10.3", "Command line profiler metrics"]
            w.writerow(base + ["gpu__time_duration.sum", "nsecond", "{:,}".format(ns)])
            w.writerow(base + ["dram__bytes_read.sum", "Mbyte", str(rd / 1e6)])
            w.writerow(base + ["dram__bytes_write.sum", "byte", str(wr)])


def _refinement(scale):
    # level 0, then two rounds of signatures + grouping of levels 1 and 2
    out = [("k_label_hash", 1000, 10e6, 0), ("k_group_insert", 2000, 4e6, 0), ("k_word_counts", 100, 0, 0)]
    for _ in range(2):
        out += [("k_sig_small<0, 4, unsigned char, unsigned int>", 3000 * scale, 30e6, 10e6),
                ("k_hub_scatter<unsigned char, unsigned int>", 500, 5e6, 1e6),
                ("k_hub_bucket<unsigned int>", 700, 7e6, 1e6),
                ("k_group_insert", 2000, 4e6, 0), ("k_group_verify", 900, 8e6, 0), ("k_pid_fill", 400, 2e6, 2e6)]
    return out


def test_last_refinement_only(tmp_path):
    path = tmp_path / "launches.csv"
    # a warm-up refinement with different numbers, then the summarised one
    _write(path, [("k_check_ids", 5000, 1e9, 0)] + _refinement(10) + _refinement(1))
    launches = ncu_summary.load(str(path))
    assert len(launches) == 1 + 2 * 15
    assert launches[0][1] == "k_check_ids"
    assert launches[1][2]["dram__bytes_read.sum"] == 10e6  # Mbyte scaled to bytes
    per_kernel, total_t, per_call = ncu_summary.summarise(launches, rounds=2)
    assert per_kernel["k_sig_small<0, 4, unsigned char, unsigned int>"][0] == 2
    # times of the last refinement only (the first had 10x the small-kernel time)
    assert abs(per_kernel["k_sig_small<0, 4, unsigned char, unsigned int>"][1] - 6000e-9) < 1e-12
    assert "k_check_ids" not in per_kernel
    # per round for signatures, per level (rounds + 1) for grouping
    assert per_call["sig_small"] == (30e6 + 10e6)
    assert per_call["sig_hub"] == (5e6 + 1e6 + 7e6 + 1e6)
    assert per_call["group"] == 3 * 4e6 / 3
    assert per_call["verify"] == 2 * 8e6 / 3
    assert per_call["renumber"] == (2 * 4e6) / 3
    assert per_call["label_group"] == 10e6
    assert abs(total_t - sum(ns for _, ns, _, _ in _refinement(1)) * 1e-9) < 1e-12


def test_traffic_record_and_digest(tmp_path, monkeypatch):
    path = tmp_path / "launches.csv"
    _write(path, _refinement(1))
    md, rec = tmp_path / "out.md", tmp_path / "traffic.json"
    monkeypatch.setattr("sys.argv", ["ncu_summary", str(path), "--rounds", "2", "--workload", "w",
                                     "--command", "c", "--md", str(md), "--traffic", str(rec)])
    ncu_summary.main()
    r = json.loads(rec.read_text())
    assert r["source_sha256"] == ncu_summary.source_digest()
    assert r["rounds"] == 2 and r["workload"] == "w" and r["command"] == "c"
    assert r["dram_bytes_per_round"]["sig_small"] == 40_000_000
    text = md.read_text()
    assert "| `k_hub_bucket<unsigned int>` | 2 |" in text
    assert "Command: `c`" in text
    # the digest covers the round-kernel sources only and is stable
    assert ncu_summary.source_digest() == ncu_summary.source_digest()
    assert set(ncu_summary.ROUND_SOURCES) == {"kbisim_round.cu", "kbisim_internal.cuh"}


def test_per_round_split(tmp_path):
    path = tmp_path / "launches.csv"
    _write(path, [("k_check_ids", 5000, 1e9, 0)] + _refinement(10) + _refinement(1))
    cols = ncu_summary.per_round(ncu_summary.load(str(path)))
    # level 0 of the last refinement, then its two rounds
    assert len(cols) == 3
    assert abs(cols[0]["label_group"] - 1000e-9) < 1e-15 and abs(cols[0]["group"] - 2000e-9) < 1e-15
    for c in cols[1:]:
        assert abs(c["sig_small"] - 3000e-9) < 1e-15
        assert abs(c["sig_hub"] - 1200e-9) < 1e-15
        assert abs(c["renumber"] - 400e-9) < 1e-15
    lines = ncu_summary.round_table(cols)
    assert lines[0] == "| class | level 0 | round 1 | round 2 |"
    assert lines[-1].startswith("| total | 0.003 | 0.008 | 0.008 |")


def test_traffic_record_units(tmp_path, monkeypatch):
    """--units stores the (edges, nodes) each kernel class processes on the
    profiled workload, which bench.py scales the traffic by."""
    import bench
    from paper_1210_0748_gb300 import synth
    g = synth.uniform_zipf_graph(2000, 40000, zipf_s=1.2, dmax=6000, node_labels=4, edge_labels=4, seed=5)
    monkeypatch.setattr(bench, "workload", lambda scale, kind="single": (g, {}))
    path = tmp_path / "launches.csv"
    _write(path, _refinement(1))
    rec = tmp_path / "traffic.json"
    monkeypatch.setattr("sys.argv", ["ncu_summary", str(path), "--rounds", "2", "--scale", "0.5", "--units",
                                     "--traffic", str(rec)])
    ncu_summary.main()
    r = json.loads(rec.read_text())
    units = bench.class_units(g)
    assert r["class_units"] == {c: {"edges": e, "nodes": n} for c, (e, n) in units.items()}
    # every edge and node is in exactly one signature class
    assert sum(r["class_units"][c]["edges"] for c in ("sig_small", "sig_medium", "sig_hub")) == g.num_edges
    assert sum(r["class_units"][c]["nodes"] for c in ("sig_small", "sig_medium", "sig_hub")) == g.num_nodes
