"""The N > 1 path of bench.py on the host: two gloo ranks (127.0.0.1) take the
job time as the slowest rank's and report whole-job throughput; the reference
arm runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]
    ms_max = bench.max_over_ranks(local_ms)
    value = bench.job_value(1000.0, world, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"ms_max": ms_max, "value": value, "env": list(bench.dist_env())}, f)


def test_two_gloo_ranks_agree_on_the_slowest(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(2)]
    for r, x in enumerate(res):
        assert x["ms_max"] == 150.0
        assert abs(x["value"] - 2 * 1000.0 / 0.150) < 1e-6
        assert x["env"] == [r, r, 2]


def test_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5) == 42.5
    assert bench.job_value(500.0, 1, 250.0) == 2000.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    class A:
        impl, gpus, steps, warmup, scale = "reference", 2, 1, 0, 1.0
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
