"""World-size-2 gloo checks of the benchmark's multi-GPU host logic (replicas, max over ranks) on CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    seeds = bench.replica_seeds(rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, seeds))


def test_max_over_ranks_and_distinct_replicas():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [t for _, t, _ in out] == [15.0, 15.0]
    assert out[0][2] != out[1][2]        # replicas draw different links and momenta


def test_reference_arm_other_ranks_do_nothing(capsys):
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""


@pytest.mark.slow
def test_reference_arm_json_line(capsys):
    """Rank 0 of `bench.py --impl reference` times the oracle on its bounded sample and prints one JSON
    line with the benchmark's metric, unit and direction, a cpu_baseline of kind "oracle" and an e2e
    object that moves no bytes between host and device."""
    import argparse
    import json

    import bench
    args = argparse.Namespace(steps=1, warmup=0, nsteps=bench.NSTEPS)
    assert bench.run_reference(args, rank=0, world=1) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "traj/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    # each step is a bounded sample covering units_per_step of one trajectory: value = units / seconds
    assert d["value"] > 0 and 0 < d["units_per_step"] < 1
    assert abs(d["value"] - d["units_per_step"] / (d["ms_per_step"] * 1e-3)) < 1e-9 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "traj/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("32^4 full RMHMC")
