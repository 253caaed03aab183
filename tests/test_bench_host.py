"""Host logic of bench.py on CPU: the rank-max aggregation over a 2-rank gloo
group (the multi-GPU path shards whole images, so this max is its only
collective), and the reference arm's JSON contract on a tiny sample."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = bench.max_over_ranks([10.0 + rank, 5.0 - rank], world)
    q.put((rank, out))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert res[0] == res[1] == [11.0, 5.0]


def test_max_over_ranks_single():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.0], 1) == [1.5, 2.0]


def test_reference_arm_contract(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "N_IMAGES", 1)
    monkeypatch.setattr(bench, "SIDE", 48)
    monkeypatch.setattr(bench, "host_cores", lambda: 3)
    line = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), 0, 1)
    assert line["impl"] == "reference" and line["unit"] == "images/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    json.dumps(line)
    assert bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), 1, 2) is None


def test_rounds_profile():
    sys.path.insert(0, ROOT)
    import bench
    # last change in phase -1 (none), 0..3 (round 1), 4 (round 2), 39 (round 10)
    sts = [{"last_change_phase": p} for p in (-1, 0, 3, 4, 39)]
    r = bench.rounds_profile(sts, bins=5)
    assert (r["jobs"], r["min"], r["max"], r["p50"]) == (5, 0, 10, 1)
    assert r["bin_width"] == 2 and r["hist"] == [3, 1, 0, 0, 1] and sum(r["hist"]) == 5
    assert bench.rounds_profile([]) == {"jobs": 0}
    json.dumps(r)
