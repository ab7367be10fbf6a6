"""The multi-rank reporting of bench.py on CPU: two gloo ranks (replicas) with different timed
regions; the whole-job rate counts every rank's solves over the slowest rank's time, and both
ranks agree on it."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 100 (r + 1) ms for 5 solves
        rate, ms_max = bench.whole_job_rate(dist, world, 5, 100.0 * (rank + 1), "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"rate": rate, "ms_max": ms_max}, f)
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms_max"] == 200.0
        assert r["rate"] == pytest.approx(world * 5 / 0.2)


def test_single_rank_rate_needs_no_process_group():
    import bench
    rate, ms = bench.whole_job_rate(None, 1, 4, 250.0, "cpu")
    assert ms == 250.0 and rate == pytest.approx(16.0)
