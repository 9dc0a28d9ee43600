"""The multi-process side of bench.py on CPU: two gloo ranks aggregate a
replicated run (units summed over ranks, time = slowest rank), and the
reference arm prints only on rank 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist = bench.dist_init("gloo")
    units, secs = bench.aggregate(100.0 * (rank + 1), 2.0 + rank, dist)
    bench.barrier(dist)
    results[rank] = (units, secs)
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    results = mgr.dict()
    mp.start_processes(_worker, args=(2, port, results), nprocs=2, join=True, start_method="spawn")
    assert results[0] == (300.0, 3.0)
    assert results[1] == (300.0, 3.0)


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0, None) == (5.0, 2.0)


def test_reference_arm_exits_quietly_off_rank0(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.main(["--impl", "reference"]) == 0
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("name", ["tvs100", "tvs2000", "tvs4000"])
def test_config_record_is_complete(name):
    import bench
    w = bench.workload(name)
    c = bench.config_of(name, w, 123, 1)
    assert c["workload"].startswith(name) and c["evals_per_dem"] == 123
