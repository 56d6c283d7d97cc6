"""The N > 1 launch path of bench.py on CPU: two gloo ranks run the same helpers the
benchmark runs under NCCL (replicas only: each rank solves its own problem, the job's
time is the slowest rank's, the job's value counts every rank's iterations)."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        ms = 10.0 + 5.0 * rank                  # rank 1 is the slower replica
        job_ms = bench.max_over_ranks(ms, dist, "cpu")
        dist.barrier()
        res = {"rank": rank, "seed": bench.replica_seed(rank), "job_ms": job_ms,
               "value": bench.job_value(ws, 30, job_ms)}
        with open(os.path.join(out, f"r{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_value(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert [r["job_ms"] for r in res] == [15.0, 15.0]           # both see the slowest rank
    assert res[0]["seed"] != res[1]["seed"]                      # independent replicas
    assert res[0]["value"] == pytest.approx(2 * 30 / 0.015)     # all ranks' iterations / job time


def test_single_process_helpers():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 10, 20.0) == pytest.approx(500.0)
