"""The benchmark's multi-rank host logic under torch.distributed with the gloo
backend, world size 2, on CPU: the job time is the slowest rank's (max over
ranks), the whole-job throughput counts every rank's units against it (weak
scaling, shots sharded as independent replicas), and the barrier releases
both ranks."""

import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist

    w, r, local = bench.dist_setup("gloo")
    assert (w, r, local) == (ws, rank, rank)
    bench.barrier(w)
    ms = bench.max_over_ranks(w, 10.0 * (rank + 1), local)  # rank 0 took 10 ms, rank 1 20 ms
    out[rank] = (ms, bench.job_value(w, 8_000_000_000, ms))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_count_all_units():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    assert abs(res[0][1] - 2 * 8.0 / 0.020) < 1e-9  # 2 ranks x 8 G units in 20 ms = 800 G units/s
    assert res[0][1] == res[1][1]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(1, 3.5, 0) == 3.5
    assert bench.job_value(1, 8_000_000_000, 20.0) == 400.0
