"""Host logic of the benchmark's multi-rank mode (N > 1: independent seeded
replicas, one per rank, no collective on the data path): the job's time is
the slowest rank's and the throughput counts every rank's steps.  Two gloo
ranks on CPU, rendezvous on 127.0.0.1."""
import os
import socket

import numpy as np

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = bench.max_over_ranks(1.0 + rank, dist)  # rank 1 is the slow one
    q.put((rank, seconds, bench.job_rate(10, world, seconds)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_all_steps():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert [o[1] for o in out] == [2.0, 2.0]           # max over ranks on every rank
    assert all(abs(o[2] - 10.0) < 1e-12 for o in out)  # 10 steps x 2 ranks / 2 s


def test_single_process_passes_through():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(100, 1, 0.5) == 200.0


def test_replicas_step_distinct_seeded_states():
    from paper_1705_03838_gb300 import inputs

    w = inputs.WORKLOADS["medium"]
    args = (w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["amplitude"])
    a = inputs.seeded_state(*args, w["seed"] + 0, w["envelope"])
    b = inputs.seeded_state(*args, w["seed"] + 1, w["envelope"])
    assert a.shape == b.shape and not np.allclose(a, b)
