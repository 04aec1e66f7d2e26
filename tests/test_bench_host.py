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


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys of the benchmark line, on the GPU arm's metric,
    unit and workload."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "timesteps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["config"]["workload"].startswith("pipe medium")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
