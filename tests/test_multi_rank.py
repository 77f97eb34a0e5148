"""Host-side logic of the multi-GPU bench path on CPU: every rank detects its
own slots (no collective on the data path); the job's rate is the total over
ranks divided by the slowest rank's time.  world_size 2, gloo, 127.0.0.1."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rate, slowest = bench.whole_job_rate(1000.0, 1.0 + rank)
        m = bench.max_over_ranks(float(10 * rank + 3))
        q.put((rank, rate, slowest, m))
    finally:
        dist.destroy_process_group()


def test_weak_scaling_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, slowest, m in res:
        assert slowest == 2.0            # slowest rank's time
        assert rate == 2 * 1000.0 / 2.0  # all ranks' units over that time
        assert m == 13.0


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.whole_job_rate(500.0, 2.0) == (250.0, 2.0)
    assert bench.max_over_ranks(4.5) == 4.5


def test_reference_arm_nonzero_ranks_do_no_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    args = type("A", (), dict(workload="4x4-qpsk-64sc", snr_index=0, n_pe=16, steps=1,
                              warmup=1, gpus=2))()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
