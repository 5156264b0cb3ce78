"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks run the replica host logic
(environment, per-rank seeds, the slowest rank's time, the whole-job value), and the
reference arm's non-zero ranks exit without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.replica_env()
        ms = bench.max_over_ranks(10.0 + 5.0 * r, dist, torch.device("cpu"))
        seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(w)]
        dist.all_gather(seeds, torch.tensor([bench.replica_seed(7, r)]))
        out[rank] = (w, r, local, ms, bench.whole_job_value(w, 100, ms), [int(x) for x in seeds])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_seeds():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, local, ms, value, seeds = res[rank]
        assert (w, r, local) == (world, rank, rank)
        assert ms == 15.0                      # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 100 / 0.015)
        assert seeds == [7, 8]                 # one realisation per replica


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        warmup, steps, gpus = 3, 2, 2

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_single_process_environment(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.replica_env() == (1, 0, 0)
    assert bench.max_over_ranks(12.5, None, None) == 12.5
