"""The N > 1 host logic of bench.py (one process per GPU, replicas): barrier, max over ranks and
rank-0-only output, exercised with world_size 2 over gloo on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    # each rank's time differs; every rank gets the maximum (the job's time)
    mx = bench.max_over_ranks(10.0 + rank, ws, torch.device("cpu"))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(mx))
    bench.barrier(ws)
    dist.destroy_process_group()


def test_two_ranks_barrier_and_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    assert vals == [11.0, 11.0]


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=3)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
