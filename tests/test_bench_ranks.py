"""The multi-rank timing of bench.py (one process per GPU under torchrun): every rank reports
the slowest rank's time, which sets the job's rate (the k-points of all ranks over that time).
Run as two gloo ranks on the CPU."""
import os
import socket

import torch.multiprocessing as tmp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as td
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.5 + rank            # rank 1 is the slower one
        slowest = bench.max_over_ranks(t, device="cpu")
        out[rank] = slowest
    finally:
        td.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    world = 2
    with tmp.Manager() as m:
        out = m.dict()
        tmp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == 2.5


def test_single_process_is_its_own_maximum():
    assert bench.max_over_ranks(3.25, device="cpu") == 3.25
