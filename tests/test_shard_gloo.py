"""Host side of the k-point sharding, on CPU: the partition of ng_shard_plan and the
torch.distributed exchange of shard.DistExchange between two gloo ranks (world size 2).

* Every rank's share is a run of whole 32-blocks (only the last rank may end ragged), and the
  shares tile 0..nk-1 in rank order.
* DistExchange.allgather moves the bytes unchanged and in rank order: after the call, both
  ranks hold bitwise the concatenation of both send buffers, for the block-sum size of the
  largest slice and for the single double of a distance.  Adding the gathered block sums in
  block order therefore gives every rank the same operands in the same order as one GPU
  holding all k-points (the kernel-side order is checked on the GPU in test_gpu_shard.py).
"""
import os

import numpy as np
import pytest
import torch
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    if not os.path.exists(ng.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    ng.load_library()
    return ng


@pytest.mark.parametrize("nk,nranks", [(512, 1), (512, 2), (512, 8), (80, 2), (80, 3), (33, 2), (1000, 7)])
def test_partition_is_whole_blocks_in_rank_order(ng, nk, nranks):
    g = ng.Grid(nt=30, ntau=20, nf=1, nbatch=1, korder=5, h=0.01, beta=10.0)
    plans = [ng.shard_plan(nk, r, nranks, g) for r in range(nranks)]
    nxt = 0
    for r, (b, c, nbytes) in enumerate(plans):
        assert b == nxt and c >= 1 and b % 32 == 0
        if r < nranks - 1:
            assert c % 32 == 0
        nxt = b + c
        maxb = max((cc + 31) // 32 for _, cc, _ in plans)
        assert nbytes >= maxb * (2 * 31 + 21) * 16
    assert nxt == nk


def test_partition_rejects_more_ranks_than_blocks(ng):
    with pytest.raises(ng.NgError):
        ng.shard_plan(40, 0, 3)        # two blocks of 32, three ranks


def _rank(rank, world, port, nk, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1911_01211_gb300 as ng
        from paper_1911_01211_gb300.shard import DistExchange
        g = ng.Grid(nt=30, ntau=20, nf=2, nbatch=1, korder=5, h=0.01, beta=10.0)
        ex = DistExchange(nk, g, "cpu")
        rng = np.random.default_rng(100 + rank)
        results = []
        for nbytes in (ex.send_bytes, 8, 16 * 37):
            n = nbytes // 8
            vals = torch.from_numpy(rng.standard_normal(n))
            ex.send[:n].copy_(vals)
            ex.recv.zero_()
            ex.allgather(nbytes)
            results.append((vals.numpy().copy(), ex.recv[:world * n].numpy().copy()))
        q.put((rank, ex.k_begin, ex.k_count, results))
    finally:
        dist.destroy_process_group()


def test_dist_exchange_two_gloo_ranks(ng):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    nk = 80
    procs = [ctx.Process(target=_rank, args=(r, 2, port, nk, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(2):
        r, b, c, res = q.get(timeout=300)
        got[r] = (b, c, res)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert got[0][0] == 0 and got[0][1] + got[1][1] == nk and got[1][0] == got[0][1]
    for i in range(3):
        sent = np.concatenate([got[0][2][i][0], got[1][2][i][0]])
        for r in (0, 1):
            assert np.array_equal(got[r][2][i][1], sent)     # bitwise, rank order
