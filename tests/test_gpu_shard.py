"""k-point sharding on one GPU: ranks emulated without any kernel waiting on another.

* ng_kreduce_partial over each rank's share, the block sums placed rank by rank as an allgather
  would place them, then ng_kreduce_combine: bitwise equal to the single-kernel
  ng_kreduce_timestep, with and without k-point weights, for 2 and 3 ranks and a ragged last
  block.
* ng_run_2b_sharded with two ranks as host threads (ThreadExchange: each rank's exchange waits
  for its own stream, meets the other at a host barrier and copies): G_k of every rank, Gloc and
  Sigma bitwise equal to one ng_run_2b over all k-points.
"""
import threading

import numpy as np
import pytest
import torch

from paper_1911_01211_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def _random_herm(ng, g, ldk, seed):
    H = ng.Herm(g, ldk=ldk)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    for t in H.tensors().values():
        t.copy_(torch.randn(t.shape, dtype=torch.complex128, generator=gen))
    return H


def _local(ng, g, H, b, c):
    """Herm with the problems b..b+c-1 of H (its own buffers, ldk = c)."""
    gl = ng.Grid(nt=g.nt, ntau=g.ntau, nf=g.nf, nbatch=c, korder=g.korder, h=g.h, beta=g.beta)
    L = ng.Herm(gl, zero=False)
    for name, t in H.tensors().items():
        getattr(L, name).copy_(t[..., b:b + c])
    return gl, L


def _slice_el(nt, ntau, n):
    return ntau + 1 if n < 0 else 2 * (n + 1) + ntau + 1


@pytest.mark.parametrize("nk,nranks", [(80, 2), (80, 3), (64, 2)])
@pytest.mark.parametrize("weighted", [False, True])
def test_partial_combine_equals_single_reduction(ng, nk, nranks, weighted):
    g = ng.Grid(nt=14, ntau=12, nf=2, nbatch=nk, korder=5, h=0.05, beta=2.0)
    ctx = ng.Context(5)
    G = _random_herm(ng, g, nk, seed=nk + nranks)
    wk = torch.rand(nk, dtype=torch.float64, device="cuda") if weighted else None
    L1, L2 = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    plans = [ng.shard_plan(nk, r, nranks, g) for r in range(nranks)]
    assert sum(p[1] for p in plans) == nk and plans[0][0] == 0
    maxb = max((c + 31) // 32 for _, c, _ in plans)
    local = [_local(ng, g, G, b, c) for b, c, _ in plans]
    for n in range(-1, g.nt + 1):
        ctx.kreduce_timestep(g, n, L1, G, wk=wk)
        per = _slice_el(g.nt, g.ntau, n) * g.nf * g.nf
        parts = []
        for (b, c, _), (gl, Gl) in zip(plans, local):
            part = torch.zeros(maxb * per, dtype=torch.complex128, device="cuda")
            ctx.kreduce_partial(gl, n, part, Gl, b, wk=wk[b:b + c].contiguous() if weighted else None)
            parts.append(part)
        # an allgather of maxb * per values per rank places rank r's block sums at r * maxb * per
        ctx.kreduce_combine(g, n, L2, torch.cat(parts), nk, nranks, weighted=weighted)
    torch.cuda.synchronize()
    for name in ("mat", "ret", "les", "tv"):
        assert torch.equal(getattr(L1, name), getattr(L2, name)), name
    ctx.close()


def _chain(ng, nk, nt, ntau):
    w = wl.chain_kspace(nk=nk, nt=nt, ntau=ntau, beta=4.0, h=0.05)
    g = ng.Grid(nt=w.nt, ntau=w.ntau, nf=1, nbatch=nk, korder=w.korder, h=w.h, beta=w.beta)
    return w, g


def test_two_thread_ranks_equal_one_gpu_run(ng):
    nk, nt, ntau = 80, 22, 16
    w, g = _chain(ng, nk, nt, ntau)
    # reference: every k-point in one run
    ctx = ng.Context(w.korder)
    G = ng.Herm(g)
    L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    it_ref = ctx.run_2b(g, G, L, S, e0, mf, U, corrector=w.corrector)
    torch.cuda.synchronize()
    ctx.close()

    from paper_1911_01211_gb300.shard import ThreadExchange
    nranks = 2
    group = ThreadExchange.Group(nranks, timeout=300.0)
    out = [None] * nranks
    errors = []

    def rank_main(r):
        try:
            b, c, _ = ng.shard_plan(nk, r, nranks, g)
            gl = ng.Grid(nt=nt, ntau=ntau, nf=1, nbatch=c, korder=w.korder, h=w.h, beta=w.beta)
            ex = ThreadExchange(group, nk, r, gl)
            cx = ng.Context(w.korder)
            Gr = ng.Herm(gl)
            Lr, Sr = ng.Herm(gl, ldk=1), ng.Herm(gl, ldk=1)
            er = ng.Func(gl, values=torch.from_numpy(np.ascontiguousarray(w.eps0[..., b:b + c])))
            mr = ng.Func(gl)
            Ur = ng.Func(gl, scalar=True)
            Ur.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
            its = cx.run_2b_sharded(gl, Gr, Lr, Sr, er, mr, Ur, ex, corrector=w.corrector)
            torch.cuda.synchronize()
            out[r] = (b, c, Gr, Lr, Sr, its)
            cx.close()
        except BaseException as e:          # noqa: BLE001 - reported by the main thread
            errors.append(e)
            group.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(nranks)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(600)
    assert not errors, errors
    for b, c, Gr, Lr, Sr, its in out:
        assert its == it_ref
        for name in ("mat", "ret", "les", "tv"):
            assert torch.equal(getattr(Gr, name), getattr(G, name)[..., b:b + c]), name
            assert torch.equal(getattr(Lr, name), getattr(L, name)), name
            assert torch.equal(getattr(Sr, name), getattr(S, name)), name
