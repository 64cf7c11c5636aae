"""Uneven batch of independent embedded clusters (ng_batch_*) and the nf = 4, 8 time step,
against the FP64 oracle (1e-10 relative per component and problem)."""
import numpy as np
import pytest
import torch

from oracle import drivers
from oracle.contour import Func as OFunc
from oracle.contour import Herm as OHerm
from oracle.freegf import green_from_H
from oracle.weights import Weights
from paper_1911_01211_gb300 import workloads as wl
from tests.layout import funcs_to_device, herm_to_oracle, oracle_to_herm
from tests.test_gpu_parity import relerr

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def _oracle_cluster(p):
    W = Weights(p["korder"])
    N, T = p["nt"], p["ntau"]
    bath = green_from_H(N, T, p["hb"], 0.0, p["beta"], p["h"])
    S = OHerm(N, T, p["nf"])
    V = p["V"]
    for c in ("mat", "ret", "les", "tv"):
        setattr(S, c, np.einsum("ab,...bc,dc->...ad", V, getattr(bath, c), V.conj()))
    eps = OFunc(N, p["nf"])
    eps.val[:] = p["hs"]
    G = OHerm(N, T, p["nf"])
    drivers.solve_fixed_sigma(G, S, eps, 0.0, p["beta"], p["h"], W)
    return G


def _device_cluster(ng, ctx, p):
    g = ng.Grid(nt=p["nt"], ntau=p["ntau"], nf=p["nf"], nbatch=1, korder=p["korder"], h=p["h"], beta=p["beta"])
    gb = ng.Grid(nt=p["nt"], ntau=p["ntau"], nf=p["hb"].shape[0], nbatch=1, korder=p["korder"], h=p["h"],
                 beta=p["beta"])
    bath = ng.Herm(gb)
    ctx.green_from_H_const(gb, bath, p["hb"][None])
    S = ng.Herm(g)
    ctx.herm_sandwich(g, S, gb, bath, p["V"])
    eps = ng.Func(g)
    eps.val[:] = torch.from_numpy(np.asarray(p["hs"], complex))[None, :, :, None]
    G = ng.Herm(g)
    return g, G, S, eps


def test_uneven_batch_against_oracle(ng):
    probs = wl.uneven_clusters(nprob=6, seed=7, nt_range=(14, 30), ntau=16, h=0.05, beta_range=(2.0, 6.0))
    for p, d in zip(probs, (1, 2, 4, 8, 2, 8)):   # cover every orbital dimension
        if p["nf"] != d:
            rng = np.random.default_rng(d + p["nt"])
            p["nf"] = d
            p["hs"] = wl.random_hermitian(rng, d)
            p["V"] = rng.normal(0.0, 0.3, (d, 4))
    ctx = ng.Context(5)
    dev = [_device_cluster(ng, ctx, p) for p in probs]
    batch = ctx.batch([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev], [x[3] for x in dev])
    threads = batch.solve()
    torch.cuda.synchronize()
    assert threads in (64, 128, 256)
    assert ctx.status_sync() == (ng.NG_OK, 0)
    for p, (g, G, S, eps) in zip(probs, dev):
        ref = _oracle_cluster(p)
        e = relerr(herm_to_oracle(G, g, 0), ref)
        assert max(e.values()) < TOL, (p["nf"], p["nt"], e)
    batch.close()


@pytest.mark.parametrize("nb", [1, 2, 3])
def test_uniform_nf4_timestep_against_oracle(ng, nb):
    """The uniform-batch ng_dyson_timestep with nf = 4 (element-wise kernels), nb problems
    stored interleaved (odd nb included), one step from the oracle's history."""
    from tests.test_gpu_parity import _oracle_problem_set
    from oracle import dyson
    k, N, T, beta, h, d = 5, 20, 14, 2.5, 0.06, 4
    W, Gs, Ss, epss = _oracle_problem_set(d, nb, N, T, beta, h, k, seed=31)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    ctx = ng.Context(k)
    G, S, eps = ng.Herm(g), ng.Herm(g), ng.Func(g)
    oracle_to_herm(Ss, S, g)
    funcs_to_device(epss, eps)
    for n in (k + 1, 2 * k + 1, N):
        oracle_to_herm(Gs, G, g, nmax=n - 1)
        ctx.dyson_timestep(g, n, G, S, eps)
        torch.cuda.synchronize()
        for kb in range(nb):
            ref = Gs[kb].copy()
            dyson.dyson_timestep(n, ref, Ss[kb], epss[kb], 0.0, beta, h, W)
            got = herm_to_oracle(G, g, kb)
            for x, y in ((got.ret[n, :n + 1], ref.ret[n, :n + 1]), (got.les[:n + 1, n], ref.les[:n + 1, n]),
                         (got.tv[n], ref.tv[n])):
                assert np.abs(x - y).max() / np.abs(y).max() < TOL, (n, kb)
    assert ctx.status_sync() == (ng.NG_OK, 0)


def test_plain_solve_of_one_cluster_matches_the_batch(ng):
    """ng_solve_fixed on single nf = 4 and nf = 8 clusters (nbatch = 1, the plain path the batch
    is compared with) gives the batch's result."""
    probs = wl.uneven_clusters(nprob=2, seed=11, nt_range=(16, 24), ntau=14, h=0.05, beta_range=(2.0, 4.0))
    for p, d in zip(probs, (4, 8)):
        rng = np.random.default_rng(d)
        p["nf"] = d
        p["hs"] = wl.random_hermitian(rng, d)
        p["V"] = rng.normal(0.0, 0.3, (d, 4))
    ctx = ng.Context(5)
    dev = [_device_cluster(ng, ctx, p) for p in probs]
    batch = ctx.batch([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev], [x[3] for x in dev])
    batch.solve()
    torch.cuda.synchronize()
    for p, (g, G, S, eps) in zip(probs, dev):
        G2 = ng.Herm(g)
        ctx.solve_fixed(g, G2, S, eps)
        torch.cuda.synchronize()
        e = relerr(herm_to_oracle(G2, g, 0), herm_to_oracle(G, g, 0))
        assert max(e.values()) < 1e-12, (p["nf"], e)
    assert ctx.status_sync() == (ng.NG_OK, 0)
    batch.close()


def _random_history(rng, N, T, d):
    """Seeded random contour data on every stored element (a time step is a linear recursion,
    so its parity with the oracle holds for any history)."""
    X = OHerm(N, T, d)
    c = lambda *s: 0.3 * (rng.normal(0, 1, s) + 1j * rng.normal(0, 1, s))
    X.mat[...] = c(T + 1, d, d)
    X.tv[...] = c(N + 1, T + 1, d, d)
    low = np.tril(np.ones((N + 1, N + 1), bool))
    X.ret[low] = c(int(low.sum()), d, d)
    X.les[low.T] = c(int(low.sum()), d, d)
    return X


def test_uneven_batch_step_with_multichunk_boundary_sources(ng):
    """ng_batch_step for nf = 4 and nf = 8 problems with ntau = 300 and 270: the (A) rows' source
    sums run over n + ntau > 256 indices, i.e. over three or more chunks of 128 whose partial
    sums k_usrc adds in order (the path of the full-size uneven workload).  One global step
    from a seeded random history at n = 2k+1 (whole lesser column by (A)) and n = 24 (mixed),
    against the oracle's step of each problem."""
    from oracle import dyson
    k, h = 5, 0.05
    specs = [(4, 24, 300, 3.0), (8, 26, 270, 5.0)]
    rng = np.random.default_rng(2024)
    W = Weights(k)
    ctx = ng.Context(k)
    grids, Gs, Ss, es, oG, oS, oe = [], [], [], [], [], [], []
    for d, N, T, beta in specs:
        g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=1, korder=k, h=h, beta=beta)
        Go, So = _random_history(rng, N, T, d), _random_history(rng, N, T, d)
        eo = OFunc(N, d)
        eo.val[:] = wl.random_hermitian(rng, d)
        G, S, e = ng.Herm(g), ng.Herm(g), ng.Func(g)
        oracle_to_herm([Go], G, g)
        oracle_to_herm([So], S, g)
        funcs_to_device([eo], e)
        grids.append(g), Gs.append(G), Ss.append(S), es.append(e)
        oG.append(Go), oS.append(So), oe.append(eo)
    batch = ctx.batch(grids, Gs, Ss, es)
    for n in (2 * k + 1, 24):
        for g, G, Go in zip(grids, Gs, oG):
            oracle_to_herm([Go], G, g, nmax=n - 1)
        batch.step(n)
        torch.cuda.synchronize()
        assert ctx.status_sync() == (ng.NG_OK, 0)
        for (d, N, T, beta), g, G, Go, So, eo in zip(specs, grids, Gs, oG, oS, oe):
            ref = Go.copy()
            dyson.dyson_timestep(n, ref, So, eo, 0.0, beta, h, W)
            got = herm_to_oracle(G, g, 0)
            for name, x, y in (("ret", got.ret[n, :n + 1], ref.ret[n, :n + 1]),
                               ("les", got.les[:n + 1, n], ref.les[:n + 1, n]), ("tv", got.tv[n], ref.tv[n])):
                err = np.abs(x - y).max() / np.abs(y).max()
                assert err < TOL, (d, n, name, err)
    batch.close()
