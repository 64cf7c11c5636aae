"""GW on the GPU against the oracle (oracle/gw.py, oracle/drivers.run_gw):

* ng_gw_polarization_timestep / ng_gw_sigma_timestep slice by slice from seeded random G and
  chi (d = 1, 2; the random equal-time G^< is not anti-hermitian, so the diagonal rule is
  exercised) at 1e-14 relative;
* the bosonic convolution P * P (grid.sig = +1) at 1e-12;
* the self-consistent ng_run_gw for the Hubbard dimer after an interaction quench, the open
  4-site chain (nf = 4) and a k-space chain (local GW), G, Sigma and chi compared on every
  stored element at 1e-10;
* the k-space GW (Eqs. Sigmak, Pol): the FFT-based slice calls against the oracle's momentum
  sums (nk = 4, 32, 128 radix-2, nk = 6, 12 direct transform) at 1e-13, and ng_run_gw_kspace
  against drivers.run_gw_kspace at 1e-10.
"""
import numpy as np
import pytest
import torch

from oracle import conv, drivers, gw
from oracle.contour import Func as OFunc
from oracle.contour import Herm as OHerm
from oracle.weights import Weights
from paper_1911_01211_gb300 import workloads as wl
from tests.layout import herm_to_oracle, oracle_to_herm
from tests.test_gpu_parity import _grid, _ofunc, _status_ok, relerr
from tests.test_gpu_vie2 import _random_herm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _slice(X, n):
    if n == -1:
        return [X.mat]
    return [X.ret[n, :n + 1], X.les[:n + 1, n], X.tv[n]]


@pytest.mark.parametrize("d", [1, 2])
def test_gw_slice_kernels_match_oracle(ng, d):
    N, T, beta, h, k = 14, 16, 2.0, 0.05, 5
    rng = np.random.default_rng(1700 + d)
    Go = _random_herm(rng, N, T, d, 1.0)
    Xo = _random_herm(rng, N, T, d, 0.7)
    Xo.sig = +1
    u = 0.9 + 0.2 * rng.random(N + 2)
    Uo = OFunc(N, 1)
    Uo.val[:, 0, 0] = u
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=1, korder=k, h=h, beta=beta)
    G, X = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    P, K, Kcc, S = (ng.Herm(g, ldk=1) for _ in range(4))
    oracle_to_herm([Go], G, g)
    oracle_to_herm([Xo], X, g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(u.astype(complex))
    ctx = ng.Context(k)
    chain = gw.GW(N, T, d, beta, h, Weights(k))
    chain.chi = Xo
    So = OHerm(N, T, d)
    for n in (-1, 0, 1, 6, N):
        ctx.gw_polarization_timestep(g, n, P, K, Kcc, G, U)
        ctx.gw_sigma_timestep(g, n, S, G, X, U)
        torch.cuda.synchronize()
        chain._kernel(n, Go, Uo)
        chain._sigma(n, Go, Uo, So)
        for name, dev, ref in (("P", P, chain.P), ("K", K, chain.K), ("Kcc", Kcc, chain.Kcc), ("Sigma", S, So)):
            got = herm_to_oracle(dev, g, 0)
            for x, y in zip(_slice(got, n), _slice(ref, n)):
                assert _rel(x, y) < 1e-14, (name, n, _rel(x, y))
    _status_ok(ctx, ng)
    ctx.close()


@pytest.mark.parametrize("d", [1, 2])
def test_bosonic_convolution_matches_oracle(ng, d):
    N, T, beta, h, k = 14, 16, 2.0, 0.05, 5
    rng = np.random.default_rng(1800 + d)
    A = _random_herm(rng, N, T, d, 0.5)
    B = _random_herm(rng, N, T, d, 0.5)
    A.sig = B.sig = +1
    W = Weights(k)
    ref = OHerm(N, T, d, sig=+1)
    for n in range(-1, N + 1):
        conv.convolution_timestep(n, ref, A, A, None, B, B, W, beta, h)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=1, korder=k, h=h, beta=beta, sig=+1)
    dA, dB, dC = ng.Herm(g), ng.Herm(g), ng.Herm(g)
    oracle_to_herm([A], dA, g)
    oracle_to_herm([B], dB, g)
    ctx = ng.Context(k)
    for n in range(-1, N + 1):
        ctx.convolution_timestep(g, n, dC, dA, dA, None, dB, dB)
    torch.cuda.synchronize()
    e = relerr(herm_to_oracle(dC, g, 0), ref)
    assert max(e.values()) < 1e-12, e
    _status_ok(ctx, ng)
    ctx.close()


def _run_gw_both(ng, w):
    g = _grid(ng, w)
    ctx = ng.Context(w.korder)
    G = ng.Herm(g)
    L, S, X = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    iters = ctx.run_gw(g, G, L, S, X, e0, mf, U, corrector=w.corrector)
    _status_ok(ctx, ng)
    ctx.close()
    W = Weights(w.korder)
    eps0 = [_ofunc(w.eps0, kb) for kb in range(w.nbatch)]
    Uo = OFunc(w.nt, 1)
    Uo.val[:, 0, 0] = w.U
    st, chain = drivers.run_gw(eps0, Uo, w.nt, w.ntau, w.beta, w.h, W, corrector=w.corrector)
    return g, G, S, X, st, chain, iters


def _check(got, ref, tol=1e-10):
    e = relerr(got, ref)
    assert max(e.values()) < tol, e


def test_run_gw_hubbard_dimer(ng):
    """The Hubbard dimer (nf = 2, quench U: 1 -> 2) with the GW self-energy."""
    w = wl.hubbard_dimer(nt=30, ntau=24, beta=5.0, h=0.05)
    g, G, S, X, st, chain, iters = _run_gw_both(ng, w)
    _check(herm_to_oracle(G, g, 0), st.G[0])
    _check(herm_to_oracle(S, g, 0), st.S)
    _check(herm_to_oracle(X, g, 0), chain.chi)


def test_run_gw_four_site_chain(ng):
    """Real-space GW of the open 4-site Hubbard chain at quarter filling after the quench of the
    first site (the paper's M = 4 chain example: U = 1.5, nbar = 1/4, w0 = 5; nf = 4 contour
    functions, chi by the nf = 4 vie2) against drivers.run_gw on every stored element."""
    w = wl.hubbard_chain(M=4, nt=20, ntau=16, beta=5.0, h=0.05, U=1.5, w0=5.0, mu=-1.0, nbar=0.25)
    g = _grid(ng, w)
    ctx = ng.Context(w.korder)
    G = ng.Herm(g)
    L, S, X = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    ctx.run_gw(g, G, L, S, X, e0, mf, U, corrector=w.corrector, nbar=w.nbar)
    _status_ok(ctx, ng)
    ctx.close()
    Uo = OFunc(w.nt, 1)
    Uo.val[:, 0, 0] = w.U
    st, chain = drivers.run_gw([_ofunc(w.eps0, 0)], Uo, w.nt, w.ntau, w.beta, w.h, Weights(w.korder), mu=w.mu,
                               nbar=w.nbar, corrector=w.corrector)
    _check(herm_to_oracle(G, g, 0), st.G[0])
    _check(herm_to_oracle(S, g, 0), st.S)
    _check(herm_to_oracle(X, g, 0), chain.chi)


def test_run_gw_local_on_kspace_chain(ng):
    """A k-space chain (nk = 4, nf = 1) with the local GW self-energy of Gloc."""
    w = wl.chain_kspace(nk=4, nt=24, ntau=20, beta=4.0, h=0.05)
    g, G, S, X, st, chain, iters = _run_gw_both(ng, w)
    for kb in range(w.nbatch):
        _check(herm_to_oracle(G, g, kb), st.G[kb])
    _check(herm_to_oracle(S, g, 0), st.S)
    _check(herm_to_oracle(X, g, 0), chain.chi)


# ---- k-space GW (Eqs. Sigmak, Pol): FFTs along k on the GPU, momentum sums in the oracle ----
@pytest.mark.parametrize("nk", [4, 6, 12, 32, 128])
def test_gw_kspace_slices_match_oracle(ng, nk):
    """ng_gw_kspace_polarization_timestep / _sigma_timestep (radix-2 FFT for nk = 4, 32 and the
    benchmark's 128, the direct transform for nk = 6, 12) against the oracle's momentum sums from
    seeded random G_k and chi_k."""
    N, T, beta, h, k = 12, 14, 2.0, 0.05, 5
    rng = np.random.default_rng(1900 + nk)
    Gk = [_random_herm(rng, N, T, 1, 1.0) for _ in range(nk)]
    Xk = [_random_herm(rng, N, T, 1, 0.7) for _ in range(nk)]
    for x in Xk:
        x.sig = +1
    u = 0.9 + 0.2 * rng.random(N + 2)
    Uo = OFunc(N, 1)
    Uo.val[:, 0, 0] = u
    g = ng.Grid(nt=N, ntau=T, nf=1, nbatch=nk, korder=k, h=h, beta=beta)
    G, X, P, K, Kcc, S = (ng.Herm(g) for _ in range(6))
    oracle_to_herm(Gk, G, g)
    oracle_to_herm(Xk, X, g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(u.astype(complex))
    ctx = ng.Context(k)
    chain = gw.GWk(N, T, nk, beta, h, Weights(k), *gw.ring_tables(nk))
    chain.chi = Xk
    Sk = [OHerm(N, T, 1) for _ in range(nk)]
    for n in (-1, 0, 1, 6, N):
        ctx.gw_kspace_polarization_timestep(g, n, P, K, Kcc, G, U)
        ctx.gw_kspace_sigma_timestep(g, n, S, G, X, U)
        torch.cuda.synchronize()
        chain._kernel(n, Gk, Uo)
        chain._sigma(n, Gk, Uo, Sk)
        for name, dev, refs in (("P", P, chain.P), ("K", K, chain.K), ("Kcc", Kcc, chain.Kcc), ("Sigma", S, Sk)):
            scale = max(np.abs(np.concatenate([np.ravel(y) for ref in refs for y in _slice(ref, n)])).max(), 1e-300)
            for kb in range(nk):
                got = herm_to_oracle(dev, g, kb)
                for x, y in zip(_slice(got, n), _slice(refs[kb], n)):
                    err = float(np.abs(x - y).max() / scale)
                    assert err < 1e-13, (name, n, kb, err)
    _status_ok(ctx, ng)
    ctx.close()


def test_run_gw_kspace_chain(ng):
    """The self-consistent k-space GW of the chain_kspace workload (nk = 4, Peierls pulse)
    against drivers.run_gw_kspace: G_k, Sigma_k and chi_k on every stored element."""
    w = wl.chain_kspace(nk=4, nt=20, ntau=16, beta=4.0, h=0.05)
    g = _grid(ng, w)
    ctx = ng.Context(w.korder)
    G, S, X = ng.Herm(g), ng.Herm(g), ng.Herm(g)
    L = ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    ctx.run_gw_kspace(g, G, L, S, X, e0, mf, U, corrector=w.corrector)
    _status_ok(ctx, ng)
    ctx.close()
    W = Weights(w.korder)
    eps0 = [_ofunc(w.eps0, kb) for kb in range(w.nbatch)]
    Uo = OFunc(w.nt, 1)
    Uo.val[:, 0, 0] = w.U
    st, chain = drivers.run_gw_kspace(eps0, Uo, w.nt, w.ntau, w.beta, w.h, W, *gw.ring_tables(w.nbatch),
                                      corrector=w.corrector)
    for kb in range(w.nbatch):
        _check(herm_to_oracle(G, g, kb), st.G[kb])
        _check(herm_to_oracle(S, g, kb), st.Sk[kb])
        _check(herm_to_oracle(X, g, kb), chain.chi[kb])
