"""ng_vie2_mat / ng_vie2_start / ng_vie2_timestep against the oracle's integral-form solver
(oracle/vie2.py, mixed schedule) at 1e-10 relative: a whole solve of downfolded clusters
(F = -g0 * Sigma, F^ddagger = -Sigma * g0, Q = g0; d = 1, 2, two problems with their own
kernels), and the Matsubara, start-up and single time steps from seeded random data with a
kernel F that is not hermitian symmetric (its partner Fcc independent), so every use of Fcc is
checked."""
import numpy as np
import pytest
import torch

from oracle import vie2
from oracle.contour import Herm as OHerm
from oracle.freegf import green_from_H
from oracle.weights import Weights
from tests.layout import herm_to_oracle, oracle_to_herm
from tests.test_oracle_vie2 import _cluster, _convolve_all

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _compare(G, ref, N, upto=None):
    upto = N if upto is None else upto
    low = np.tril(np.ones((N + 1, N + 1), bool))
    low[upto + 1:] = False
    return {"mat": _rel(G.mat, ref.mat), "ret": _rel(G.ret[low], ref.ret[low]),
            "les": _rel(G.les[low.T], ref.les[low.T]), "tv": _rel(G.tv[:upto + 1], ref.tv[:upto + 1])}


@pytest.mark.parametrize("d", [1, 2, 4])
def test_vie2_downfolding_solve(ng, d):
    k, N, T, beta, h, nb = 5, 24, 30, 1.5, 0.05, 2
    W = Weights(k)
    Fs, Fccs, Qs, refs = [], [], [], []
    for p in range(nb):
        hc, hb, V = _cluster(d, 2, 40 + 7 * d + p)
        g0 = green_from_H(N, T, hc, 0.0, beta, h)
        bath = green_from_H(N, T, hb, 0.0, beta, h)
        S = OHerm(N, T, d)
        for c in ("mat", "ret", "les", "tv"):
            setattr(S, c, np.einsum("ab,...bc,dc->...ad", V, getattr(bath, c), V.conj()))
        F = _convolve_all(N, T, g0, S, W, beta, h, -1.0)
        Fcc = _convolve_all(N, T, S, g0, W, beta, h, -1.0)
        ref = OHerm(N, T, d)
        vie2.solve_vie2(ref, F, Fcc, g0, beta, h, W)
        Fs.append(F), Fccs.append(Fcc), Qs.append(g0), refs.append(ref)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    dF, dFcc, dQ, G = ng.Herm(g), ng.Herm(g), ng.Herm(g), ng.Herm(g)
    oracle_to_herm(Fs, dF, g)
    oracle_to_herm(Fccs, dFcc, g)
    oracle_to_herm(Qs, dQ, g)
    ctx = ng.Context(k)
    ctx.vie2_mat(g, G, dF, dQ)
    ctx.vie2_start(g, G, dF, dFcc, dQ)
    for n in range(k + 1, N + 1):
        ctx.vie2_timestep(g, n, G, dF, dFcc, dQ)
    torch.cuda.synchronize()
    assert ctx.status_sync() == (ng.NG_OK, 0)
    for kb in range(nb):
        e = _compare(herm_to_oracle(G, g, kb), refs[kb], N)
        assert max(e.values()) < TOL, (kb, e)
    ctx.close()


def _random_herm(rng, N, T, d, scale):
    X = OHerm(N, T, d)
    c = lambda *s: scale * (rng.normal(0, 1, s) + 1j * rng.normal(0, 1, s))
    X.mat[...] = c(T + 1, d, d)
    X.tv[...] = c(N + 1, T + 1, d, d)
    low = np.tril(np.ones((N + 1, N + 1), bool))
    X.ret[low] = c(int(low.sum()), d, d)
    X.les[low.T] = c(int(low.sum()), d, d)
    return X


@pytest.mark.parametrize("tvsrc,bulk", [("fft", "thread"), ("fft", "warp"), ("direct", "thread")])
@pytest.mark.parametrize("d", [1, 2, 4])
def test_vie2_steps_from_random_data(ng, d, tvsrc, bulk):
    """Matsubara, start-up and the steps n = k+1, 2k+1, 2k+2, N from a random history, with F,
    Fcc and Q drawn independently (single steps are linear in their inputs); the left-mixing
    source from the FFT pre-pass with its corrections, or from the direct sums."""
    k, N, T, beta, h, nb = 5, 22, 18, 2.0, 0.06, 2
    rng = np.random.default_rng(900 + d)
    W = Weights(k)
    F = [_random_herm(rng, N, T, d, 0.2) for _ in range(nb)]
    Fcc = [_random_herm(rng, N, T, d, 0.2) for _ in range(nb)]
    Q = [_random_herm(rng, N, T, d, 1.0) for _ in range(nb)]
    Hs = [_random_herm(rng, N, T, d, 0.5) for _ in range(nb)]
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    dF, dFcc, dQ = ng.Herm(g), ng.Herm(g), ng.Herm(g)
    oracle_to_herm(F, dF, g)
    oracle_to_herm(Fcc, dFcc, g)
    oracle_to_herm(Q, dQ, g)
    ctx = ng.Context(k)
    ctx.set_tv_source(ng.NG_TVSRC_AUTO if tvsrc == "fft" else ng.NG_TVSRC_DIRECT)
    ctx.set_bulk_split(ng.NG_BULK_THREAD if bulk == "thread" else ng.NG_BULK_WARP)
    # Matsubara and start-up
    G = ng.Herm(g)
    ctx.vie2_mat(g, G, dF, dQ)
    ctx.vie2_start(g, G, dF, dFcc, dQ)
    torch.cuda.synchronize()
    for kb in range(nb):
        ref = OHerm(N, T, d)
        vie2.vie2_mat(ref, F[kb], Q[kb], beta, W)
        vie2.vie2_start(ref, F[kb], Fcc[kb], Q[kb], beta, h, W)
        e = _compare(herm_to_oracle(G, g, kb), ref, N, upto=k)
        assert max(e.values()) < TOL, ("start", kb, e)
    # single steps from the random history
    for n in (k + 1, 2 * k + 1, 2 * k + 2, N):
        G = ng.Herm(g)
        oracle_to_herm(Hs, G, g, nmax=n - 1)
        ctx.vie2_timestep(g, n, G, dF, dFcc, dQ)
        torch.cuda.synchronize()
        for kb in range(nb):
            ref = Hs[kb].copy()
            vie2.vie2_timestep(n, ref, F[kb], Fcc[kb], Q[kb], beta, h, W)
            got = herm_to_oracle(G, g, kb)
            for name, x, y in (("ret", got.ret[n, :n + 1], ref.ret[n, :n + 1]),
                               ("les", got.les[:n + 1, n], ref.les[:n + 1, n]), ("tv", got.tv[n], ref.tv[n])):
                assert _rel(x, y) < TOL, (n, kb, name, _rel(x, y))
    with pytest.raises(ng.NgError):
        ctx.vie2_timestep(g, N, G, dF, dFcc, dQ, schedule=ng.NG_SERIAL)
    assert ctx.status_sync() == (ng.NG_OK, 0)
    ctx.close()
