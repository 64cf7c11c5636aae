"""Double-float time steps (NG_DF64) against the FP64 oracle at the FP64 parity bar (1e-10
relative per component)."""
import numpy as np
import pytest
import torch

from oracle import drivers, dyson
from oracle.contour import Func as OFunc
from oracle.weights import Weights
from paper_1911_01211_gb300 import workloads as wl
from tests.layout import funcs_to_device, herm_to_oracle, oracle_to_herm
from tests.test_gpu_parity import _oracle_problem_set, _ofunc, relerr

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


@pytest.mark.parametrize("d", [1, 2])
def test_df64_timestep_from_oracle_history(ng, d):
    k, N, T, beta, h, nb = 5, 26, 18, 2.5, 0.06, 3
    W, Gs, Ss, epss = _oracle_problem_set(d, nb, N, T, beta, h, k, seed=51 + d)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    ctx = ng.Context(k)
    G, S, eps = ng.Herm(g), ng.Herm(g), ng.Func(g)
    oracle_to_herm(Ss, S, g)
    funcs_to_device(epss, eps)
    for n in (k + 1, 2 * k, 2 * k + 1, N):
        oracle_to_herm(Gs, G, g, nmax=n - 1)
        ctx.precision_reset()
        ctx.dyson_timestep(g, n, G, S, eps, precision=ng.NG_DF64)
        torch.cuda.synchronize()
        assert ctx.status_sync() == (ng.NG_OK, 0)
        for kb in range(nb):
            ref = Gs[kb].copy()
            dyson.dyson_timestep(n, ref, Ss[kb], epss[kb], 0.0, beta, h, W)
            got = herm_to_oracle(G, g, kb)
            for x, y in ((got.ret[n, :n + 1], ref.ret[n, :n + 1]), (got.les[:n + 1, n], ref.les[:n + 1, n]),
                         (got.tv[n], ref.tv[n])):
                assert np.abs(x - y).max() / np.abs(y).max() < TOL, (n, kb)


def test_df64_2b_chain_against_oracle(ng):
    w = wl.chain_kspace(nk=6, nt=40, ntau=30, beta=4.0, h=0.05)
    g = ng.Grid(nt=w.nt, ntau=w.ntau, nf=1, nbatch=w.nbatch, korder=5, h=w.h, beta=w.beta)
    ctx = ng.Context(5)
    G = ng.Herm(g)
    L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    ctx.run_2b(g, G, L, S, e0, mf, U, corrector=w.corrector, precision=ng.NG_DF64)
    torch.cuda.synchronize()
    assert ctx.status_sync() == (ng.NG_OK, 0)
    Uo = OFunc(w.nt, 1)
    Uo.val[:, 0, 0] = w.U
    st = drivers.run_2b([_ofunc(w.eps0, kb) for kb in range(w.nbatch)], Uo, w.nt, w.ntau, w.beta, w.h,
                        Weights(5), corrector=w.corrector)
    for kb in range(w.nbatch):
        e = relerr(herm_to_oracle(G, g, kb), st.G[kb])
        assert max(e.values()) < TOL, (kb, e)
