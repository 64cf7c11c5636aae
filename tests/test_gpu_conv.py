"""ng_convolution_timestep against the oracle's convolution_timestep (Eqs. cm1-cles3) on seeded
random contour data: every slice -1..nt, so that the start-up quadratures (n <= k), the
boundary-weight pieces (m <= k, m >= ntau - k) and the Gregory bulk are all covered, with a
hermitian-conjugate partner that is not the function itself, per-problem and shared operands,
and a matrix-valued time-dependent f."""
import numpy as np
import pytest
import torch

from oracle import conv
from oracle.contour import Func as OFunc
from oracle.contour import Herm as OHerm
from oracle.weights import Weights
from tests.layout import herm_to_oracle, oracle_to_herm

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def _random_herm(rng, N, T, d):
    """Random values on the stored triangles (ret lower, les upper, tv, mat)."""
    X = OHerm(N, T, d)
    c = lambda *s: rng.normal(0, 1, s) + 1j * rng.normal(0, 1, s)
    X.mat[...] = c(T + 1, d, d)
    X.tv[...] = c(N + 1, T + 1, d, d)
    low = np.tril(np.ones((N + 1, N + 1), bool))
    X.ret[low] = c(int(low.sum()), d, d)
    X.les[low.T] = c(int(low.sum()), d, d)
    return X


def _random_func(rng, N, d):
    f = OFunc(N, d)
    f.val[...] = rng.normal(0, 1, (N + 2, d, d)) + 1j * rng.normal(0, 1, (N + 2, d, d))
    return f


def _to_dev(ng, g, objs, ldk):
    H = ng.Herm(g, ldk=ldk)
    oracle_to_herm(objs, H, g)
    return H


@pytest.mark.parametrize("d,nb,with_f", [(1, 3, True), (2, 2, True), (2, 1, False), (4, 2, True), (8, 1, True)])
def test_convolution_against_oracle(ng, d, nb, with_f):
    N, T, beta, h, k = 16, 20, 2.5, 0.07, 5
    rng = np.random.default_rng(1000 + 10 * d + nb)
    W = Weights(k)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    A = [_random_herm(rng, N, T, d) for _ in range(nb)]
    Acc = [_random_herm(rng, N, T, d) for _ in range(nb)]
    Bs = _random_herm(rng, N, T, d)          # B and its partner shared by the batch (ldk = 1)
    Bccs = _random_herm(rng, N, T, d)
    fs = [_random_func(rng, N, d) for _ in range(nb)] if with_f else None
    dA, dAcc = _to_dev(ng, g, A, nb), _to_dev(ng, g, Acc, nb)
    dB, dBcc = _to_dev(ng, g, [Bs], 1), _to_dev(ng, g, [Bccs], 1)
    df = None
    if with_f:
        df = ng.Func(g)
        df.val.copy_(torch.from_numpy(np.ascontiguousarray(np.stack([f.val for f in fs], axis=-1))))
    C = ng.Herm(g)
    ctx = ng.Context(k)
    for n in range(-1, N + 1):
        ctx.convolution_timestep(g, n, C, dA, dAcc, df, dB, dBcc)
    torch.cuda.synchronize()
    assert ctx.status_sync() == (ng.NG_OK, 0)
    for kb in range(nb):
        ref = OHerm(N, T, d)
        f = fs[kb] if with_f else None
        for n in range(-1, N + 1):
            conv.convolution_timestep(n, ref, A[kb], Acc[kb], f, Bs, Bccs, W, beta, h)
        got = herm_to_oracle(C, g, kb)
        low = np.tril(np.ones((N + 1, N + 1), bool))
        for name, a, b in (("mat", got.mat, ref.mat), ("ret", got.ret[low], ref.ret[low]),
                           ("les", got.les[low.T], ref.les[low.T]), ("tv", got.tv, ref.tv)):
            err = np.abs(a - b).max() / np.abs(b).max()
            assert err < TOL, (d, kb, name, err)
    ctx.close()


def test_convolution_shared_output(ng):
    """C.ldk = 1 with every operand shared: one problem's result, equal to the oracle."""
    N, T, beta, h, k, d = 13, 14, 1.5, 0.1, 5, 2
    rng = np.random.default_rng(77)
    W = Weights(k)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=4, korder=k, h=h, beta=beta)
    A, B = _random_herm(rng, N, T, d), _random_herm(rng, N, T, d)
    dA, dB = _to_dev(ng, g, [A], 1), _to_dev(ng, g, [B], 1)
    C = ng.Herm(g, ldk=1)
    ctx = ng.Context(k)
    for n in range(-1, N + 1):
        ctx.convolution_timestep(g, n, C, dA, dA, None, dB, dB)
    torch.cuda.synchronize()
    ref = OHerm(N, T, d)
    for n in range(-1, N + 1):
        conv.convolution_timestep(n, ref, A, A, None, B, B, W, beta, h)
    got = herm_to_oracle(C, g, 0)
    low = np.tril(np.ones((N + 1, N + 1), bool))
    for a, b in ((got.mat, ref.mat), (got.ret[low], ref.ret[low]), (got.les[low.T], ref.les[low.T]),
                 (got.tv, ref.tv)):
        assert np.abs(a - b).max() / np.abs(b).max() < TOL
    with pytest.raises(ng.NgError):          # shared output with a per-problem operand
        ctx.convolution_timestep(g, 3, C, _to_dev(ng, g, [A] * 4, 4), dA, None, dB, dB)
    ctx.close()
