"""A time step whose element offsets exceed 2^31: 2048 k-points interleaved innermost with
nt = 1500 (the packed retarded triangle alone spans 2048 * tri(1501) = 2.3e9 elements per
component), one ng_dyson_timestep at n = 1500 from a seeded random history, checked against the
oracle's own step for the first and the last k-point (the largest offsets).  About 75 GB of
device memory."""
import numpy as np
import pytest
import torch

from oracle import dyson
from oracle.contour import Func as OFunc
from oracle.contour import Herm as OHerm
from oracle.weights import Weights

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def _fill(H, seed, scale):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    for t in H.tensors().values():
        v = torch.view_as_real(t)
        for i in range(0, v.shape[0], 1 << 16):     # chunks: bounded temporary memory
            v[i:i + (1 << 16)].normal_(0.0, scale, generator=gen)


def _oracle_herm(ng, H, kb, N, T, upto):
    X = OHerm(N, T, 1)
    X.mat[:, 0, 0] = H.mat[:, 0, 0, kb].cpu().numpy()
    ret = H.ret[:ng.tri(upto + 1), 0, 0, kb].cpu().numpy()
    les = H.les[:ng.tri(upto + 1), 0, 0, kb].cpu().numpy()
    tv = H.tv[:(upto + 1) * (T + 1), 0, 0, kb].cpu().numpy()
    for m in range(upto + 1):
        X.ret[m, :m + 1, 0, 0] = ret[ng.tri(m):ng.tri(m) + m + 1]
        X.les[:m + 1, m, 0, 0] = les[ng.tri(m):ng.tri(m) + m + 1]
        X.tv[m, :, 0, 0] = tv[m * (T + 1):(m + 1) * (T + 1)]
    return X


def test_timestep_with_offsets_beyond_2_31(ng):
    nk, N, T, k, beta, h = 2048, 1500, 16, 5, 3.0, 0.02
    free, _ = torch.cuda.mem_get_info()
    if free < 85e9:
        pytest.skip(f"needs about 75 GB of free device memory, {free / 1e9:.0f} GB free")
    g = ng.Grid(nt=N, ntau=T, nf=1, nbatch=nk, korder=k, h=h, beta=beta)
    assert ng.tri(N + 1) * nk > 2 ** 31
    G = ng.Herm(g, zero=False)
    S = ng.Herm(g, ldk=1, zero=False)       # a local self-energy shared by every k-point
    _fill(G, 1, 0.3)
    _fill(S, 2, 0.05)
    eps = ng.Func(g)
    kk = torch.arange(nk, dtype=torch.float64, device="cuda")
    eps.val[:, 0, 0, :] = (-2.0 * torch.cos(2 * np.pi * kk / nk)).to(torch.complex128)[None, :]
    ctx = ng.Context(k)
    ctx.dyson_timestep(g, N, G, S, eps)
    torch.cuda.synchronize()
    assert ctx.status_sync() == (ng.NG_OK, 0)
    W = Weights(k)
    for kb in (0, nk - 1):
        Go = _oracle_herm(ng, G, kb, N, T, N - 1)
        So = _oracle_herm(ng, S, 0, N, T, N)
        eo = OFunc(N, 1)
        eo.val[:, 0, 0] = eps.val[:, 0, 0, kb].cpu().numpy()
        dyson.dyson_timestep(N, Go, So, eo, 0.0, beta, h, W)
        got = _oracle_herm(ng, G, kb, N, T, N)
        for name, x, y in (("ret", got.ret[N, :N + 1], Go.ret[N, :N + 1]), ("les", got.les[:N + 1, N], Go.les[:N + 1, N]),
                           ("tv", got.tv[N], Go.tv[N])):
            err = np.abs(x - y).max() / np.abs(y).max()
            assert err < TOL, (kb, name, err)
    del G, S
    torch.cuda.empty_cache()
