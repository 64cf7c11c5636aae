"""ng_run_2b_host (the second-Born driver with host-memory inputs and outputs) against
ng_run_2b with device inputs: bitwise the same contour functions, and the host copies of
Gloc^<(t_n, t_n) equal to the device values; plus the FP64 throughput probe."""
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


def _setup(ng, w):
    g = ng.Grid(nt=w.nt, ntau=w.ntau, nf=w.nf, nbatch=w.nbatch, korder=w.korder, h=w.h, beta=w.beta)
    G = ng.Herm(g)
    L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0, mf = ng.Func(g), ng.Func(g)
    U = ng.Func(g, scalar=True)
    return g, G, L, S, e0, mf, U


def test_host_buffer_driver_equals_device_driver(ng):
    w = wl.chain_kspace(nk=40, nt=30, ntau=20, beta=4.0, h=0.05)
    ctx = ng.Context(w.korder)
    g, G1, L1, S1, e01, mf1, U1 = _setup(ng, w)
    e01.val.copy_(torch.from_numpy(w.eps0))
    U1.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    it1 = ctx.run_2b(g, G1, L1, S1, e01, mf1, U1, corrector=w.corrector)
    g, G2, L2, S2, e02, mf2, U2 = _setup(ng, w)
    eps_host = torch.from_numpy(np.ascontiguousarray(w.eps0)).pin_memory()
    U_host = torch.from_numpy(w.U.astype(np.complex128)).pin_memory()
    gd = torch.zeros((w.nt + 1, 1, 1), dtype=torch.complex128).pin_memory()
    # in two calls, as a caller that times a window would
    nmid = 17
    it2 = ctx.run_2b_host(g, G2, L2, S2, e02, mf2, U2, eps_host, U_host, gd, corrector=w.corrector, n_to=nmid)
    ctx.run_2b_host(g, G2, L2, S2, e02, mf2, U2, eps_host, U_host, gd, corrector=w.corrector, n_from=nmid + 1,
                    do_setup=False)
    torch.cuda.synchronize()
    assert it1 == it2
    for name in ("mat", "ret", "les", "tv"):
        assert torch.equal(getattr(G1, name), getattr(G2, name)), name
        assert torch.equal(getattr(S1, name), getattr(S2, name)), name
    diag = torch.tensor([ng.tri(n) + n for n in range(w.nt + 1)], device="cuda")
    # Gloc slices 0..k are those of the bootstrapping; later ones as the last pass reduced them
    assert torch.equal(gd.cuda(), L2.les[diag, :, :, 0])
    assert torch.equal(e02.val, e01.val)


def test_fp64_probe(ng):
    r = ng.fp64_probe()
    assert r["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    # plausible FP64 rates of a current data-centre GPU (tens of GFLOP/s .. 100 TFLOP/s)
    assert 0.05 < r["dfma_tflops"] < 100 and 0.05 < r["dmma_tflops"] < 100, r
