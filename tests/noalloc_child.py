"""Child process of tests/test_zz_no_alloc.py (a fresh CUDA context per run).

Usage: python -m tests.noalloc_child {noalloc_first|context_first}
Runs, in the given order, one allocation-free start-up and the small second-Born adjoint
gradient of a 2x2 lattice (nt = 18), then prints the gradient as one JSON line.  The
gradient must not depend on which libng call came first in the process.
"""
import json
import sys

import numpy as np
import torch


def _noalloc_once(ng):
    g = ng.Grid(nt=12, ntau=12, nf=1, nbatch=2, korder=5, h=0.05, beta=2.0)
    G, S, eps = ng.Herm(g), ng.Herm(g), ng.Func(g)
    eps.val[:] = 0.3
    st = ng.dyson_start_noalloc(g, G, S, eps)
    torch.cuda.synchronize()
    assert st == ng.NG_OK, st


def _gradient(ng):
    from paper_1911_01211_gb300.adjoint import densities
    L, nt, ntau, beta, h, U = 2, 18, 12, 2.0, 0.1, 1.0
    rng = np.random.default_rng(1911)
    A = np.zeros(nt + 2)
    A[2:] = 0.4 * rng.standard_normal(nt)
    kx, ky = np.meshgrid(2 * np.pi * np.arange(L) / L, 2 * np.pi * np.arange(L) / L, indexing="ij")
    kx = torch.as_tensor(kx.ravel(), device="cuda")
    ky = torch.as_tensor(ky.ravel(), device="cuda")
    g = ng.Grid(nt=nt, ntau=ntau, nf=1, nbatch=L * L, korder=5, h=h, beta=beta)
    ctx = ng.Context(5)
    Ut = torch.full((nt + 2,), U, dtype=torch.float64, device="cuda")
    At = torch.tensor(A, dtype=torch.float64, device="cuda", requires_grad=True)
    e0 = -2.0 * torch.cos(kx[None, :] - At[:, None]) - 2.0 * torch.cos(ky[None, :])
    rho = densities(e0, ctx, g, Ut)
    loss = (rho[nt].real * e0[nt + 1]).mean()
    loss.backward()
    out = At.grad.cpu().numpy()
    ctx.close()
    return out


def main(order):
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    if order == "noalloc_first":
        _noalloc_once(ng)
        grad = _gradient(ng)
    elif order == "context_first":
        grad = _gradient(ng)
        _noalloc_once(ng)
    else:
        raise SystemExit(f"unknown order {order}")
    print(json.dumps({"order": order, "grad": grad.tolist()}))


if __name__ == "__main__":
    main(sys.argv[1])
