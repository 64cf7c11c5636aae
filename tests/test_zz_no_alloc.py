"""Allocation-free start-up entry point (ng_dyson_start_noalloc).

Some callers cannot allocate device memory at the point where they need the start-up
slices: their own caching allocator owns all free memory, or cudaFree's implicit device
synchronisation would stall a latency-critical loop, or their host forbids libraries from
managing device memory.  ng_dyson_start_noalloc serves them with a fixed static device array
instead of context-owned workspace.  These tests call it through the C ABI and check that it
reproduces ng_dyson_start (the existing entry point) within the parity tolerance, on two
calls in a row with different problem sizes, and that an oversized batch is refused before
anything is launched.  When this file runs alone the first call is the first libng call of
the process; the last test makes sure of that case whatever ran before, by running the
allocation-free start-up first in a child process with its own CUDA context and checking
that the contexts created after it still compute the same adjoint gradient.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from tests.layout import funcs_to_device, herm_to_oracle, oracle_to_herm

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _inputs(ng, d, nb, seed):
    """Sigma, eps and G^M of nb embedded problems, computed by the CPU oracle."""
    from tests.test_gpu_parity import _oracle_problem_set
    k, N, T, beta, h = 5, 14, 20, 3.0, 0.05
    W, Gs, Ss, epss = _oracle_problem_set(d, nb, N, T, beta, h, k, seed=seed)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    S, eps, Gmat_only = ng.Herm(g), ng.Func(g), ng.Herm(g)
    oracle_to_herm(Ss, S, g)
    funcs_to_device(epss, eps)
    oracle_to_herm(Gs, Gmat_only, g, nmax=-1)      # only the Matsubara slice is filled
    return g, S, eps, Gmat_only


def _fresh_copy(ng, g, src):
    G = ng.Herm(g)
    G.mat.copy_(src.mat)
    return G


def _max_rel(ng, g, A, B, k):
    worst = 0.0
    for kb in range(g.nbatch):
        a, b = herm_to_oracle(A, g, kb), herm_to_oracle(B, g, kb)
        for x, y in ((a.ret[:k + 1, :k + 1], b.ret[:k + 1, :k + 1]), (a.les[:k + 1, :k + 1], b.les[:k + 1, :k + 1]),
                     (a.tv[:k + 1], b.tv[:k + 1])):
            worst = max(worst, float(np.abs(x - y).max() / np.abs(y).max()))
    return worst


def test_noalloc_start_matches_dyson_start_twice():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    cases = [(1, 3, 41), (2, 2, 43), (4, 1, 47)]   # (nf, nbatch, seed): calls in a row, different sizes
    prepared = [_inputs(ng, d, nb, seed) for d, nb, seed in cases]
    results = []
    for g, S, eps, G0 in prepared:    # allocation-free calls first (possibly the first libng calls)
        G = _fresh_copy(ng, g, G0)
        st = ng.dyson_start_noalloc(g, G, S, eps)
        assert st == ng.NG_OK, st
        torch.cuda.synchronize()
        results.append(G)
    ctx = ng.Context(5)
    for (g, S, eps, G0), Gna in zip(prepared, results):
        Gref = _fresh_copy(ng, g, G0)
        ctx.dyson_start(g, Gref, S, eps)
        torch.cuda.synchronize()
        assert ctx.status_sync() == (ng.NG_OK, 0)
        assert bool(torch.isfinite(torch.view_as_real(Gna.tv)).all())
        assert _max_rel(ng, g, Gna, Gref, g.korder) < TOL
    ctx.close()


def test_noalloc_start_rejects_oversized_batch():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    # nf = 2, k = 5: 256 + 16 * 2000 * (100 + 20) bytes > 2 MiB
    g = ng.Grid(nt=12, ntau=12, nf=2, nbatch=2000, korder=5, h=0.05, beta=2.0)
    G, S, eps = ng.Herm(g), ng.Herm(g), ng.Func(g)
    assert ng.dyson_start_noalloc(g, G, S, eps) == ng.NG_ESCRATCH
    torch.cuda.synchronize()
    assert float(G.tv.abs().max()) == 0.0      # nothing was launched


def _child_gradient(order):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "tests.noalloc_child", order], cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("{")][-1]
    return np.array(json.loads(line)["grad"])


def test_noalloc_first_call_leaves_later_contexts_intact():
    """The one-time set-up of a first allocation-free call loads the integration weights for the
    whole library: an adjoint gradient computed after it in the same process equals the one of
    a process that created its context first."""
    g_first = _child_gradient("noalloc_first")
    g_ref = _child_gradient("context_first")
    scale = np.abs(g_ref).max()
    assert scale > 1e-6
    assert np.abs(g_first - g_ref).max() <= 1e-13 * scale, (g_first, g_ref)
