"""GPU parity: every libng entry point against the FP64 CPU oracle on the same seeded
inputs, element by element.  Tolerance: 1e-10 relative to the component's maximum
(max |gpu - oracle| / max |oracle| per component and problem)."""
import numpy as np
import pytest
import torch

from oracle import bubble, drivers, dyson, extrap
from oracle.contour import Func as OFunc
from oracle.contour import Herm as OHerm
from oracle.freegf import green_from_H
from oracle.weights import Weights
from paper_1911_01211_gb300 import workloads as wl
from tests.layout import device_to_funcs, funcs_to_device, herm_to_oracle, oracle_to_herm, tri

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def relerr(a, b, comps=("mat", "ret", "les", "tv"), nmax=None):
    """Per-component max |a-b| / max |b| over the stored triangles up to slice nmax."""
    out = {}
    N = b.nt if nmax is None else nmax
    for c in comps:
        x, y = getattr(a, c), getattr(b, c)
        if c == "ret":
            m = np.tril(np.ones((b.nt + 1, b.nt + 1), bool))
            m[N + 1:] = False
            x, y = x[m], y[m]
        elif c == "les":
            m = np.triu(np.ones((b.nt + 1, b.nt + 1), bool))
            m[:, N + 1:] = False
            x, y = x[m], y[m]
        elif c == "tv":
            x, y = x[:N + 1], y[:N + 1]
        den = np.abs(y).max()
        out[c] = float(np.abs(x - y).max() / (den if den > 0 else 1.0))
    return out


def assert_close(a, b, tol=TOL, **kw):
    e = relerr(a, b, **kw)
    assert max(e.values()) < tol, e


def _ofunc(arr, kb):
    f = OFunc(arr.shape[0] - 2, arr.shape[1])
    f.val[...] = arr[..., kb]
    return f


def _grid(ng, w, nbatch=None):
    return ng.Grid(nt=w.nt, ntau=w.ntau, nf=w.nf, nbatch=w.nbatch if nbatch is None else nbatch,
                   korder=w.korder, h=w.h, beta=w.beta, mu=w.mu)


def _status_ok(ctx, ng):
    torch.cuda.synchronize()
    st, flags = ctx.status_sync()
    assert st == ng.NG_OK and flags == 0, (st, flags)


# --------------------------------------------------------------------------------------
def test_free_gf(ng):
    rng = np.random.default_rng(191101211)
    for d in (1, 2):
        nb = 3
        eps = np.stack([wl.random_hermitian(rng, d) for _ in range(nb)])
        g = ng.Grid(nt=14, ntau=16, nf=d, nbatch=nb, korder=5, h=0.07, beta=3.0, mu=0.1)
        ctx = ng.Context(5)
        G = ng.Herm(g)
        ctx.green_from_H_const(g, G, eps, scale=0.7)
        _status_ok(ctx, ng)
        for kb in range(nb):
            ref = green_from_H(g.nt, g.ntau, eps[kb], 0.1, g.beta, g.h)
            for c in ("mat", "ret", "les", "tv"):
                setattr(ref, c, getattr(ref, c) * 0.7)
            assert_close(herm_to_oracle(G, g, kb), ref, tol=1e-13)


def test_fixed_sigma_embedded_level(ng):
    """Embedded level (embedded_level workload at reduced size) through ng_solve_fixed."""
    from tests.oracle_cases import embedded_level
    w = wl.embedded_level(nt=40, ntau=40, beta=2.0, h=0.05)
    g = _grid(ng, w)
    ctx = ng.Context(5)
    G, S = ng.Herm(g), ng.Herm(g)
    ctx.green_from_H_const(g, S, np.array([w.extra["eb"]]), scale=w.extra["V"] ** 2)
    eps = ng.Func(g, values=torch.from_numpy(w.eps0))
    ctx.solve_fixed(g, G, S, eps)
    _status_ok(ctx, ng)
    Go, _, _ = embedded_level(w.nt, w.ntau, w.beta, w.h)
    assert_close(herm_to_oracle(G, g, 0), Go)


def _oracle_problem_set(d, nb, N, T, beta, h, k, seed):
    """nb embedded problems with d orbitals, each with its own bath (per-problem Sigma)."""
    rng = np.random.default_rng(seed)
    W = Weights(k)
    Gs, Ss, epss = [], [], []
    for _ in range(nb):
        hs = wl.random_hermitian(rng, d)
        hb = wl.random_hermitian(rng, 2)
        V = rng.normal(0, 0.4, (d, 2))
        full = np.block([[hs, V], [V.T, hb]])
        bath = green_from_H(N, T, hb, 0.0, beta, h)
        S = OHerm(N, T, d)
        for c in ("mat", "ret", "les", "tv"):
            setattr(S, c, np.einsum("ab,...bc,dc->...ad", V, getattr(bath, c), V))
        eps = OFunc(N, d)
        eps.val[:] = hs
        G = OHerm(N, T, d)
        drivers.solve_fixed_sigma(G, S, eps, 0.0, beta, h, W)
        Gs.append(G), Ss.append(S), epss.append(eps)
    return W, Gs, Ss, epss


_STEP_CASES = [(d, "mixed", "auto", "thread") for d in (1, 2, 4)] + [(d, "mixed", "auto", "warp") for d in (1, 2)] + \
    [(d, "mixed", "direct", b) for d in (1, 2) for b in ("thread", "warp")] + [(d, "serial", "auto", "auto") for d in (1, 2)]


@pytest.mark.parametrize("d,schedule,tvsrc,bulk", _STEP_CASES)
def test_timestep_from_oracle_history(ng, d, schedule, tvsrc, bulk):
    """ng_dyson_timestep on the oracle's history reproduces the oracle's step in the same
    schedule for n in {k+1, 2k, 2k+1, 2k+2, N} (all branches of the mixed schedule), with
    per-problem Sigma, with the left-mixing source by FFT (auto) and by the direct sums, with
    one thread or one warp per bulk item (nf = 4: the element-wise form)."""
    k, N, T, beta, h, nb = 5, 26, 18, 2.5, 0.06, 3
    W, Gs, Ss, epss = _oracle_problem_set(d, nb, N, T, beta, h, k, seed=11 + d)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    ctx = ng.Context(k)
    ctx.set_tv_source(ng.NG_TVSRC_DIRECT if tvsrc == "direct" else ng.NG_TVSRC_AUTO)
    ctx.set_bulk_split({"auto": ng.NG_BULK_AUTO, "thread": ng.NG_BULK_THREAD, "warp": ng.NG_BULK_WARP}[bulk])
    G, S, eps = ng.Herm(g), ng.Herm(g), ng.Func(g)
    oracle_to_herm(Ss, S, g)
    funcs_to_device(epss, eps)
    for n in (k + 1, 2 * k, 2 * k + 1, 2 * k + 2, N):
        oracle_to_herm(Gs, G, g, nmax=n - 1)
        ctx.dyson_timestep(g, n, G, S, eps, schedule=ng.NG_SERIAL if schedule == "serial" else ng.NG_MIXED)
        _status_ok(ctx, ng)
        for kb in range(nb):
            ref = Gs[kb].copy()
            # the oracle's own step n from the same history
            dyson.dyson_timestep(n, ref, Ss[kb], epss[kb], 0.0, beta, h, W, schedule=schedule)
            got = herm_to_oracle(G, g, kb)
            e = {}
            for c, x, y in (("ret", got.ret[n, :n + 1], ref.ret[n, :n + 1]),
                            ("les", got.les[:n + 1, n], ref.les[:n + 1, n]),
                            ("tv", got.tv[n], ref.tv[n])):
                e[c] = np.abs(x - y).max() / np.abs(y).max()
            assert max(e.values()) < TOL, (n, kb, e)


def _random_history(rng, N, T, d, scale=0.3):
    X = OHerm(N, T, d)
    c = lambda *sh: scale * (rng.normal(0, 1, sh) + 1j * rng.normal(0, 1, sh))
    X.mat[...] = c(T + 1, d, d)
    X.tv[...] = c(N + 1, T + 1, d, d)
    low = np.tril(np.ones((N + 1, N + 1), bool))
    X.ret[low] = c(int(low.sum()), d, d)
    X.les[low.T] = c(int(low.sum()), d, d)
    return X


@pytest.mark.parametrize("d,T", [(1, 500), (1, 1023), (2, 500)])
def test_fft_source_at_large_ntau(ng, d, T):
    """The FFT pre-pass at transform lengths 1024 and 2048 (one step from a seeded random
    history, two problems with their own Sigma): both source evaluations against the oracle,
    and against each other at rounding level."""
    k, N, beta, h, nb = 5, 20, 4.0, 0.05, 2
    rng = np.random.default_rng(500 + d + T)
    W = Weights(k)
    Gs = [_random_history(rng, N, T, d) for _ in range(nb)]
    Ss = [_random_history(rng, N, T, d, 0.05) for _ in range(nb)]
    epss = []
    for _ in range(nb):
        e = OFunc(N, d)
        e.val[:] = wl.random_hermitian(rng, d)
        epss.append(e)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    ctx = ng.Context(k)
    S, eps = ng.Herm(g), ng.Func(g)
    oracle_to_herm(Ss, S, g)
    funcs_to_device(epss, eps)
    out = {}
    for mode in (ng.NG_TVSRC_AUTO, ng.NG_TVSRC_DIRECT):
        ctx.set_tv_source(mode)
        for n in (k + 1, 2 * k + 2, N):
            G = ng.Herm(g)
            oracle_to_herm(Gs, G, g, nmax=n - 1)
            ctx.dyson_timestep(g, n, G, S, eps)
            _status_ok(ctx, ng)
            out[mode, n] = [herm_to_oracle(G, g, kb).tv[n].copy() for kb in range(nb)]
            for kb in range(nb):
                ref = Gs[kb].copy()
                dyson.dyson_timestep(n, ref, Ss[kb], epss[kb], 0.0, beta, h, W)
                x, y = out[mode, n][kb], ref.tv[n]
                assert np.abs(x - y).max() / np.abs(y).max() < TOL, (mode, n, kb)
    for n in (k + 1, 2 * k + 2, N):
        for kb in range(nb):
            a, b = out[ng.NG_TVSRC_AUTO, n][kb], out[ng.NG_TVSRC_DIRECT, n][kb]
            assert np.abs(a - b).max() / np.abs(b).max() < 1e-13


def test_serial_schedule_propagation(ng):
    """A whole fixed-Sigma propagation with every step in the serial schedule (d = 2, two
    problems) against the oracle's serial solve, and the serial-mixed difference at
    discretisation level."""
    from tests.oracle_cases import embedded_cluster
    k, N, T, beta, h = 5, 24, 16, 1.0, 0.05
    Gos, Sos, epss = [], [], []
    for seed in (3, 4):
        Go, _, So, eo = embedded_cluster(2, 2, N, T, beta, h, seed=seed, schedule="serial")
        Gos.append(Go), Sos.append(So), epss.append(eo)
    g = ng.Grid(nt=N, ntau=T, nf=2, nbatch=2, korder=k, h=h, beta=beta)
    ctx = ng.Context(k)
    G, S, eps = ng.Herm(g), ng.Herm(g), ng.Func(g)
    oracle_to_herm(Sos, S, g)
    funcs_to_device(epss, eps)
    ctx.dyson_mat(g, G, S, eps)
    ctx.dyson_start(g, G, S, eps)
    for n in range(k + 1, N + 1):
        ctx.dyson_timestep(g, n, G, S, eps, schedule=ng.NG_SERIAL)
    _status_ok(ctx, ng)
    Gm = ng.Herm(g)
    ctx.solve_fixed(g, Gm, S, eps)
    _status_ok(ctx, ng)
    for kb in range(2):
        assert_close(herm_to_oracle(G, g, kb), Gos[kb])
        diff = relerr(herm_to_oracle(Gm, g, kb), Gos[kb])
        assert 0 < max(diff.values()) < 1e-4, diff


@pytest.mark.parametrize("d", [1, 2])
def test_mat_and_start(ng, d):
    k, N, T, beta, h, nb = 5, 14, 22, 3.0, 0.05, 2
    W, Gs, Ss, epss = _oracle_problem_set(d, nb, N, T, beta, h, k, seed=5 + d)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    ctx = ng.Context(k)
    G, S, eps = ng.Herm(g), ng.Herm(g), ng.Func(g)
    oracle_to_herm(Ss, S, g)
    funcs_to_device(epss, eps)
    ctx.dyson_mat(g, G, S, eps)
    ctx.dyson_start(g, G, S, eps)
    _status_ok(ctx, ng)
    for kb in range(nb):
        assert_close(herm_to_oracle(G, g, kb), Gs[kb], nmax=k)


def test_slice_operations(ng):
    """k-reduction, second-Born, Hartree and extrapolation slices against the oracle."""
    k, N, T, beta, h, nb, d = 5, 16, 12, 2.0, 0.05, 3, 2
    W, Gs, Ss, epss = _oracle_problem_set(d, nb, N, T, beta, h, k, seed=3)
    g = ng.Grid(nt=N, ntau=T, nf=d, nbatch=nb, korder=k, h=h, beta=beta)
    ctx = ng.Context(k)
    G = ng.Herm(g)
    oracle_to_herm(Gs, G, g)
    L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    U = ng.Func(g, scalar=True)
    Uo = OFunc(N, 1)
    Uo.val[:, 0, 0] = 1.3
    Uo.set(-1, np.array([[0.7]]))
    U.val[:, 0, 0, 0] = torch.from_numpy(Uo.val[:, 0, 0])
    Lo, So = OHerm(N, T, d), OHerm(N, T, d)
    for n in range(-1, N + 1):
        ctx.kreduce_timestep(g, n, L, G)
        ctx.sigma2b_timestep(g, n, S, L, U)
        bubble.kreduce(n, Gs, Lo)
        bubble.sigma_2b(n, Lo, Uo, So)
    _status_ok(ctx, ng)
    assert_close(herm_to_oracle(L, g, 0), Lo, tol=1e-14)
    assert_close(herm_to_oracle(S, g, 0), So, tol=1e-13)
    # Hartree
    e0 = ng.Func(g)
    funcs_to_device(epss, e0)
    mf = ng.Func(g)
    for n in (-1, 0, 7):
        ctx.hartree_timestep(g, n, mf, e0, L, U, 0.5)
    torch.cuda.synchronize()
    mfo = device_to_funcs(mf, g)
    for n in (-1, 0, 7):
        rho = bubble.density_matrix(n, Lo)
        for kb in range(nb):
            assert np.abs(mfo[kb](n) - bubble.hartree(n, rho, epss[kb](n), Uo, 0.5)).max() < 1e-13
    # extrapolation of slice 11 from slices 6..10
    H = ng.Herm(g)
    oracle_to_herm(Gs, H, g, nmax=10)
    ctx.extrapolate_timestep(g, 10, H)
    torch.cuda.synchronize()
    for kb in range(nb):
        ref = Gs[kb].copy()
        extrap.extrapolate_timestep(10, ref, W)
        got = herm_to_oracle(H, g, kb)
        assert np.abs(got.ret[11, :12] - ref.ret[11, :12]).max() < 1e-12
        assert np.abs(got.les[:12, 11] - ref.les[:12, 11]).max() < 1e-12
        assert np.abs(got.tv[11] - ref.tv[11]).max() < 1e-12


def _run_2b_both(ng, w, nmax=None, bulk=None):
    g = _grid(ng, w)
    ctx = ng.Context(w.korder)
    if bulk is not None:
        ctx.set_bulk_split(bulk)
    G = ng.Herm(g)
    L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    nto = w.nt if nmax is None else nmax
    iters = ctx.run_2b(g, G, L, S, e0, mf, U, corrector=w.corrector, n_to=nto)
    _status_ok(ctx, ng)
    W = Weights(w.korder)
    eps0 = [_ofunc(w.eps0, kb) for kb in range(w.nbatch)]
    Uo = OFunc(w.nt, 1)
    Uo.val[:, 0, 0] = w.U
    st = drivers.run_2b(eps0, Uo, w.nt, w.ntau, w.beta, w.h, W, corrector=w.corrector, nmax=nto)
    return g, G, st, iters


def test_2b_kspace_chain_small(ng):
    """chain_kspace workload on a small grid: nk = 6, nt = 24, ntau = 20, all k compared."""
    w = wl.chain_kspace(nk=6, nt=24, ntau=20, beta=4.0, h=0.05)
    g, G, st, iters = _run_2b_both(ng, w)
    for kb in range(w.nbatch):
        assert_close(herm_to_oracle(G, g, kb), st.G[kb])


def test_observables_against_oracle(ng):
    """ng_observables (N, E_kin, E_mf, E_corr, E_tot) after a small self-consistent chain run,
    against the oracle's density matrix and Galitskii-Migdal correlation energy."""
    from oracle import bubble, observables
    w = wl.chain_kspace(nk=4, nt=20, ntau=20, beta=4.0, h=0.05)
    g = _grid(ng, w)
    ctx = ng.Context(w.korder)
    G = ng.Herm(g)
    L, S = ng.Herm(g, ldk=1), ng.Herm(g, ldk=1)
    e0 = ng.Func(g, values=torch.from_numpy(w.eps0))
    mf = ng.Func(g)
    U = ng.Func(g, scalar=True)
    U.val[:, 0, 0, 0] = torch.from_numpy(w.U.astype(complex))
    ctx.run_2b(g, G, L, S, e0, mf, U, corrector=w.corrector)
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    W = Weights(w.korder)
    Gk = [herm_to_oracle(G, g, kb) for kb in range(w.nbatch)]
    So = herm_to_oracle(S, g, 0)
    mfo = device_to_funcs(mf, g)
    for n in (0, 3, w.korder + 1, w.nt):
        ctx.observables(g, n, G, S, e0, mf, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = np.zeros(5)
        for kb in range(w.nbatch):
            rho = observables.density_matrix(n, Gk[kb])
            e0k = w.eps0[n + 1, :, :, kb]
            ref[0] += np.real(np.trace(rho))
            ref[1] += np.real(np.trace(rho @ e0k))
            ref[2] += 0.5 * np.real(np.trace(rho @ (mfo[kb](n) - e0k)))
            ref[3] += observables.correlation_energy(n, Gk[kb], So, W, w.beta, w.h)
        ref /= w.nbatch
        ref[4] = ref[1] + ref[2] + ref[3]
        assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max()), (n, got, ref)
    _status_ok(ctx, ng)


@pytest.mark.parametrize("bulk", ["thread", "warp"])
def test_2b_hubbard_dimer_small(ng, bulk):
    """hubbard_dimer workload on a small grid (nf = 2, quench U: 1 -> 2), one thread or one warp
    per bulk item."""
    w = wl.hubbard_dimer(nt=30, ntau=24, beta=5.0, h=0.05)
    g, G, st, iters = _run_2b_both(ng, w, bulk=ng.NG_BULK_THREAD if bulk == "thread" else ng.NG_BULK_WARP)
    assert_close(herm_to_oracle(G, g, 0), st.G[0])


def test_embedded_level_full_size(ng):
    """embedded_level workload at its full size (nt = ntau = 200, beta = 10, h = 0.025)."""
    from tests.oracle_cases import embedded_level
    w = wl.embedded_level()
    g = _grid(ng, w)
    ctx = ng.Context(5)
    G, S = ng.Herm(g), ng.Herm(g)
    ctx.green_from_H_const(g, S, np.array([w.extra["eb"]]), scale=w.extra["V"] ** 2)
    eps = ng.Func(g, values=torch.from_numpy(w.eps0))
    ctx.solve_fixed(g, G, S, eps)
    _status_ok(ctx, ng)
    Go, ex, _ = embedded_level(w.nt, w.ntau, w.beta, w.h)
    assert_close(herm_to_oracle(G, g, 0), Go)
