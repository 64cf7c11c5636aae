"""Pins of the oracle's GW self-energy (oracle/gw.py) by facts independent of its code:

* a free single level (and diagonal levels): P is constant on every component, P^R = 0, so the
  susceptibility equation has the closed form chi^M = c / (1 - c U(0^-) beta), c = -f(1 - f),
  chi^< = chi^> = chi^tv = i chi^M, chi^R = 0, and Sigma(t,t') = -U(t) U(t') chi^M G(t,t') on
  every component, also for a time-dependent U(t);
* the contour boundary conditions C^tv(0, tau) = i C^M(-tau) and C^<(0,0) = C^tv(0,0) for P and
  Sigma of a non-diagonal cluster (they tie the Matsubara rule of each bubble to its real-time
  rules);
* the expansion in U: Sigma_GW - Sigma_2B = O(U^3), with the U^3 term i G U (P * U * P) U
  computed by the convolution oracle (pins the sign of the kernel K = -P U of the chi equation);
* planted errors (the printed sign of the Bubble1 Matsubara rule, a sign of K) fail these pins.
"""
import numpy as np
import pytest

from oracle import bubble, conv, gw
from oracle.contour import Func, Herm
from oracle.freegf import fermi, green_from_H
from oracle.weights import Weights

K = 5


def _ufunc(N, u):
    U = Func(N, 1)
    for n in range(-1, N + 1):
        U.set(n, np.array([[u(n)]], complex))
    return U


def _run_gw(G, U, beta, h, W):
    N, T, d = G.nt, G.ntau, G.d
    chain = gw.GW(N, T, d, beta, h, W)
    S = Herm(N, T, d)
    chain.mat(G, U, S)
    chain.start(G, U, S)
    for n in range(W.k + 1, N + 1):
        chain.step(n, G, U, S)
    return chain, S


def _low(N):
    return np.tril(np.ones((N + 1, N + 1), bool))


@pytest.mark.parametrize("levels", [[0.4], [0.4, -0.7]])
def test_free_levels_closed_form(levels):
    N, T, beta, h, U0 = 16, 20, 2.0, 0.05, 0.8
    W = Weights(K)
    G = green_from_H(N, T, np.diag(levels), 0.0, beta, h)
    u = lambda n: U0 if n < 0 else U0 * (1.0 + 0.3 * np.sin(0.7 * n * h))
    chain, S = _run_gw(G, _ufunc(N, u), beta, h, W)
    d = len(levels)
    low = _low(N)
    for a in range(d):
        f = fermi(levels[a], beta)
        c = -f * (1.0 - f)
        chim = c / (1.0 - c * U0 * beta)
        chi = chain.chi
        assert np.abs(chi.mat[:, a, a] - chim).max() < 1e-13
        assert np.abs(chi.tv[:, :, a, a] - 1j * chim).max() < 1e-13
        assert np.abs(chi.les[low.T][:, a, a] - 1j * chim).max() < 1e-13
        assert np.abs(chi.ret[low][:, a, a]).max() < 1e-13
        us = np.array([u(n) for n in range(N + 1)])
        assert np.abs(S.mat[:, a, a] + U0 ** 2 * chim * G.mat[:, a, a]).max() < 1e-13
        for n in range(N + 1):
            for j in range(n + 1):
                w = -us[n] * us[j] * chim
                assert abs(S.ret[n, j, a, a] - w * G.ret[n, j, a, a]) < 1e-13
                assert abs(S.les[j, n, a, a] - w * G.les[j, n, a, a]) < 1e-13
            assert np.abs(S.tv[n, :, a, a] + us[n] * U0 * chim * G.tv[n, :, a, a]).max() < 1e-13
    if d > 1:
        off = ~np.eye(d, dtype=bool)
        for X in (chain.chi, S):
            assert np.abs(X.mat[:, off]).max() < 1e-14
            assert np.abs(X.tv[:, :, off]).max() < 1e-14


def _cluster_G(N, T, beta, h, seed=3):
    rng = np.random.default_rng(seed)
    a = rng.normal(0, 1, (2, 2)) + 1j * rng.normal(0, 1, (2, 2))
    return green_from_H(N, T, 0.5 * (a + a.conj().T), 0.1, beta, h)


def test_boundary_conditions_of_P_and_sigma():
    N, T, beta, h = 12, 24, 1.5, 0.05
    W = Weights(K)
    G = _cluster_G(N, T, beta, h)
    chain, S = _run_gw(G, _ufunc(N, lambda n: 0.6), beta, h, W)
    P = chain.P
    for X, xi in ((P, +1), (S, -1), (chain.chi, +1)):
        # C^tv(0, tau_m) = i C^M(-tau_m) = i xi C^M(beta - tau_m)
        assert np.abs(X.tv[0] - 1j * xi * X.mat[::-1]).max() < 1e-13 * max(1.0, np.abs(X.mat).max())
    # C^<(0,0) = C^tv(0,0): exact for P; for chi (so for Sigma) only up to the quadrature error
    # of the Matsubara solve, whose chi^M(beta) is hermitian to that accuracy
    assert np.abs(P.les[0, 0] - P.tv[0, 0]).max() < 1e-15
    assert np.abs(S.les[0, 0] - S.tv[0, 0]).max() < 1e-8
    # the equal-time bosonic P is anti-hermitian on the lesser component: P^<(t,t)^dagger = -P^<(t,t)
    for n in range(N + 1):
        assert np.abs(P.les[n, n] + P.les[n, n].conj().T).max() < 1e-14


def _sigma_2b_all(G, U):
    S = Herm(G.nt, G.ntau, G.d)
    for n in range(-1, G.nt + 1):
        bubble.sigma_2b(n, G, U, S)
    return S


def _pp(P, beta, h, W):
    C = Herm(P.nt, P.ntau, P.d, sig=+1)
    for n in range(-1, P.nt + 1):
        conv.convolution_timestep(n, C, P, P, None, P, P, W, beta, h)
    return C


def _flat(X):
    N = X.nt
    low = _low(N)
    return np.concatenate([X.mat.ravel(), X.ret[low].ravel(), X.les[low.T].ravel(), X.tv.ravel()])


def _expansion_errors(N, T, beta, h, U0s):
    W = Weights(K)
    G = _cluster_G(N, T, beta, h)
    e2, e3, size3 = [], [], []
    PP = None
    for U0 in U0s:
        U = _ufunc(N, lambda n: U0)
        chain, S = _run_gw(G, U, beta, h, W)
        if PP is None:
            PP = _pp(chain.P, beta, h, W)
        s2 = _sigma_2b_all(G, U)
        dW3 = Herm(N, T, G.d, sig=+1)
        for c in ("mat", "ret", "les", "tv"):
            setattr(dW3, c, U0 ** 3 * getattr(PP, c))
        s3 = Herm(N, T, G.d)
        for n in range(-1, N + 1):
            gw.bubble2(n, G, dW3, s3)
        d2 = _flat(S) - _flat(s2)
        e2.append(np.abs(d2).max())
        e3.append(np.abs(d2 - _flat(s3)).max())
        size3.append(np.abs(_flat(s3)).max())
    return np.array(e2), np.array(e3), np.array(size3)


def test_expansion_in_U_matches_second_born_and_third_order():
    e2, e3, size3 = _expansion_errors(12, 24, 1.5, 0.05, (0.2, 0.1))
    # Sigma_GW - Sigma_2B is the third-order term up to O(U^4)
    assert 6.5 < e2[0] / e2[1] < 9.5, e2
    assert 13.0 < e3[0] / e3[1] < 19.0, e3
    assert np.all(e3 < 0.25 * size3), (e3, size3)


def test_planted_bubble1_matsubara_sign_fails_closed_form(monkeypatch):
    orig = gw.bubble1

    def printed_sign(n, A, B, C):
        orig(n, A, B, C)
        if n == -1:
            C.mat *= -1.0

    monkeypatch.setattr(gw, "bubble1", printed_sign)
    with pytest.raises(AssertionError):
        test_free_levels_closed_form([0.4])


def test_planted_kernel_sign_fails_expansion(monkeypatch):
    orig = gw.GW._kernel

    def flipped(self, n, G, U):
        orig(self, n, G, U)
        for X in (self.K, self.Kcc):
            if n == -1:
                X.mat *= -1.0
            else:
                X.ret[n, :n + 1] *= -1.0
                X.les[:n + 1, n] *= -1.0
                X.tv[n] *= -1.0

    monkeypatch.setattr(gw.GW, "_kernel", flipped)
    with pytest.raises(AssertionError):
        test_expansion_in_U_matches_second_born_and_third_order()


def _quench_U(N, u_after, u_before):
    U = Func(N, 1)
    U.val[:] = u_after
    U.set(-1, np.array([[u_before]], complex))
    return U


@pytest.mark.slow
def test_dimer_quench_conservation_gw():
    """Self-consistent GW Hubbard dimer after the quench U: 1 -> 2 (GW is a conserving
    approximation): the Galitskii-Migdal energy (Eq. Total_ener) and the particle number stay
    constant for t > 0 up to the discretisation, and the energy drift falls under halving of h."""
    from oracle import drivers, observables
    drifts, ndrift = [], []
    for N, h in ((40, 0.1), (80, 0.05)):
        W = Weights(K)
        e0 = Func(N, 2)
        e0.val[:] = np.array([[0.0, -1.0], [-1.0, 0.0]])
        U = _quench_U(N, 2.0, 1.0)
        st, chain = drivers.run_gw([e0], U, N, 30, 5.0, h, W, corrector=3)
        G, S = st.G[0], st.S
        E, Nn = [], []
        for n in range(N + 1):
            rho = observables.density_matrix(n, G)
            E.append(0.5 * np.real(np.trace(rho @ (e0(n) + st.epsmf[0](n))))
                     + observables.correlation_energy(n, G, S, W, 5.0, h))
            Nn.append(np.real(np.trace(rho)))
        drifts.append(np.ptp(E[1:]))
        ndrift.append(np.ptp(Nn))
    assert drifts[1] < drifts[0] / 8 and drifts[1] < 1e-3, drifts
    assert ndrift[1] < 1e-4, ndrift


# ---- k-space GW (Eqs. Sigmak, Pol) against the real-space GW of the same ring ----------------
def _ring_k(nk):
    return 2 * np.pi * np.arange(nk) / nk


def _to_real_space(Gk, N, T, sig=-1):
    """G_ij = (1/N_k) sum_k exp(i k (r_i - r_j)) G_k on a ring of N_k sites (d = N_k)."""
    nk = len(Gk)
    ks = _ring_k(nk)
    r = np.arange(nk)
    ph = np.exp(1j * ks[None, None, :] * (r[:, None, None] - r[None, :, None])) / nk   # [i, j, k]
    X = Herm(N, T, nk, sig=sig)
    for c in ("mat", "ret", "les", "tv"):
        stack = np.stack([getattr(g, c)[..., 0, 0] for g in Gk], axis=-1)         # [..., k]
        setattr(X, c, np.einsum("...k,ijk->...ij", stack, ph))
    return X


def _to_momentum(X, nk, comp):
    """X_q = sum_r exp(-i q r) X(r), X(r) = X_{r,0} of a translation-invariant real-space herm."""
    ks = _ring_k(nk)
    a = getattr(X, comp)[..., :, 0]                                                 # [..., r]
    ph = np.exp(-1j * ks[:, None] * np.arange(nk)[None, :])                         # [q, r]
    return np.einsum("...r,qr->...q", a, ph)


def _kspace_fixed_G(nk, N, T, beta, h, A0):
    ks = _ring_k(nk)
    return [green_from_H(N, T, np.array([[-2.0 * np.cos(k - A0)]]), 0.1, beta, h) for k in ks]


def _run_kspace_chain(Gk, U, beta, h, W):
    N, T, nk = Gk[0].nt, Gk[0].ntau, len(Gk)
    add, neg = gw.ring_tables(nk)
    chain = gw.GWk(N, T, nk, beta, h, W, add, neg)
    Sk = [Herm(N, T, 1) for _ in range(nk)]
    chain.mat(Gk, U, Sk)
    chain.start(Gk, U, Sk)
    for n in range(W.k + 1, N + 1):
        chain.step(n, Gk, U, Sk)
    return chain, Sk


def test_kspace_gw_equals_real_space_gw_on_a_ring():
    """For fixed G_k of a shifted dispersion (no k -> -k symmetry), the momentum sums of the
    k-space chain reproduce, after the lattice Fourier transform, the real-space GW chain of
    the ring (P, chi and Sigma as d x d functions of the site indices)."""
    nk, N, T, beta, h = 4, 12, 16, 2.0, 0.05
    W = Weights(K)
    Gk = _kspace_fixed_G(nk, N, T, beta, h, A0=0.4)
    U = _ufunc(N, lambda n: 0.7 if n < 0 else 0.7 + 0.2 * np.sin(0.5 * n * h))
    chain_k, Sk = _run_kspace_chain(Gk, U, beta, h, W)
    Greal = _to_real_space(Gk, N, T)
    chain_r, Sreal = _run_gw(Greal, U, beta, h, W)
    low = _low(N)
    for name, xk, xr in (("P", chain_k.P, chain_r.P), ("chi", chain_k.chi, chain_r.chi), ("Sigma", Sk, Sreal)):
        for c in ("mat", "ret", "les", "tv"):
            got = np.stack([getattr(x, c)[..., 0, 0] for x in xk], axis=-1)
            ref = _to_momentum(xr, nk, c)
            if c == "ret":
                got, ref = got[low], ref[low]
            if c == "les":
                got, ref = got[low.T], ref[low.T]
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err < 1e-12, (name, c, err)


def test_kspace_gw_planted_momentum_sign_fails(monkeypatch):
    orig = gw.ring_tables

    def k_minus_q(nk):
        add, neg = orig(nk)
        return add[:, neg], neg          # Pi_k from G_{k-q} G_q instead of G_{k+q} G_q

    monkeypatch.setattr(gw, "ring_tables", k_minus_q)
    with pytest.raises(AssertionError):
        test_kspace_gw_equals_real_space_gw_on_a_ring()


@pytest.mark.slow
def test_kspace_gw_self_consistent_equals_real_space_ring():
    """Self-consistent GW of a 4-site ring with a Peierls pulse: the k-space driver (nk = 4,
    one band, Sigma_k) and the real-space driver (one problem, d = 4 sites) give the same local
    Green's function on every stored element."""
    from oracle import drivers
    nk, N, T, beta, h = 4, 16, 16, 3.0, 0.05
    W = Weights(K)
    ks = _ring_k(nk)
    A = np.array([0.0] + [0.6 * np.sin(0.8 * n * h) for n in range(N + 1)])   # A(0^-) = 0
    eps_k = -2.0 * np.cos(ks[None, :] - A[:, None])                           # [nt+2, k]
    e0k = []
    for kk in range(nk):
        f = Func(N, 1)
        f.val[:, 0, 0] = eps_k[:, kk]
        e0k.append(f)
    r = np.arange(nk)
    ph = np.exp(1j * ks[None, None, :] * (r[:, None, None] - r[None, :, None])) / nk
    e0r = Func(N, nk)
    e0r.val[...] = np.einsum("tk,ijk->tij", eps_k, ph)
    U = _ufunc(N, lambda n: 1.0 if n < 0 else 1.5)
    stk, _ = drivers.run_gw_kspace(e0k, U, N, T, beta, h, W, *gw.ring_tables(nk), corrector=3)
    str_, _ = drivers.run_gw([e0r], U, N, T, beta, h, W, corrector=3)
    # st.Gloc holds the k-average taken before the last corrector's Dyson solve: average anew
    Gl, Gr = Herm(N, T, 1), str_.G[0]
    for c in ("mat", "ret", "les", "tv"):
        setattr(Gl, c, sum(getattr(g, c) for g in stk.G) / nk)
    low = _low(N)
    for c in ("mat", "ret", "les", "tv"):
        a, b = getattr(Gl, c)[..., 0, 0], getattr(Gr, c)[..., 0, 0]
        if c == "ret":
            a, b = a[low], b[low]
        if c == "les":
            a, b = a[low.T], b[low.T]
        assert np.abs(a - b).max() < 1e-10 * max(1.0, np.abs(b).max()), (c, np.abs(a - b).max())
