"""Pins for the oracle's Dyson solver: closed forms, downfolding brute force, convergence
rates, schedule agreement and the contour identities."""
import numpy as np
import pytest

from oracle import conv, drivers, dyson
from oracle.contour import Func, Herm, dag
from oracle.freegf import green_from_H
from oracle.weights import Weights
from tests.oracle_cases import embedded_level, max_err


def test_free_closed_form_identities():
    """Jump G^M(0+) - xi G^M(beta-) = -1, KMS (Eq. kmsbound_keld), G^R(t,t) = -i (Eq. gretdiag)
    and the equation of motion i dG^R/dt = (eps - mu) G^R by central differences."""
    eps = np.array([[0.4, 0.2 - 0.1j], [0.2 + 0.1j, -0.7]])
    N, T, beta, h = 12, 16, 3.0, 0.01
    G = green_from_H(N, T, eps, 0.1, beta, h)
    assert np.allclose(G.mat[0] - G.sig * G.mat[T], -np.eye(2), atol=1e-14)
    for m in range(T + 1):
        assert np.allclose(G.tv[0, m], 1j * G.sig * G.mat[T - m], atol=1e-14)
    for n in range(N + 1):
        assert np.allclose(G.ret[n, n], -1j * np.eye(2), atol=1e-14)
        assert np.allclose(G.les[0, n], -dag(G.tv[n, 0]), atol=1e-14)
    for n in range(1, N):
        dG = (G.ret[n + 1, 0] - G.ret[n - 1, 0]) / (2 * h)
        assert np.allclose(1j * dG, (eps - 0.1 * np.eye(2)) @ G.ret[n, 0], atol=1e-4)


def test_sigma_zero_gives_free_gf():
    """With Sigma = 0 the solver reproduces the closed-form free GF to BDF accuracy."""
    N, T, beta, h = 30, 30, 5.0, 0.05
    ex = green_from_H(N, T, np.array([[0.3]]), 0.0, beta, h)
    G, S = Herm(N, T, 1), Herm(N, T, 1)
    eps = Func(N, 1)
    eps.val[:] = 0.3
    drivers.solve_fixed_sigma(G, S, eps, 0.0, beta, h, Weights(5))
    e = max_err(G, ex)
    assert e["mat"] < 1e-13 and max(e.values()) < 1e-9, e


def test_downfolding_brute_force_and_rate():
    """Embedded level vs the exact 2x2 eigen-evolution; the error falls ~2^k per halving of h
    (k = 5; the paper's average error is O(h^(k+1)))."""
    errs = []
    for N in (20, 40, 80):
        G, ex, _ = embedded_level(N, 40, 2.0, 2.0 / N)
        e = max_err(G, ex)
        assert e["mat"] < 1e-12
        errs.append(max(e["ret"], e["les"], e["tv"]))
    assert errs[-1] < 3e-10
    for a, b in zip(errs, errs[1:]):
        assert a / b > 2 ** 5 * 0.7, errs


def test_matsubara_converges_fast_in_htau():
    """Matsubara downfolding error falls roughly as h_tau^(k+2) (Fig. test_eq), k = 3."""
    W = Weights(3)
    errs = []
    beta = 20.0
    e1, lam, e2 = -1.0, 0.5, 1.0
    for T in (50, 100, 200):
        ex = green_from_H(0, T, np.array([[e1, 1j * lam], [-1j * lam, e2]]), 0.0, beta, 0.1)
        S = green_from_H(0, T, np.array([[e2]]), 0.0, beta, 0.1)
        S.mat *= lam ** 2
        G = Herm(0, T, 1)
        eps = Func(0, 1)
        eps.val[:] = e1
        dyson.dyson_mat(G, S, eps, 0.0, beta, W)
        errs.append(np.abs(G.mat[:, 0, 0] - ex.mat[:, 0, 0]).mean())
    rate = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert min(rate) > 3.5, (errs, rate)


def test_serial_and_mixed_schedules_agree_to_discretisation():
    """Implementations (A) and (B) differ only at the discretisation level."""
    Gm, ex, _ = embedded_level(40, 30, 2.0, 0.05, schedule="mixed")
    Gs, _, _ = embedded_level(40, 30, 2.0, 0.05, schedule="serial")
    d = max_err(Gm, Gs, sub=(slice(None), slice(None)))
    e = max_err(Gm, ex)
    assert 0 < max(d.values()) < 10 * max(e.values())


def test_contour_identities_of_solution():
    """Solution satisfies G^R(t,t) = -i, KMS for tv and les, hermitian density matrix."""
    G, _, _ = embedded_level(25, 20, 2.0, 0.05)
    T = G.ntau
    for n in range(G.nt + 1):
        assert abs(G.ret[n, n, 0, 0] + 1j) < 1e-13
        assert np.allclose(G.les[0, n], -dag(G.tv[n, 0]), atol=1e-13)
        assert abs(np.real(G.les[n, n, 0, 0])) < 1e-10     # rho = -iG^< real up to discretisation
    for m in range(T + 1):
        assert np.allclose(G.tv[0, m], 1j * G.sig * G.mat[T - m], atol=1e-13)


def _d_eps_free(N, T, e, beta, h, de=1e-5):
    """dG0/de by central difference of the closed form; equals [G0 * G0] (G0 = (i d_t - e)^-1)."""
    gp = green_from_H(N, T, np.array([[e + de]]), 0.0, beta, h)
    gm = green_from_H(N, T, np.array([[e - de]]), 0.0, beta, h)
    out = Herm(N, T, 1)
    for c in ("mat", "ret", "les", "tv"):
        setattr(out, c, (getattr(gp, c) - getattr(gm, c)) / (2 * de))
    return out


def test_convolution_timestep_equals_energy_derivative():
    """[G0 * G0] = dG0/de for a free GF: pins every piece C^M, C^R, C^tv_1..3, C^<_1..3."""
    N, T, beta, h, e = 24, 60, 3.0, 0.05, 0.35
    W = Weights(5)
    g = green_from_H(N, T, np.array([[e]]), 0.0, beta, h)
    C = Herm(N, T, 1)
    for n in range(-1, N + 1):
        conv.convolution_timestep(n, C, g, g, None, g, g, W, beta, h)
    ref = _d_eps_free(N, T, e, beta, h)
    err = max_err(C, ref)
    assert max(err.values()) < 2e-7, err


def test_planted_kernel_sign_error_is_caught(monkeypatch):
    """Planting a wrong sign in the tv history kernel breaks the downfolding pin."""
    orig = dyson.tv_row

    def broken(G, S, eps, mu, h, beta, W, n, Mn_inv):
        S2 = S.copy()
        S2.ret = -S2.ret
        return orig(G, S2, eps, mu, h, beta, W, n, Mn_inv)

    monkeypatch.setattr(dyson, "tv_row", broken)
    G, ex, _ = embedded_level(20, 20, 2.0, 0.1)
    assert max_err(G, ex)["tv"] > 1e-4


def test_equilibrium_time_translation_invariance():
    """A time-independent problem in equilibrium (the embedded level, Sigma = V^2 g0) has
    G(t, t') depending on t - t' only and a constant density: the discrete solution keeps
    this to discretisation accuracy, and the deviation falls with h like the solver's error."""
    devs = []
    for N in (20, 40):
        h = 2.0 / N
        G, _, _ = embedded_level(N, 40, 2.0, h)
        R, L = G.ret[..., 0, 0], G.les[..., 0, 0]
        d = 0.0
        for lag in range(0, N // 2):
            r = np.array([R[n, n - lag] for n in range(lag, N + 1)])
            l = np.array([L[n - lag, n] for n in range(lag, N + 1)])
            d = max(d, np.abs(r - r[0]).max(), np.abs(l - l[0]).max())
        dens = np.array([L[n, n] for n in range(N + 1)])
        d = max(d, np.abs(dens - dens[0]).max())
        devs.append(d)
    assert devs[-1] < 1e-8, devs
    assert devs[0] / devs[1] > 2 ** 5 * 0.7, devs
