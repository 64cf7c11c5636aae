"""Pins for the oracle's integral-form Dyson solver (oracle/vie2.py, Sec. "vie2: Dyson
equation in integral form"): the identity F = 0, brute-force downfolding written as
G = g0 + g0 * Sigma * G, i.e. (1 + F) * G = Q with F = -g0 * Sigma, F^ddagger = -Sigma * g0,
Q = g0 (Sec. "Test of accuracy and scaling analysis"), for a single level and a d = 2 cluster
with a complex coupling, agreement of the two schedules and of the integro-differential
solver, and a planted error."""
import numpy as np
import pytest

from oracle import conv, drivers, vie2
from oracle.contour import Func, Herm
from oracle.freegf import green_from_H
from oracle.weights import Weights
from tests.oracle_cases import max_err


def _convolve_all(N, T, A, B, W, beta, h, sign=1.0):
    C = Herm(N, T, A.d)
    for n in range(-1, N + 1):
        conv.convolution_timestep(n, C, A, A, None, B, B, W, beta, h)
    for c in ("mat", "ret", "les", "tv"):
        setattr(C, c, sign * getattr(C, c))
    return C


def _cluster(d, nbath, seed, vscale=0.4):
    rng = np.random.default_rng(seed)

    def herm(n):
        a = rng.normal(0, 1, (n, n)) + 1j * rng.normal(0, 1, (n, n))
        return 0.5 * (a + a.conj().T)

    hc, hb = herm(d), herm(nbath)
    V = vscale * (rng.normal(0, 1, (d, nbath)) + 1j * rng.normal(0, 1, (d, nbath)))
    return hc, hb, V


def _downfold_vie2(hc, hb, V, N, T, beta, h, schedule="mixed", k=5):
    """G of the cluster from (1 + F) * G = Q with F = -g0 * Sigma, Q = g0; and the exact block."""
    d = hc.shape[0]
    W = Weights(k)
    full = np.block([[hc, V], [V.conj().T, hb]])
    ex = green_from_H(N, T, full, 0.0, beta, h)
    g0 = green_from_H(N, T, hc, 0.0, beta, h)
    bath = green_from_H(N, T, hb, 0.0, beta, h)
    S = Herm(N, T, d)
    for c in ("mat", "ret", "les", "tv"):
        setattr(S, c, np.einsum("ab,...bc,dc->...ad", V, getattr(bath, c), V.conj()))
    F = _convolve_all(N, T, g0, S, W, beta, h, -1.0)
    Fcc = _convolve_all(N, T, S, g0, W, beta, h, -1.0)
    G = Herm(N, T, d)
    vie2.solve_vie2(G, F, Fcc, g0, beta, h, W, schedule=schedule)
    return G, ex, S


def test_zero_kernel_gives_the_source():
    """F = 0: G = Q on every component (the solver only copies and solves identities)."""
    N, T, beta, h = 16, 20, 2.0, 0.05
    W = Weights(5)
    Q = green_from_H(N, T, np.array([[0.3, 0.1j], [-0.1j, -0.4]]), 0.0, beta, h)
    F = Herm(N, T, 2)
    G = Herm(N, T, 2)
    vie2.solve_vie2(G, F, F, Q, beta, h, W)
    e = max_err(G, Q, sub=(slice(None), slice(None)))
    assert max(e.values()) < 1e-13, e


def test_embedded_level_brute_force_and_rate():
    """The embedded level (eps = 0.5, V = 0.3, eps_b = -0.2) through vie2 against the exact 2 x 2
    eigen-evolution; the error falls by more than 2^(k+1) per halving of h (the paper's average
    error of the integral form is O(h^(k+2)))."""
    hc, hb, V = np.array([[0.5]]), np.array([[-0.2]]), np.array([[0.3]])
    errs = []
    for N in (10, 20, 40):
        G, ex, _ = _downfold_vie2(hc, hb, V, N, 40, 2.0, 2.0 / N)
        e = max_err(G, ex)
        assert e["mat"] < 1e-12, e
        errs.append(max(e["ret"], e["les"], e["tv"]))
    assert errs[-1] < 1e-11, errs
    for a, b in zip(errs, errs[1:]):
        assert a / b > 0.7 * 2 ** 6, errs


@pytest.mark.parametrize("schedule", ["mixed", "serial"])
def test_multiorbital_downfolding_vie2(schedule):
    """A d = 2 cluster with complex h_c and V, 2-site bath: every component against the cluster
    block of the exact 4-level evolution, the error falling at least 2^(k+1) per halving."""
    hc, hb, V = _cluster(2, 2, 17)
    errs = []
    for N in (20, 40):
        G, ex, _ = _downfold_vie2(hc, hb, V, N, 64, 1.0, 1.0 / N, schedule=schedule)
        errs.append(max_err(G, ex, sub=(slice(0, 2), slice(0, 2))))
    assert errs[-1]["mat"] < 1e-10, errs
    for c in ("ret", "les", "tv"):
        assert errs[0][c] / errs[1][c] > 0.7 * 2 ** 6, (c, errs)
    assert max(errs[-1].values()) < 1e-8, errs


def test_schedules_and_integro_differential_form_agree():
    """The serial (A) and mixed (B) vie2 schedules, and the integro-differential dyson solver on
    the same problem, differ at discretisation level only."""
    hc, hb, V = _cluster(2, 2, 23)
    N, T, beta, h = 30, 40, 1.5, 0.05
    Gm, ex, S = _downfold_vie2(hc, hb, V, N, T, beta, h, "mixed")
    Gs, _, _ = _downfold_vie2(hc, hb, V, N, T, beta, h, "serial")
    Gd = Herm(N, T, 2)
    eps = Func(N, 2)
    eps.val[:] = hc
    drivers.solve_fixed_sigma(Gd, S, eps, 0.0, beta, h, Weights(5))
    full = (slice(None), slice(None))
    e_ex = max(max_err(Gm, ex, sub=(slice(0, 2), slice(0, 2))).values())
    d_sm = max(max_err(Gm, Gs, sub=full).values())
    d_dy = max(max_err(Gm, Gd, sub=full).values())
    assert 0 < d_sm < 10 * e_ex + 1e-12, (d_sm, e_ex)
    dyson_err = max(max_err(Gd, ex, sub=(slice(0, 2), slice(0, 2))).values())
    assert d_dy < 2 * (dyson_err + e_ex), (d_dy, dyson_err, e_ex)


def test_planted_kernel_conjugation_error_is_caught(monkeypatch):
    """Dropping the hermitian conjugations of the conjugate (B) lesser step (its kernel
    [F^R(n,l)]^dagger and the continuation of G^<) breaks the d = 2 brute-force pin."""
    hc, hb, V = _cluster(2, 2, 17)
    ok = max_err(*_downfold_vie2(hc, hb, V, 20, 40, 1.0, 0.05)[:2], sub=(slice(0, 2), slice(0, 2)))
    orig_dag = vie2.dag

    def broken(G, F, Fcc, Q, h, beta, W, n):
        vie2.dag = lambda x: x
        try:
            # every conjugation in the step becomes the identity: the kernel and G^<(n, l), l < n
            return orig_les(G, F, Fcc, Q, h, beta, W, n)
        finally:
            vie2.dag = orig_dag

    orig_les = vie2.les_col_B
    monkeypatch.setattr(vie2, "les_col_B", broken)
    bad = max_err(*_downfold_vie2(hc, hb, V, 20, 40, 1.0, 0.05)[:2], sub=(slice(0, 2), slice(0, 2)))
    assert bad["les"] > 100 * ok["les"], (ok, bad)
