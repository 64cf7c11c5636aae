"""Pins for the oracle's integration weights against the paper's printed tables and
against exactness, closed forms and convergence rates."""
from fractions import Fraction
from math import comb
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import weights as wt

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    with open(os.path.join(GOLD, name)) as f:
        return [l.strip() for l in f if l.strip() and not l.startswith("#")]


def test_bdf_table():
    """Table tab:integrator_bd, k = 1..6 exactly."""
    for line in _read("bdf_table.txt"):
        k, vals = line.split(":")
        want = [Fraction(v) for v in vals.split()]
        assert list(wt.bdf(int(k))) == want


def test_gregory_table():
    """Table tab:gregory for k = 0, 1, 2 exactly (s block rows n <= k, Sigma block rows
    n = k+1..2k+1)."""
    for line in _read("gregory_table.txt"):
        head, rest = line.split(":")
        k, row = map(int, head.split())
        s_txt, sig_txt = rest.split("|")
        s = [Fraction(v) for v in s_txt.split()]
        sig = [Fraction(v) for v in sig_txt.split()]
        assert list(wt.gregory_row(k, row))[:k + 1] == s
        assert list(wt.gregory_row(k, k + 1 + row))[:k + 1] == sig


@pytest.mark.parametrize("k", range(0, 6))
def test_gregory_structure(k):
    """Row sums are n; for n >= 2k+1 both ends carry omega_j, interior weights are 1;
    the diagonal weight w_{n,n} = omega_0 for every n > k."""
    om = wt.gregory_row(k, 2 * k + 1)[:k + 1]
    for n in range(0, 4 * k + 8):
        w = wt.gregory_row(k, n)
        assert sum(w) == n
        if n > k:
            assert w[n] == om[0]
        if n >= 2 * k + 1:
            for j in range(k + 1):
                assert w[j] == om[j] and w[n - j] == om[j]
            for j in range(k + 1, n - k):
                assert w[j] == 1


@pytest.mark.parametrize("k", range(1, 6))
def test_gregory_polynomial_exactness(k):
    """The k-th order rule integrates polynomials of degree <= k exactly for every n."""
    for n in range(0, 3 * k + 6):
        w = wt.gregory_row(k, n)
        for deg in range(k + 1):
            exact = Fraction(n ** (deg + 1), deg + 1)
            approx = sum(w[j] * Fraction(j) ** deg for j in range(len(w)))
            assert approx == exact, (k, n, deg)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_gregory_convergence_rate(k):
    """Experiment of Fig. gregoryintegration: mean error of int_0^{x_n} exp(ix) on
    [0, 5 pi/2] falls as N^-(k+2)."""
    xmax = 2.5 * np.pi
    errs, Ns = [], [40, 80, 160]
    for N in Ns:
        h = xmax / N
        y = np.exp(1j * h * np.arange(N + 1))
        e = []
        for n in range(N + 1):
            w = np.array(wt.gregory_row(k, n), dtype=float)
            approx = h * np.dot(w, y[:len(w)])
            exact = -1j * (np.exp(1j * n * h) - 1)
            e.append(abs(approx - exact))
        errs.append(np.mean(e))
    slope = -np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert slope > k + 2 - 0.6, (k, slope, errs)


@pytest.mark.parametrize("k", range(1, 6))
def test_interpolation_differentiation_integration_exact(k):
    """P interpolates, D differentiates and I integrates polynomials of degree <= k exactly
    (Eqs. integrator_P, integrator_D, integrator_I)."""
    P, D, I = wt.P(k), wt.D(k), wt.I(k)
    for deg in range(k + 1):
        y = [Fraction(j) ** deg for j in range(k + 1)]
        for a in range(k + 1):
            coef = sum(P[a][l] * y[l] for l in range(k + 1))
            assert coef == (1 if a == deg else 0)
        for m in range(k + 1):
            dy = sum(D[m][l] * y[l] for l in range(k + 1))
            assert dy == (deg * Fraction(m) ** (deg - 1) if deg > 0 else 0)
            for n in range(k + 1):
                iy = sum(I[(m, n)][l] * y[l] for l in range(k + 1))
                assert iy == Fraction(n ** (deg + 1) - m ** (deg + 1), deg + 1)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_boundary_convolution_weights_vs_quadrature(k):
    """R^(k)_{m;r,s} equals the numerically integrated product of Lagrange basis
    polynomials, int_0^m L_r(m-x) L_s(x) dx (Eq. integrator_R)."""
    nodes = np.arange(k + 1)

    def lag(r, x):
        others = [j for j in nodes if j != r]
        return np.prod([(x - j) / (r - j) for j in others])

    for m in range(k + 1):
        R = np.array(wt.R(k, m), dtype=float)
        for r in range(k + 1):
            for s in range(k + 1):
                q = integrate.quad(lambda x: lag(r, m - x) * lag(s, x), 0, m, epsabs=1e-13)[0] if m else 0.0
                assert abs(R[r, s] - q) < 1e-9


@pytest.mark.parametrize("k", range(1, 6))
def test_extrapolation_closed_form(k):
    """C^(k)_l = (-1)^l binom(k+1, l+1), and extrapolation is exact for degree <= k."""
    C = wt.extrap(k)
    assert list(C) == [(-1) ** l * comb(k + 1, l + 1) for l in range(k + 1)]
    for deg in range(k + 1):
        n = 7
        pred = sum(C[l] * Fraction(n - l) ** deg for l in range(k + 1))
        assert pred == Fraction(n + 1) ** deg


def test_planted_gregory_sign_error_is_caught(monkeypatch):
    """A plausible mistake (dropping the sign flip of the backward differences) must fail
    the table pin."""
    orig = wt.gregory_row

    def broken(k, n):
        if n <= k:
            return orig(k, n)
        G = wt.gregory_coefficients(k + 1)
        w = [Fraction(1)] * (n + 1)
        for i in range(1, k + 2):
            p = i - 1
            for q in range(p + 1):
                w[n - q] -= abs(G[i]) * comb(p, q)
                w[q] -= abs(G[i]) * (-1) ** p * (-1) ** (p - q) * comb(p, q)
        return w

    monkeypatch.setattr(wt, "gregory_row", broken)
    with pytest.raises(AssertionError):
        test_gregory_table()


def test_layout_sizes_match_printed_hdf5_example():
    """Triangle and block sizes of the stored components (Eq. storage_herm) agree with the
    sizes printed for nt=200, ntau=400, d=1."""
    (line,) = _read("hdf5_sizes.txt")
    kv = dict(x.split("=") for x in line.split())
    nt, ntau = int(kv["nt"]), int(kv["ntau"])
    assert (nt + 1) * (nt + 2) // 2 == int(kv["ret"]) == int(kv["les"])
    assert (nt + 1) * (ntau + 1) == int(kv["tv"])
    assert ntau + 1 == int(kv["mat"])
