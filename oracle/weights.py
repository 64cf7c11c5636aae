"""Integration weights from exact rational arithmetic (oracle; test infrastructure only).

Follows the paper's Sec. "Basic integration and differentiation rules":
  * polynomial interpolation P^(k) = M^-1 with M_ja = j^a          (Eq. integrator_P)
  * polynomial differentiation D^(k)_{m,l}                          (Eq. integrator_D)
  * polynomial integration I^(k)_{m,n,l}                            (Eq. integrator_I)
  * backward differentiation a^(k)_j = -D^(k)_{0,j}                 (Eq. integrator_bd, Table tab:integrator_bd)
  * Gregory weights w^(k)_{n,j}                                     (Eq. integrator_greg, Table tab:gregory)
  * boundary convolution R^(k)_{m;r,s}                              (Eq. integrator_R)
  * extrapolation C^(k)_l                                           (Eq. polyextrap)

Reading of the Gregory weights (the paper's prose and its table disagree): for n <= k the
starting weights s_{n,j} = I_{0,n,j}; for n > k the classical Gregory rule, i.e. the
trapezoidal rule with end corrections made of forward differences at t=0 and backward
differences at t=nh up to order k, coefficients taken from the Gregory coefficients
G_i defined by t/ln(1+t) = sum_i G_i t^i.  This reproduces the printed table for k=0,1,2.
The BDF-based construction in the prose does not (k=1 would give the rectangle rule).
"""
from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

import numpy as np


def _inverse(mat):
    """Gauss-Jordan inverse of a square matrix of Fractions (exact)."""
    n = len(mat)
    a = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(mat)]
    for c in range(n):
        p = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[p] = a[p], a[c]
        piv = a[c][c]
        a[c] = [x / piv for x in a[c]]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [row[n:] for row in a]


@lru_cache(maxsize=None)
def P(k):
    """P^(k)_{a,l} = (M^-1)_{a,l}, M_{j,a} = j^a, j,a = 0..k (Eq. integrator_P)."""
    M = [[Fraction(j) ** a for a in range(k + 1)] for j in range(k + 1)]
    return tuple(tuple(r) for r in _inverse(M))


@lru_cache(maxsize=None)
def D(k):
    """D^(k)_{m,l} = sum_{a=1..k} P_{a,l} a m^(a-1), m,l = 0..k (Eq. integrator_D)."""
    p = P(k)
    return tuple(tuple(sum((p[a][l] * a * Fraction(m) ** (a - 1) for a in range(1, k + 1)), Fraction(0))
                       for l in range(k + 1)) for m in range(k + 1))


@lru_cache(maxsize=None)
def I(k):
    """I^(k)_{m,n,l} = sum_a P_{a,l} (n^(a+1) - m^(a+1))/(a+1), m,n,l = 0..k (Eq. integrator_I)."""
    p = P(k)
    out = {}
    for m in range(k + 1):
        for n in range(k + 1):
            out[(m, n)] = tuple(sum((p[a][l] * (Fraction(n) ** (a + 1) - Fraction(m) ** (a + 1)) / (a + 1)
                                     for a in range(k + 1)), Fraction(0)) for l in range(k + 1))
    return out


@lru_cache(maxsize=None)
def bdf(k):
    """a^(k)_j = -D^(k)_{0,j}, j = 0..k (Eq. integrator_bd)."""
    return tuple(-x for x in D(k)[0])


@lru_cache(maxsize=None)
def gregory_coefficients(nmax):
    """G_0..G_nmax from t/ln(1+t) = sum G_i t^i (series inversion of ln(1+t)/t)."""
    c = [Fraction((-1) ** i, i + 1) for i in range(nmax + 1)]  # ln(1+t)/t
    g = [Fraction(0)] * (nmax + 1)
    g[0] = Fraction(1)
    for i in range(1, nmax + 1):
        g[i] = -sum((c[j] * g[i - j] for j in range(1, i + 1)), Fraction(0))
    return tuple(g)


def gregory_row(k, n):
    """Exact weights w^(k)_{n,j}, j = 0..m(n,k) (Eq. integrator_greg).

    n <= k: starting weights s_{n,j} = I_{0,n,j}, j = 0..k.
    n > k : trapezoid plus end corrections of forward/backward differences up to order k.
    """
    if n <= k:
        return list(I(k)[(0, n)])
    G = gregory_coefficients(k + 1)
    w = [Fraction(1)] * (n + 1)
    # integral = sum_j f_j - sum_{i=1..k+1} |G_i| (nabla^{i-1} f_n + (-1)^{i-1} Delta^{i-1} f_0)
    for i in range(1, k + 2):
        p = i - 1
        g = abs(G[i])
        for q in range(p + 1):
            w[n - q] -= g * (-1) ** q * comb(p, q)               # nabla^p f_n
            w[q] -= g * (-1) ** p * (-1) ** (p - q) * comb(p, q)  # (-1)^p Delta^p f_0
    return w


@lru_cache(maxsize=None)
def R(k, m):
    """R^(k)_{m;r,s} = sum_{a,b} P_{a,r} P_{b,s} int_0^m (m-x)^a x^b dx (Eq. integrator_R).

    The inner integral is the Beta integral m^(a+b+1) a! b! / (a+b+1)!.
    """
    p = P(k)
    out = [[Fraction(0)] * (k + 1) for _ in range(k + 1)]
    for r in range(k + 1):
        for s in range(k + 1):
            acc = Fraction(0)
            for a in range(k + 1):
                for b in range(k + 1):
                    acc += p[a][r] * p[b][s] * Fraction(m) ** (a + b + 1) * Fraction(
                        factorial(a) * factorial(b), factorial(a + b + 1))
            out[r][s] = acc
    return tuple(tuple(r) for r in out)


@lru_cache(maxsize=None)
def extrap(k):
    """C^(k)_l, y_{n+1} = sum_l C_l y_{n-l}: the interpolant through y_{n-k..n} at one step
    beyond (Eq. polyextrap)."""
    p = P(k)
    # points z_j = y_{n-k+j}, j=0..k; evaluate at j = k+1; y_{n-l} = z_{k-l}
    return tuple(sum((Fraction(k + 1) ** a * p[a][k - l] for a in range(k + 1)), Fraction(0))
                 for l in range(k + 1))


class Weights:
    """FP64 copies of the exact weights for one order k (the oracle's integrator)."""

    def __init__(self, k):
        if not 0 <= k <= 6:
            raise ValueError("order k must be 0..6")
        self.k = k
        self.P = np.array(P(k), dtype=float)
        self.D = np.array(D(k), dtype=float)
        Ik = I(k)
        self.I = np.array([[Ik[(m, n)] for n in range(k + 1)] for m in range(k + 1)], dtype=float)
        self.a = np.array(bdf(k), dtype=float)
        self.C = np.array(extrap(k), dtype=float)
        self._R = {}
        self._w = {}

    def w(self, n):
        """Gregory row w_{n, 0..m(n,k)} as a float array."""
        if n not in self._w:
            self._w[n] = np.array(gregory_row(self.k, n), dtype=float)
        return self._w[n]

    def R(self, m):
        if m not in self._R:
            self._R[m] = np.array(R(self.k, m), dtype=float)
        return self._R[m]
