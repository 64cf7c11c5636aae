"""Closed-form free Green's functions of a constant hermitian d x d Hamiltonian (oracle).

Sec. "Implementation: Free Green's functions", Eq. G0_free, for eps constant in time, so
that the propagator U_{n,j} = exp(-i (eps - mu)(t_n - t_j)) is exact.  Readings of the
printed formulas (fixed by the jump condition G^M(0+) - xi G^M(beta-) = -1 and by KMS,
Eq. kmsbound_keld):
    G^M(tau)    = -R diag{(1 + xi f(e_a)) exp(-e_a tau)} R^dagger
    G^R(t,t')   = -i U(t,t')
    G^<(t,t')   = -xi i R diag{f(e_a) exp(-i e_a (t - t'))} R^dagger
    G^tv(t,tau) = -i xi R diag{f(e_a) exp(-i e_a t) exp(e_a tau)} R^dagger
with e_a = eps_a - mu and f the Fermi (xi=-1) or Bose (xi=+1) function.
Only fermions (xi = -1) are exercised by the tests.
"""
import numpy as np

from .contour import Herm


def _fermi_terms(e, beta, tau, xi):
    """Return (1 + xi f(e)) exp(-e tau) and f(e) exp(e tau) in an overflow-safe form."""
    if xi != -1:
        f = 1.0 / (np.exp(beta * e) - 1.0)
        return (1.0 + f) * np.exp(-e * tau), f * np.exp(e * tau)
    if e >= 0:
        x = np.exp(-beta * e)
        one_minus_f = 1.0 / (1.0 + x)
        return one_minus_f * np.exp(-e * tau), x / (1.0 + x) * np.exp(e * tau)
    x = np.exp(beta * e)
    # 1-f = x/(1+x); (1-f) e^{-e tau} = e^{e(beta - tau)}/(1+x)
    return np.exp(e * (beta - tau)) / (1.0 + x), np.exp(e * tau) / (1.0 + x)


def fermi(e, beta):
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


def green_from_H(nt, ntau, eps, mu, beta, h, xi=-1):
    """Free Green's function for the constant Hamiltonian eps (d x d hermitian)."""
    eps = np.atleast_2d(np.asarray(eps, complex))
    d = eps.shape[0]
    ev, R = np.linalg.eigh(eps)
    e = ev - mu
    G = Herm(nt, ntau, d, xi)
    htau = beta / ntau
    Rd = R.conj().T
    for m in range(ntau + 1):
        tau = m * htau
        g = np.array([_fermi_terms(x, beta, tau, xi)[0] for x in e])
        G.mat[m] = -(R * g) @ Rd
    f = np.array([fermi(x, beta) if xi == -1 else 1.0 / (np.exp(beta * x) - 1.0) for x in e])
    for n in range(nt + 1):
        t = n * h
        for j in range(n + 1):
            ph = np.exp(-1j * e * (n - j) * h)
            G.ret[n, j] = -1j * (R * ph) @ Rd
            G.les[j, n] = -xi * 1j * (R * (f * np.conj(ph))) @ Rd
        for m in range(ntau + 1):
            tau = m * htau
            v = np.array([_fermi_terms(x, beta, tau, xi)[1] for x in e])
            G.tv[n, m] = -1j * xi * (R * (np.exp(-1j * e * t) * v)) @ Rd
    return G
