"""Observables of a solved contour Green's function (oracle).

* density matrix rho(t) = -i G^<(t,t) (Sec. "Hubbard chain", density_matrix)
* particle number N(t) = Tr rho(t)
* kinetic energy E_kin(t) = (1/N_k) sum_k Tr[rho_k(t) eps_k(t)]  (Sec. "GW ... Hubbard model")
* correlation energy E_corr(t) = 1/2 Im Tr[Sigma * G]^<(t,t) through the convolution pieces
  C^<_1 + C^<_2 + C^<_3 at (t,t) (Eq. Total_ener, Galitskii-Migdal).
"""
import numpy as np

from . import conv


def density_matrix(n, G):
    return -1j * G.les[n, n]


def particle_number(n, G):
    return float(np.real(np.trace(density_matrix(n, G))))


def kinetic_energy(n, Gks, eps):
    return float(np.real(sum(np.trace(density_matrix(n, G) @ e(n)) for G, e in zip(Gks, eps)))) / len(Gks)


def correlation_energy(n, G, S, W, beta, h):
    c = (conv.cles1(S, S, None, G, G, n, n, W, h) + conv.cles2(S, S, None, G, G, n, n, W, h)
         + conv.cles3(S, S, None, G, G, n, n, W, beta))
    return 0.5 * float(np.imag(np.trace(c)))
