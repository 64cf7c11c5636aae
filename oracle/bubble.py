"""Second-Born self-energy, Hartree mean field and k-point reduction (oracle).

Second-Born (Eq. sigma_hubb_2b), spin-symmetric, elementwise in the orbital indices:
    Sigma_ab(t,t') = U(t) U(t') G_ab(t,t') G_ab(t,t') G_ba(t',t).
Keldysh components by the Langreth rules for products (Eqs. def_bubble1, def_bubble2):
    Sigma^<_ab(j,n)  = U_j U_n G^<_ab(j,n)^2 G^>_ba(n,j)
    Sigma^>_ab(n,j)  = U_n U_j G^>_ab(n,j)^2 G^<_ba(j,n)
    Sigma^R(n,j)     = Sigma^>(n,j) - Sigma^<(n,j)                        (Eq. defretarded)
    Sigma^tv_ab(n,m) = U_n U_{-1} G^tv_ab(n,m)^2 G^vt_ba(m,n)
    Sigma^M_ab(tau)  = -U_{-1}^2 G^M_ab(tau)^2 G^M_ba(-tau),  G^M(-tau) = xi G^M(beta - tau)
The Matsubara sign follows from Sigma(-i tau, 0) with C^M(tau) = -i C(-i tau, 0)
(Eq. matsconv); the individually printed bubble Matsubara rules are not used.

Hartree (Sec. "Hubbard chain", mean-field Hamiltonian):
    eps^MF_n = eps^(0)_n + U_n diag(n_i - nbar),  n_i = Re rho_ii,
    rho(t) = -i G^<(t,t) for n >= 0 and rho = -G^M(beta^-) for n = -1.
k-point reduction (Sec. "GW for the translationally invariant Hubbard model"):
    G_loc = (1/N_k) sum_k G_k.
"""
import numpy as np

from .contour import Herm, dag


def sigma_2b(n, G, U, S):
    """Fill slice n (n = -1: Matsubara) of S from the local G; U is a scalar Func."""
    xi, T = G.sig, G.ntau
    u = lambda t: U(t)[0, 0]
    if n == -1:
        for m in range(T + 1):
            Gneg = xi * G.mat[T - m]
            S.mat[m] = -u(-1) ** 2 * G.mat[m] ** 2 * Gneg.T
        return
    for j in range(n + 1):
        g_les_jn = G.les[j, n]
        g_gtr_nj = G.ret[n, j] + (-dag(G.les[j, n]))   # G^>(n,j) = G^R + G^<(n,j)
        g_les_nj = -dag(G.les[j, n])
        g_gtr_jn = -dag(g_gtr_nj)                        # G^>(j,n) = -[G^>(n,j)]^dagger
        s_gtr_nj = u(n) * u(j) * g_gtr_nj ** 2 * g_les_jn.T
        s_les_nj = u(n) * u(j) * g_les_nj ** 2 * g_gtr_jn.T
        S.ret[n, j] = s_gtr_nj - s_les_nj
        S.les[j, n] = u(j) * u(n) * g_les_jn ** 2 * g_gtr_nj.T
    for m in range(T + 1):
        gvt = -xi * dag(G.tv[n, T - m])                   # G^vt(tau_m, t_n)
        S.tv[n, m] = u(n) * u(-1) * G.tv[n, m] ** 2 * gvt.T


def density_matrix(n, G):
    """rho(t_n) = -i G^<(t_n,t_n) (n >= 0); rho = -G^M(beta^-) for n = -1."""
    if n == -1:
        return -G.mat[G.ntau]
    return -1j * G.les[n, n]


def hartree(n, rho, eps0, U, nbar):
    """eps^MF_n = eps^(0)_n + U_n diag(Re rho_ii - nbar)."""
    d = rho.shape[0]
    return eps0 + U(n)[0, 0] * np.diag(np.real(np.diag(rho)) - nbar) * np.eye(d)


def kreduce(n, Gks, Gloc):
    """Slice n of G_loc = (1/N_k) sum_k G_k, summed in k order."""
    nk = len(Gks)
    if n == -1:
        acc = np.zeros_like(Gloc.mat)
        for Gk in Gks:
            acc = acc + Gk.mat
        Gloc.mat[...] = acc / nk
        return
    r = np.zeros_like(Gloc.ret[n, :n + 1])
    l = np.zeros_like(Gloc.les[:n + 1, n])
    t = np.zeros_like(Gloc.tv[n])
    for Gk in Gks:
        r = r + Gk.ret[n, :n + 1]
        l = l + Gk.les[:n + 1, n]
        t = t + Gk.tv[n]
    Gloc.ret[n, :n + 1] = r / nk
    Gloc.les[:n + 1, n] = l / nk
    Gloc.tv[n] = t / nk
