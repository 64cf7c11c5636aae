"""Exact diagonalisation of a small Hubbard cluster: the reference the second-Born and GW
dynamics of the oracle are checked against to second order in U.

Test infrastructure only; it shares nothing with the oracle or the CUDA path.  Fock space of
M sites x 2 spins (2^(2M) states, Jordan-Wigner ordering of the modes p = 2 i + s), dense
matrices:

    H(U) = sum_s sum_ij eps_ij c^+_is c_js + U sum_i (n_iup - nbar)(n_idn - nbar) - mu N,

the interaction written about the reference filling nbar as the oracle's mean-field term
eps^MF = eps + U diag(rho_ii - nbar) assumes.  The initial state is the grand-canonical
ensemble of H(U0) at inverse temperature beta; for t >= 0 the system evolves with H(U1)
(a sudden quench at t = 0).  Spin-up Green's functions (the paramagnetic state is spin
symmetric):

    G^M_ij(tau)  = -<c_i(tau) c^+_j>_0              (0 <= tau < beta, imaginary-time Heisenberg)
    rho_ij(t)    = <c^+_j(t) c_i(t)> = -i G^<_ij(t, t)
    G^<_ij(t, t') = i <c^+_j(t') c_i(t)>
"""
import numpy as np


def fermion_ops(nmodes):
    """Annihilators c_p (dense 2^nmodes square matrices), Jordan-Wigner with mode 0 first."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1| on one mode (basis |0>, |1>)
    z = np.diag([1.0, -1.0])
    eye = np.eye(2)
    ops = []
    for p in range(nmodes):
        m = np.array([[1.0]])
        for q in range(nmodes):
            m = np.kron(m, z if q < p else (a if q == p else eye))
        ops.append(m)
    return ops


class HubbardED:
    def __init__(self, eps, mu=0.0, nbar=0.5):
        eps = np.asarray(eps, dtype=complex)
        self.M = eps.shape[0]
        self.c = fermion_ops(2 * self.M)
        self.eps, self.mu, self.nbar = eps, mu, nbar
        dim = self.c[0].shape[0]
        self.h0 = np.zeros((dim, dim), dtype=complex)
        self.N = np.zeros((dim, dim))
        for s in range(2):
            for i in range(self.M):
                ci = self.c[2 * i + s]
                self.N = self.N + ci.T @ ci
                for j in range(self.M):
                    self.h0 = self.h0 + eps[i, j] * (ci.T @ self.c[2 * j + s])
        self.vint = np.zeros((dim, dim))
        one = np.eye(dim)
        for i in range(self.M):
            nu = self.c[2 * i].T @ self.c[2 * i]
            nd = self.c[2 * i + 1].T @ self.c[2 * i + 1]
            self.vint = self.vint + (nu - nbar * one) @ (nd - nbar * one)

    def hamiltonian(self, U):
        return self.h0 + U * self.vint - self.mu * self.N

    def thermal(self, U0, beta):
        """Eigen-decomposition of H(U0) and the Boltzmann weights."""
        E, V = np.linalg.eigh(self.hamiltonian(U0))
        w = np.exp(-beta * (E - E.min()))
        return E, V, w / w.sum()

    def gmat(self, U0, beta, taus):
        """G^M_ij(tau) for the spin-up modes, shape (len(taus), M, M)."""
        E, V, p = self.thermal(U0, beta)
        cu = [V.conj().T @ self.c[2 * i] @ V for i in range(self.M)]   # eigenbasis
        out = np.zeros((len(taus), self.M, self.M), dtype=complex)
        for t, tau in enumerate(taus):
            # <c_i(tau) c_j^+> = sum_ab p_a e^{tau (E_a - E_b)} (c_i)_ab (c_j^+)_ba
            f = p[:, None] * np.exp(tau * (E[:, None] - E[None, :]))
            for i in range(self.M):
                for j in range(self.M):
                    out[t, i, j] = -np.sum(f * cu[i] * cu[j].conj())   # (c_j^+)_ba = conj (c_j)_ab
        return out

    def _evolved(self, U0, U1, beta, times):
        """Heisenberg spin-up annihilators c_i(t) = e^{i H1 t} c_i e^{-i H1 t} and rho0."""
        E0, V0, p0 = self.thermal(U0, beta)
        rho0 = (V0 * p0) @ V0.conj().T
        E1, V1 = np.linalg.eigh(self.hamiltonian(U1))
        cs = []
        for t in times:
            u = (V1 * np.exp(-1j * E1 * t)) @ V1.conj().T   # e^{-i H1 t}
            cs.append([u.conj().T @ self.c[2 * i] @ u for i in range(self.M)])
        return rho0, cs

    def density(self, U0, U1, beta, times):
        """rho_ij(t) = <c^+_j(t) c_i(t)>, shape (len(times), M, M)."""
        rho0, cs = self._evolved(U0, U1, beta, times)
        out = np.zeros((len(times), self.M, self.M), dtype=complex)
        for t, ct in enumerate(cs):
            for i in range(self.M):
                for j in range(self.M):
                    out[t, i, j] = np.trace(rho0 @ ct[j].conj().T @ ct[i])
        return out

    def gles(self, U0, U1, beta, times):
        """G^<_ij(t_a, t_b) = i <c^+_j(t_b) c_i(t_a)>, shape (T, T, M, M)."""
        rho0, cs = self._evolved(U0, U1, beta, times)
        nT = len(times)
        out = np.zeros((nT, nT, self.M, self.M), dtype=complex)
        for a in range(nT):
            for b in range(nT):
                for i in range(self.M):
                    for j in range(self.M):
                        out[a, b, i, j] = 1j * np.trace(rho0 @ cs[b][j].conj().T @ cs[a][i])
        return out
