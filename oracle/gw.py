"""GW self-energy of a real-space cluster with a local interaction (oracle; test infrastructure).

Sec. "Self-energy approximation: GW" (Eq. SigmaGW, Eq. dyson_chi) with the contour products of
Eqs. def_bubble1 (Bubble1) and def_bubble2 (Bubble2), all elementwise in the orbital indices:
    P_ij(t,t')   = -i G_ij(t,t') G_ji(t',t)             polarization, -Bubble1[G, G] (bosonic)
    chi          = P + P * U * chi                      (1 + K) * chi = P, K = -P U, K^ddagger = -U P
    dW_ij(t,t')  = U(t) chi_ij(t,t') U(t')              dynamical part of the screened interaction
    Sigma_ij     = i G_ij(t,t') dW_ij(t,t')             Bubble2[G, dW]
The susceptibility equation is solved with the integral-form Dyson solver (oracle/vie2.py)
for bosonic functions (xi = +1).

Keldysh components of the bubbles (Langreth rules for products):
    Bubble1 C = i A(t,t') B(t',t):  C^<(j,n) = i A^<(j,n) B^>(n,j),  C^R(n,j) = C^>(n,j) - C^<(n,j)
        with C^>(n,j) = i A^>(n,j) B^<(j,n);  C^tv(n,m) = i A^tv(n,m) B^vt(m,n)
    Bubble2 C = i A(t,t') B(t,t'):  C^<(j,n) = i A^<(j,n) B^<(j,n),  C^>(n,j) = i A^>(n,j) B^>(n,j),
        C^tv(n,m) = i A^tv(n,m) B^tv(n,m)
Matsubara component (reading, with C^M(tau) = -i C(-i tau, 0) and A(-i tau, 0) = i A^M(tau),
the convention of Eq. matsconv): Bubble1 C^M(tau) = -A^M(tau) B^M(-tau), B^M(-tau) = xi_B
B^M(beta - tau); Bubble2 C^M(tau) = -A^M(tau) B^M(tau).  The individually printed Matsubara
rules carry the opposite sign; composed as Sigma = -U^2 Bubble2[G, Bubble1[G, G]] they give the
second-Born Sigma^M(tau) = -U^2 G^M(tau)^2 G^M(-tau) of oracle/bubble.py, whose sign the KMS
relation fixes.
"""
import numpy as np

from . import vie2
from .contour import Herm


def bubble1(n, A, B, C):
    """Slice n (n = -1: Matsubara) of C_ij(t,t') = i A_ij(t,t') B_ji(t',t)."""
    T = A.ntau
    if n == -1:
        for m in range(T + 1):
            C.mat[m] = -A.mat[m] * (B.sig * B.mat[T - m]).T
        return
    for j in range(n + 1):
        C.les[j, n] = 1j * A.lesx(j, n) * B.gtrx(n, j).T
        c_gtr = 1j * A.gtrx(n, j) * B.lesx(j, n).T
        c_les = 1j * A.lesx(n, j) * B.gtrx(j, n).T
        C.ret[n, j] = c_gtr - c_les
    for m in range(T + 1):
        C.tv[n, m] = 1j * A.tv[n, m] * B.vt(m, n).T


def bubble2(n, A, B, C):
    """Slice n (n = -1: Matsubara) of C_ij(t,t') = i A_ij(t,t') B_ij(t,t')."""
    T = A.ntau
    if n == -1:
        for m in range(T + 1):
            C.mat[m] = -A.mat[m] * B.mat[m]
        return
    for j in range(n + 1):
        C.les[j, n] = 1j * A.lesx(j, n) * B.lesx(j, n)
        C.ret[n, j] = 1j * A.gtrx(n, j) * B.gtrx(n, j) - 1j * A.lesx(n, j) * B.lesx(n, j)
    for m in range(T + 1):
        C.tv[n, m] = 1j * A.tv[n, m] * B.tv[n, m]


class GW:
    """The GW self-energy chain for a cluster with d orbitals; keeps P, K, K^ddagger, chi and dW
    (bosonic) on the contour of the run."""

    def __init__(self, nt, ntau, d, beta, h, W):
        self.beta, self.h, self.W = beta, h, W
        self.P, self.K, self.Kcc, self.chi, self.dW = (Herm(nt, ntau, d, sig=+1) for _ in range(5))

    def _kernel(self, n, G, U):
        """P, K = -P U(t') and K^ddagger = -U(t) P on slice n."""
        u = lambda t: U(t)[0, 0]
        P, K, Kcc = self.P, self.K, self.Kcc
        bubble1(n, G, G, P)
        if n == -1:
            P.mat *= -1.0
            K.mat[...] = -P.mat * u(-1)
            Kcc.mat[...] = -u(-1) * P.mat
            return
        P.ret[n, :n + 1] *= -1.0
        P.les[:n + 1, n] *= -1.0
        P.tv[n] *= -1.0
        for j in range(n + 1):
            K.ret[n, j] = -P.ret[n, j] * u(j)
            Kcc.ret[n, j] = -u(n) * P.ret[n, j]
            K.les[j, n] = -P.les[j, n] * u(n)
            Kcc.les[j, n] = -u(j) * P.les[j, n]
        K.tv[n] = -P.tv[n] * u(-1)
        Kcc.tv[n] = -u(n) * P.tv[n]

    def _sigma(self, n, G, U, S):
        u = lambda t: U(t)[0, 0]
        chi, dW = self.chi, self.dW
        if n == -1:
            dW.mat[...] = u(-1) * chi.mat * u(-1)
        else:
            for j in range(n + 1):
                dW.ret[n, j] = u(n) * chi.ret[n, j] * u(j)
                dW.les[j, n] = u(j) * chi.les[j, n] * u(n)
            dW.tv[n] = u(n) * chi.tv[n] * u(-1)
        bubble2(n, G, dW, S)

    def mat(self, G, U, S):
        self._kernel(-1, G, U)
        vie2.vie2_mat(self.chi, self.K, self.P, self.beta, self.W)
        self._sigma(-1, G, U, S)

    def start(self, G, U, S):
        k = self.W.k
        for n in range(k + 1):
            self._kernel(n, G, U)
        vie2.vie2_start(self.chi, self.K, self.Kcc, self.P, self.beta, self.h, self.W)
        for n in range(k + 1):
            self._sigma(n, G, U, S)

    def step(self, n, G, U, S):
        self._kernel(n, G, U)
        vie2.vie2_timestep(n, self.chi, self.K, self.Kcc, self.P, self.beta, self.h, self.W)
        self._sigma(n, G, U, S)


def _slice_axpy(n, dst, src, s):
    """dst += s * src on slice n (n = -1: Matsubara)."""
    if n == -1:
        dst.mat += s * src.mat
        return
    dst.ret[n, :n + 1] += s * src.ret[n, :n + 1]
    dst.les[:n + 1, n] += s * src.les[:n + 1, n]
    dst.tv[n] += s * src.tv[n]


def _slice_zero(n, X):
    _slice_axpy(n, X, X, -1.0)


class GWk:
    """GW of a translation-invariant one-band lattice with a local interaction U(t)
    (Sec. "GW for the translationally invariant Hubbard model"), momenta k = 0..N_k-1 of a cyclic
    group with the addition table add[k, q] = index of k + q and neg[q] = index of -q:
        Pi_k(t,t')   = -(i/N_k) sum_q G_{k+q}(t,t') G_q(t',t)          (Eq. Pol)
        chi_k        = Pi_k + Pi_k * U * chi_k,  (1 + K_k) * chi_k = Pi_k, K_k = -Pi_k U(t'),
                       K_k^ddagger = -U(t) Pi_k                        (the local form of Eq. dyson_chi)
        dW_k(t,t')   = U(t) chi_k(t,t') U(t')
        Sigma_k      = (i/N_k) sum_q G_{k-q}(t,t') dW_q(t,t')          (Eq. Sigmak)
    Each product is a Bubble1 / Bubble2 of two momentum components (Eqs. def_bubble1,
    def_bubble2), so Pi_k = -(1/N_k) sum_q Bubble1[G_{k+q}, G_q] and
    Sigma_k = (1/N_k) sum_q Bubble2[G_{k-q}, dW_q].  The driver runs it with kspace = True: the
    Dyson equation of G_k takes Sigma_k."""

    kspace = True

    def __init__(self, nt, ntau, nk, beta, h, W, add, neg):
        self.beta, self.h, self.W, self.nk = beta, h, W, nk
        self.add, self.neg = np.asarray(add), np.asarray(neg)
        mk = lambda: [Herm(nt, ntau, 1, sig=+1) for _ in range(nk)]
        self.P, self.K, self.Kcc, self.chi, self.dW = mk(), mk(), mk(), mk(), mk()
        self._tmpb = Herm(nt, ntau, 1, sig=+1)
        self._tmpf = Herm(nt, ntau, 1)

    def _kernel(self, n, Gk, U):
        u = lambda t: U(t)[0, 0]
        N = self.nk
        for k in range(N):
            P = self.P[k]
            _slice_zero(n, P)
            for q in range(N):
                bubble1(n, Gk[self.add[k, q]], Gk[q], self._tmpb)
                _slice_axpy(n, P, self._tmpb, -1.0 / N)
            K, Kcc = self.K[k], self.Kcc[k]
            if n == -1:
                K.mat[...] = -P.mat * u(-1)
                Kcc.mat[...] = -u(-1) * P.mat
                continue
            for j in range(n + 1):
                K.ret[n, j] = -P.ret[n, j] * u(j)
                Kcc.ret[n, j] = -u(n) * P.ret[n, j]
                K.les[j, n] = -P.les[j, n] * u(n)
                Kcc.les[j, n] = -u(j) * P.les[j, n]
            K.tv[n] = -P.tv[n] * u(-1)
            Kcc.tv[n] = -u(n) * P.tv[n]

    def _sigma(self, n, Gk, U, Sk):
        u = lambda t: U(t)[0, 0]
        N = self.nk
        for q in range(N):
            chi, dW = self.chi[q], self.dW[q]
            if n == -1:
                dW.mat[...] = u(-1) * chi.mat * u(-1)
                continue
            for j in range(n + 1):
                dW.ret[n, j] = u(n) * chi.ret[n, j] * u(j)
                dW.les[j, n] = u(j) * chi.les[j, n] * u(n)
            dW.tv[n] = u(n) * chi.tv[n] * u(-1)
        for k in range(N):
            _slice_zero(n, Sk[k])
            for q in range(N):
                bubble2(n, Gk[self.add[k, self.neg[q]]], self.dW[q], self._tmpf)
                _slice_axpy(n, Sk[k], self._tmpf, 1.0 / N)

    def mat(self, Gk, U, Sk):
        self._kernel(-1, Gk, U)
        for k in range(self.nk):
            vie2.vie2_mat(self.chi[k], self.K[k], self.P[k], self.beta, self.W)
        self._sigma(-1, Gk, U, Sk)

    def start(self, Gk, U, Sk):
        for n in range(self.W.k + 1):
            self._kernel(n, Gk, U)
        for k in range(self.nk):
            vie2.vie2_start(self.chi[k], self.K[k], self.Kcc[k], self.P[k], self.beta, self.h, self.W)
        for n in range(self.W.k + 1):
            self._sigma(n, Gk, U, Sk)

    def step(self, n, Gk, U, Sk):
        self._kernel(n, Gk, U)
        for k in range(self.nk):
            vie2.vie2_timestep(n, self.chi[k], self.K[k], self.Kcc[k], self.P[k], self.beta, self.h, self.W)
        self._sigma(n, Gk, U, Sk)


def ring_tables(nk):
    """Addition and negation tables of the momenta k_m = 2 pi m / N_k of a ring of N_k sites."""
    m = np.arange(nk)
    return (m[:, None] + m[None, :]) % nk, (-m) % nk
