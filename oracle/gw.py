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
