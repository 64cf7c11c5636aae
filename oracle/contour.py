"""Full-storage contour functions for the oracle (test infrastructure only).

A hermitian-symmetric contour function C is represented by its minimal set
{C^M, C^R, C^<, C^tv} on C[h, N_t, h_tau, N_tau] (Eq. storage_herm):
    mat[m]     = C^M(m h_tau),          m = 0..N_tau
    ret[n, j]  = C^R(n h, j h),         0 <= j <= n   (lower triangle)
    les[j, n]  = C^<(j h, n h),         0 <= j <= n   (upper triangle)
    tv[n, m]   = C^tv(n h, m h_tau)
Each element is a d x d complex matrix.  The oracle keeps full square arrays for
clarity; only the triangles named above carry data.

The accessors reconstruct the other components from the hermitian conjugate
(Eq. hermconjg), with C^ddagger = C for a hermitian-symmetric function:
    C^<(t,t') for t > t'   = -[C^<(t',t)]^dagger                        (Eq. hermconjg_gtrless)
    C^R continued to t<t'  = -[C^R(t',t)]^dagger  (modified retarded, Eq. Cretmod)
    C^A(t,t')              = [C^R(t',t)]^dagger                        (Eq. hermconjg_ret)
    C^vt(tau, t)           = -xi [C^tv(t, beta - tau)]^dagger            (Eq. hermconjg_vt)
    C^>(t,t') for t >= t'  = C^R(t,t') + C^<(t,t')                      (Eq. defretarded)
"""
import numpy as np


def dag(x):
    """Hermitian conjugate of the trailing d x d matrix axes."""
    return np.conj(np.swapaxes(x, -1, -2))


class Herm:
    """Hermitian-symmetric contour function on C[h, nt, h_tau, ntau] with d x d values."""

    def __init__(self, nt, ntau, d, sig=-1):
        self.nt, self.ntau, self.d, self.sig = nt, ntau, d, sig
        self.mat = np.zeros((ntau + 1, d, d), complex)
        self.ret = np.zeros((nt + 1, nt + 1, d, d), complex)
        self.les = np.zeros((nt + 1, nt + 1, d, d), complex)
        self.tv = np.zeros((nt + 1, ntau + 1, d, d), complex)

    def copy(self):
        c = Herm(self.nt, self.ntau, self.d, self.sig)
        for name in ("mat", "ret", "les", "tv"):
            getattr(c, name)[...] = getattr(self, name)
        return c

    # --- accessors (Eq. hermconjg) -------------------------------------------------
    def retx(self, n, j):
        """C^R(n,j) for j <= n; the modified retarded continuation for j > n."""
        return self.ret[n, j] if j <= n else -dag(self.ret[j, n])

    def lesx(self, j, n):
        """C^<(j,n) for any j, n."""
        return self.les[j, n] if j <= n else -dag(self.les[n, j])

    def gtrx(self, n, j):
        """C^>(n,j) for any n, j: C^R + C^< on n >= j, hermitian conjugate otherwise."""
        if n >= j:
            return self.ret[n, j] + self.lesx(n, j)
        return -dag(self.ret[j, n] + self.lesx(j, n))

    def adv(self, j, n):
        """C^A(j,n) = [C^R(n,j)]^dagger (j <= n)."""
        return dag(self.ret[n, j])

    def advx(self, j, n):
        """C^A(j,n) with the modified retarded continuation for j > n."""
        return dag(self.retx(n, j))

    def vt(self, m, n):
        """C^vt(tau_m, t_n) = -xi [C^tv(t_n, beta - tau_m)]^dagger."""
        return -self.sig * dag(self.tv[n, self.ntau - m])

    def matneg(self, m):
        """C^M(-tau_m) = xi C^M(beta - tau_m) (Eq. dyson_ini_m)."""
        return self.sig * self.mat[self.ntau - m]


class Func:
    """Single-time contour function f_n, n = -1..nt; f[n+1] holds f_n (f_{-1} = f(0^-))."""

    def __init__(self, nt, d):
        self.nt, self.d = nt, d
        self.val = np.zeros((nt + 2, d, d), complex)

    def __call__(self, n):
        return self.val[n + 1]

    def set(self, n, x):
        self.val[n + 1] = x
