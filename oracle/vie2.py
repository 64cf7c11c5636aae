"""Dyson equation in integral form, (1 + F) * G = Q (oracle; test infrastructure only).

Sec. "vie2: Dyson equation in integral form" (Eq. vie2, conjugate Eq. vie2_cc) and
Sec. "Implementation: vie2": the Langreth rules (Eqs. vie2_langreth_m/_r/_tv/_les) turn the
equation into Volterra integral equations of the second kind, solved with the k-th order
start-up (Eq. MBCVSAMx01_start) and time stepping (Eq. MBCVSAMx01_t, and Eq. MBCVSAMx01_cc)t
for the conjugate form) of Sec. "Volterra Integral equation of the second kind".  F is a
given kernel with its hermitian partner Fcc = F^ddagger, Q a hermitian source; G is hermitian
when F * Q = Q * F^ddagger (Eq. ,masbX,.).

Readings (listed with the others in the design notes):
  * ret start-up matrix M_{n,l} = delta_{nl} + h I_{m,n;l} F~^R_{n,l} (the printed "epsilon_n"
    is the identity of the integral equation).
  * ret time step for n - m <= k: the quadrature of Eq. cr1 over the k+1 points n, n-1, ..,
    n-k with the start-up weights s_{n-m,j}; the unknown G^R(n,m) is its j = 0 term, the other
    terms are known (earlier rows, continued by -[G^R(m, n-j)]^dagger), so every m < n is an
    explicit single step; the printed "+" before the sum is the "-" of the integral equation.
  * les, mixed schedule: G^<(0,n) from Eq. vie2_ini_les; the conjugate single steps (B) for
    m = 1..n-1, then m = n, whose history needs G^<(n, n-1) = -[G^<(n-1, n)]^dagger.
  * les, serial schedule (A): start-up for m = 1..k, then single steps m = k+1..n.
"""
import numpy as np

from . import conv, dyson
from .contour import dag


def _retx(X, Xcc, n, j):
    return conv.retx(X, Xcc, n, j)


def _solve_left(M, rhs):
    return np.linalg.solve(M, rhs)


def _solve_right(rhs, M):
    """x with x M = rhs."""
    return np.linalg.solve(M.T, rhs.T).T


# ---- Matsubara (Eq. vie2_langreth_m) ------------------------------------------------------
def vie2_mat(G, F, Q, beta, W):
    """G^M + [F * G]^M = Q^M: the k-th order discretised equation (Eqs. cm1, cm2) solved
    exactly by a dense linear solve, (I + A_F) G = Q."""
    T, d = G.ntau, G.d
    A = dyson.mat_operator(F.mat, W, beta, G.sig)
    big = np.eye((T + 1) * d, dtype=complex) + A.transpose(0, 2, 1, 3).reshape((T + 1) * d, (T + 1) * d)
    G.mat[...] = np.linalg.solve(big, Q.mat.reshape((T + 1) * d, d)).reshape(T + 1, d, d)


# ---- sources of the tv and les equations -----------------------------------------------------
def q_tv(G, F, Q, n, m, W, beta):
    """Q^tv(n,m) - (C^tv_2 + C^tv_3)[F, 1, G^M](n, m) (Eq. map_vie_tv)."""
    return Q.tv[n, m] - conv.ctv2(F, None, G, n, m, W, beta) - conv.ctv3(F, None, G, n, m, W, beta)


def q_les_A(G, F, Fcc, Q, m, n, W, h, beta):
    """Q^<(m,n) - (C^<_2 + C^<_3)[F, 1, G](m, n) (Eq. map_les_vie2); for m > n (start-up rows
    beyond the column) Q^<(m,n) = -[Q^<(n,m)]^dagger."""
    return (conv.lesx(Q, Q, m, n) - conv.cles2(F, Fcc, None, G, G, m, n, W, h)
            - conv.cles3(F, Fcc, None, G, G, m, n, W, beta))


def q_les_B(G, F, Fcc, Q, m, n, W, h, beta):
    """Q^<(m,n) - (C^<_1 + C^<_3)[G, 1, F^ddagger](m, n), the source of the conjugate equation."""
    return (Q.les[m, n] - conv.cles1(G, G, None, Fcc, F, m, n, W, h)
            - conv.cles3(G, G, None, Fcc, F, m, n, W, beta))


def start_matrix(F, Fcc, h, W, d):
    """M_{n,l} = delta_{nl} + h s_{n,l} F~^R(n,l), n = 1..k, l = 0..k (Eq. MBCVSAMx01_start with
    the kernel F^R continued to l > n)."""
    k = W.k
    M = np.zeros((k + 1, k + 1, d, d), complex)
    for n in range(1, k + 1):
        s = W.w(n)
        for l in range(k + 1):
            M[n, l] = h * s[l] * _retx(F, Fcc, n, l)
            if l == n:
                M[n, l] += np.eye(d)
    return M


# ---- start-up, slices 0..k ----------------------------------------------------------------
def vie2_start(G, F, Fcc, Q, beta, h, W):
    k, T, d, xi = W.k, G.ntau, G.d, G.sig
    I = np.eye(d)
    # retarded: column systems (Eq. vie2_langreth_r with the continuation of Eq. y_to_GR)
    for m in range(k + 1):
        y = np.zeros((k + 1, d, d), complex)
        for l in range(m):
            y[l] = -dag(G.ret[m, l])
        y[m] = Q.ret[m, m]
        if m < k:
            Mf = np.zeros((k + 1, k + 1, d, d), complex)
            for n in range(m + 1, k + 1):
                for l in range(k + 1):
                    Mf[n, l] = h * W.I[m, n][l] * _retx(F, Fcc, n, l)
                    if l == n:
                        Mf[n, l] += I
            rhs = np.zeros((k - m, d, d), complex)
            for n in range(m + 1, k + 1):
                rhs[n - m - 1] = Q.ret[n, m]
                for l in range(m + 1):
                    rhs[n - m - 1] -= Mf[n, l] @ y[l]
            y[m + 1:] = dyson._solve_blocks(Mf[m + 1:, m + 1:], rhs)
        for n in range(m, k + 1):
            G.ret[n, m] = y[n]
    # left-mixing: one VIE start-up per tau_m, y_0 = i xi G^M(beta - tau_m) (Eq. vie2_ini_tv)
    M = start_matrix(F, Fcc, h, W, d)
    for m in range(T + 1):
        y0 = 1j * xi * G.mat[T - m]
        rhs = np.stack([q_tv(G, F, Q, n, m, W, beta) - M[n, 0] @ y0 for n in range(1, k + 1)])
        G.tv[0, m] = y0
        G.tv[1:k + 1, m] = dyson._solve_blocks(M[1:, 1:], rhs)
    # lesser: one VIE start-up per column n, y_0 = -[G^tv(n, 0)]^dagger (Eq. vie2_ini_les)
    for n in range(k + 1):
        y0 = -dag(G.tv[n, 0])
        rhs = np.stack([q_les_A(G, F, Fcc, Q, m, n, W, h, beta) - M[m, 0] @ y0 for m in range(1, k + 1)])
        sol = dyson._solve_blocks(M[1:, 1:], rhs)
        G.les[0, n] = y0
        for m in range(1, n + 1):
            G.les[m, n] = sol[m - 1]


# ---- time step n > k ----------------------------------------------------------------------
def ret_row(G, F, Q, h, W, n):
    """G^R(n,n) = Q^R(n,n) (Eq. vie2_ini_r) and the single steps for m < n."""
    k, d = W.k, G.d
    I = np.eye(d)
    G.ret[n, n] = Q.ret[n, n]
    for m in range(n):
        L = n - m
        if L > k:
            w = W.w(L)
            acc = Q.ret[n, m].copy()
            for j in range(m, n):
                acc -= h * w[j - m] * F.ret[n, j] @ G.ret[j, m]
            Mn = I + h * w[L] * F.ret[n, n]
        else:
            s = W.w(L)
            acc = Q.ret[n, m].copy()
            for j in range(1, k + 1):
                acc -= h * s[j] * F.ret[n, n - j] @ _retx(G, G, n - j, m)
            Mn = I + h * s[0] * F.ret[n, n]
        G.ret[n, m] = _solve_left(Mn, acc)


def tv_row(G, F, Q, h, beta, W, n):
    d = G.d
    w = W.w(n)
    Mn = np.eye(d) + h * w[n] * F.ret[n, n]
    for m in range(G.ntau + 1):
        acc = q_tv(G, F, Q, n, m, W, beta)
        for j in range(n):
            acc = acc - h * w[j] * F.ret[n, j] @ G.tv[j, m]
        G.tv[n, m] = _solve_left(Mn, acc)


def les_col_A(G, F, Fcc, Q, h, beta, W, n):
    """Standard VIE along column n in the first argument: start-up m = 1..k, steps m = k+1..n."""
    k, d = W.k, G.d
    G.les[0, n] = -dag(G.tv[n, 0])
    M = start_matrix(F, Fcc, h, W, d)
    y0 = G.les[0, n]
    rhs = np.stack([q_les_A(G, F, Fcc, Q, m, n, W, h, beta) - M[m, 0] @ y0 for m in range(1, k + 1)])
    sol = dyson._solve_blocks(M[1:, 1:], rhs)
    for m in range(1, k + 1):
        G.les[m, n] = sol[m - 1]
    for m in range(k + 1, n + 1):
        w = W.w(m)
        acc = q_les_A(G, F, Fcc, Q, m, n, W, h, beta)
        for l in range(m):
            acc = acc - h * w[l] * F.ret[m, l] @ G.les[l, n]
        G.les[m, n] = _solve_left(np.eye(d) + h * w[m] * F.ret[m, m], acc)


def les_col_B(G, F, Fcc, Q, h, beta, W, n):
    """Conjugate single steps in the second argument (kernel F^ddagger,A(l,n) =
    [F^R(n,l)]^dagger): m = 1..n-1, then m = n; G^<(0,n) from Eq. vie2_ini_les."""
    d = G.d
    w = W.w(n)
    G.les[0, n] = -dag(G.tv[n, 0])
    Mn = np.eye(d) + h * w[n] * dag(F.ret[n, n])
    for m in list(range(1, n)) + [n]:
        acc = q_les_B(G, F, Fcc, Q, m, n, W, h, beta)
        for l in range(n):
            Gml = G.les[m, l] if m <= l else -dag(G.les[l, m])
            acc = acc - h * w[l] * Gml @ dag(F.ret[n, l])
        G.les[m, n] = _solve_right(acc, Mn)


def vie2_timestep(n, G, F, Fcc, Q, beta, h, W, schedule="mixed"):
    """Slice n > k from slices < n: ret row, tv row, then the les column."""
    if n <= W.k:
        raise ValueError("vie2_timestep needs n > k")
    ret_row(G, F, Q, h, W, n)
    tv_row(G, F, Q, h, beta, W, n)
    if schedule == "serial":
        les_col_A(G, F, Fcc, Q, h, beta, W, n)
    elif schedule == "mixed":
        les_col_B(G, F, Fcc, Q, h, beta, W, n)
    else:
        raise ValueError(schedule)


def solve_vie2(G, F, Fcc, Q, beta, h, W, schedule="mixed", n_to=None):
    """vie2_mat, vie2_start, then vie2_timestep for n = k+1..n_to (the three-step procedure of
    Sec. "Test of accuracy and scaling analysis")."""
    vie2_mat(G, F, Q, beta, W)
    vie2_start(G, F, Fcc, Q, beta, h, W)
    for n in range(W.k + 1, (G.nt if n_to is None else n_to) + 1):
        vie2_timestep(n, G, F, Fcc, Q, beta, h, W, schedule)
