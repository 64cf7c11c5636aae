"""Dyson equation in integro-differential form on the L-shaped contour (oracle).

Sec. "Implementation: dyson".  The equation (Eq. dyson)
    i d/dt G - eps(t) G - Sigma * G = delta_C
is split by the Langreth rules (Eqs. dyson_langreth_m/_r/_tv/_les and the conjugate
forms _r_cc/_les_cc) into Volterra integro-differential equations (VIDEs) that are solved
with the k-th order start-up (Eq. vdiff_start, MBCVSAMx_cc_start) and time-stepping
(Eqs. MBCVSAMx_t, MBCVSAMx_cc_t) rules.  The chemical potential enters as eps - mu.

Readings of garbled or ambiguous passages (listed with the others in the design notes):
  * ret start-up matrix: M_{n,l} = i D_{n,l}/h - delta_{nl}(eps_n - mu) - h I_{m,n;l} Sigma~^R_{n,l}
    (the printed +delta eps_n contradicts Eq. dyson_langreth_r).
  * les, implementation (B): kernel k(s,t) = -i Sigma^A(s,t) = -i [Sigma^R(t,s)]^dagger,
    p = -i(eps - mu), source q = i (C^<_1 + C^<_3)[G,1,Sigma](m,n), derived from
    Eq. dyson_langreth_les_cc whose printed source and kernel terms are swapped.
  * les, mixed schedule: G^<(0,n) from Eq. dyson_ini_les; (B) for 1 <= m <= n-k-1, then
    the serial VIDE steps (A) for m = n-k..n.  For n <= 2k the whole column uses (A)
    (start-up for m = 1..k, then steps), because (A) time steps need m > k.
  * ret, mixed schedule: (B) single steps for 0 <= m <= n-k-1; (A) start-up for m = n-k..n.
  * Matsubara: the exact root of the k-th order discretised Eq. Gmat_dyson_integ is found
    by a dense linear solve, the fixed point of the paper's Newton iteration.

Conventions: Herm/Func containers of oracle.contour; W = oracle.weights.Weights(k);
xi = G.sig.  G and Sigma are hermitian symmetric.
"""
import numpy as np

from . import conv
from .contour import dag
from .freegf import _fermi_terms


def _p(eps, mu, n, d):
    return 1j * (eps(n) - mu * np.eye(d))


def _sigR(S, n, j):
    """Sigma^R(n,j), with the modified retarded continuation for j > n (Eq. Cretmod)."""
    return conv.retx(S, S, n, j)


# ==================================================================================
# Matsubara
# ==================================================================================
def g_mat(eps_m1, mu, beta, ntau, xi=-1):
    """g^M(tau_m) solving the Matsubara Dyson equation with Sigma = 0:
    g^M(tau) = -R diag{(1 + xi f(e_a)) exp(-e_a tau)} R^dagger, e_a eigenvalues of eps(0^-) - mu."""
    ev, R = np.linalg.eigh(np.asarray(eps_m1))
    e = ev - mu
    htau = beta / ntau
    out = np.zeros((ntau + 1,) + R.shape, complex)
    for m in range(ntau + 1):
        g = np.array([_fermi_terms(x, beta, m * htau, xi)[0] for x in e])
        out[m] = -(R * g) @ R.conj().T
    return out


def mat_operator(K, W, beta, xi):
    """Dense matrix A of the linear map X -> C^M_1[K,1,X] + C^M_2[K,1,X] (Eqs. cm1, cm2),
    acting on the stacked unknowns X_l (l = 0..T) column by column: (A X)_m = sum_l A_{m,l} X_l."""
    T = K.shape[0] - 1
    d = K.shape[1]
    k = W.k
    ht = beta / T
    A = np.zeros((T + 1, T + 1, d, d), complex)
    for m in range(T + 1):
        # C^M_1: int_0^{tau_m}
        if m <= k:
            Rm = W.R(m)
            for j in range(k + 1):
                for l in range(k + 1):
                    A[m, l] += ht * Rm[j, l] * K[j]
        else:
            w = W.w(m)
            for l in range(m + 1):
                A[m, l] += ht * w[l] * K[m - l]
        # C^M_2: int_{tau_m}^beta
        if m >= T - k:
            Rm = W.R(T - m)
            for j in range(k + 1):
                for l in range(k + 1):
                    A[m, T - l] += ht * Rm[j, l] * xi * K[T - j]
        else:
            w = W.w(T - m)
            for l in range(T - m + 1):
                A[m, m + l] += ht * w[l] * xi * K[T - l]
    return A


def dyson_mat(G, S, eps, mu, beta, W):
    """Matsubara slice: solve G^M = g^M + [K * G]^M, K = [g * Sigma]^M (Eq. Gmat_dyson_integ)."""
    T, d, xi = G.ntau, G.d, G.sig
    g = g_mat(eps(-1), mu, beta, T, xi)

    class _M:  # minimal Matsubara-only view for conv.cmat1/2
        def __init__(self, mat):
            self.mat, self.ntau, self.d, self.sig = mat, T, d, xi
    gv, Sv = _M(g), _M(S.mat)
    K = np.stack([conv.cmat1(gv, None, Sv, m, W, beta) + conv.cmat2(gv, None, Sv, m, W, beta)
                  for m in range(T + 1)])
    A = mat_operator(K, W, beta, xi)
    big = np.eye((T + 1) * d, dtype=complex) - A.transpose(0, 2, 1, 3).reshape((T + 1) * d, (T + 1) * d)
    rhs = g.reshape((T + 1) * d, d)
    G.mat[...] = np.linalg.solve(big, rhs).reshape(T + 1, d, d)


# ==================================================================================
# Sources built from the convolution pieces
# ==================================================================================
def q_tv(G, S, n, m, W, beta):
    """q = -i (C^tv_2 + C^tv_3)[Sigma, 1, G^M](n, m)."""
    return -1j * (conv.ctv2(S, None, G, n, m, W, beta) + conv.ctv3(S, None, G, n, m, W, beta))


def q_les_A(G, S, m, n, W, h, beta):
    """Source of the standard les VIDE: -i (C^<_2 + C^<_3)[Sigma, 1, G](m, n)."""
    return -1j * (conv.cles2(S, S, None, G, G, m, n, W, h) + conv.cles3(S, S, None, G, G, m, n, W, beta))


def q_les_B(G, S, m, n, W, h, beta):
    """Source of the conjugate les VIDE: i (C^<_1 + C^<_3)[G, 1, Sigma](m, n)."""
    return 1j * (conv.cles1(G, G, None, S, S, m, n, W, h) + conv.cles3(G, G, None, S, S, m, n, W, beta))


# ==================================================================================
# Generic VIDE start-up solves (Eq. vdiff_start and its conjugate, Eq. MBCVSAMx_cc_start)
# ==================================================================================
def _solve_blocks(Mblk, rhs):
    """Solve sum_l Mblk[n,l] y_l = rhs_n for block matrices (left multiplication)."""
    kk, _, d, _ = Mblk.shape
    big = Mblk.transpose(0, 2, 1, 3).reshape(kk * d, kk * d)
    return np.linalg.solve(big, rhs.reshape(kk * d, -1)).reshape(kk, d, -1)


def _solve_blocks_right(Mblk, rhs):
    """Solve sum_l y_l Mblk[l,n] = rhs_n (right multiplication) via the transpose."""
    MT = np.swapaxes(np.swapaxes(Mblk, 0, 1), 2, 3)       # (M^T)[n,l] = (M[l,n])^T
    rT = np.swapaxes(rhs, 1, 2)
    y = _solve_blocks(MT, rT)
    return np.swapaxes(y, 1, 2)


def vide_start_matrix(S, eps, mu, h, W, d):
    """M_{n,l} = D_{n,l}/h + delta_{nl} p_n + h s_{n,l} k_{n,l}, n = 1..k, l = 0..k, with
    p = i(eps - mu) and k(t,s) = i Sigma^R(t,s) (continued to s > t); shared by the tv and les
    start-up (Eq. vdiff_start)."""
    k = W.k
    M = np.zeros((k + 1, k + 1, d, d), complex)
    for n in range(1, k + 1):
        s = W.w(n)
        for l in range(k + 1):
            M[n, l] = W.D[n, l] / h * np.eye(d) + h * s[l] * 1j * _sigR(S, n, l)
            if l == n:
                M[n, l] += _p(eps, mu, n, d)
    return M


# ==================================================================================
# Start-up slices n = 0..k (Sec. "Start")
# ==================================================================================
def dyson_start(G, S, eps, mu, beta, h, W):
    k, T, d, xi = W.k, G.ntau, G.d, G.sig
    I = np.eye(d)
    # ---- retarded: column systems for m = 0..k --------------------------------------
    for m in range(k + 1):
        y = np.zeros((k + 1, d, d), complex)
        for l in range(m):
            y[l] = -dag(G.ret[m, l])
        y[m] = -1j * I
        if m < k:
            Mfull = np.zeros((k + 1, k + 1, d, d), complex)
            for n in range(m + 1, k + 1):
                Imn = W.I[m, n]
                for l in range(k + 1):
                    Mfull[n, l] = 1j * W.D[n, l] / h * I - h * Imn[l] * _sigR(S, n, l)
                    if l == n:
                        Mfull[n, l] -= eps(n) - mu * I
            rhs = np.zeros((k - m, d, d), complex)
            for n in range(m + 1, k + 1):
                for l in range(m + 1):
                    rhs[n - m - 1] -= Mfull[n, l] @ y[l]
            sol = _solve_blocks(Mfull[m + 1:, m + 1:], rhs)
            y[m + 1:] = sol
        for n in range(m, k + 1):
            G.ret[n, m] = y[n]
    # ---- left-mixing: VIDE start-up per tau_m --------------------------------------
    M = vide_start_matrix(S, eps, mu, h, W, d)
    for m in range(T + 1):
        y0 = 1j * xi * G.mat[T - m]
        rhs = np.stack([q_tv(G, S, n, m, W, beta) - M[n, 0] @ y0 for n in range(1, k + 1)])
        sol = _solve_blocks(M[1:, 1:], rhs)
        G.tv[0, m] = y0
        G.tv[1:k + 1, m] = sol
    # ---- lesser: VIDE start-up per column n ----------------------------------------
    for n in range(k + 1):
        y0 = -dag(G.tv[n, 0])
        rhs = np.stack([q_les_A(G, S, m, n, W, h, beta) - M[m, 0] @ y0 for m in range(1, k + 1)])
        sol = _solve_blocks(M[1:, 1:], rhs)
        G.les[0, n] = y0
        for m in range(1, n + 1):
            G.les[m, n] = sol[m - 1]


# ==================================================================================
# Time step n > k (Sec. "Time stepping")
# ==================================================================================
def step_matrix(S, eps, mu, h, W, n, d):
    """M_n = a_0/h + i(eps_n - mu) + h w_{n,n} i Sigma^R(n,n) (Eq. MBCVSAMx_t, w_{n,n} = omega_0)."""
    return W.a[0] / h * np.eye(d) + _p(eps, mu, n, d) + h * W.w(n)[n] * 1j * S.ret[n, n]


def ret_row_A(G, S, eps, mu, h, W, n, full):
    """Conjugate VIDE along row n: y_j = G^R(n, n-j), p_j = i(eps_{n-j} - mu),
    kernel k_{l,j} = i Sigma^R(n-l, n-j), y_0 = -i (Eq. dyson_langreth_r_cc).
    Start-up for j = 1..k; if ``full`` the time steps j = k+1..n follow (serial schedule)."""
    k, d = W.k, G.d
    I = np.eye(d)
    y = np.zeros((n + 1, d, d), complex)
    y[0] = -1j * I
    kern = lambda l, j: 1j * _sigR(S, n - l, n - j)
    # start-up: sum_{l=1..k} y_l Mh[l,j] = -y_0 Mh[0,j], Mh[l,j] = D_{j,l}/h + delta p_j + h s_{j,l} k_{l,j}
    Mh = np.zeros((k + 1, k + 1, d, d), complex)
    for j in range(1, k + 1):
        s = W.w(j)
        for l in range(k + 1):
            Mh[l, j] = W.D[j, l] / h * I + h * s[l] * kern(l, j)
            if l == j:
                Mh[l, j] += _p(eps, mu, n - j, d)
    rhs = np.stack([-y[0] @ Mh[0, j] for j in range(1, k + 1)])
    y[1:k + 1] = _solve_blocks_right(Mh[1:, 1:], rhs)
    if full:
        for j in range(k + 1, n + 1):
            w = W.w(j)
            acc = np.zeros((d, d), complex)
            for l in range(1, k + 1):
                acc -= W.a[l] / h * y[j - l]
            for l in range(j):
                acc -= h * w[l] * y[l] @ kern(l, j)
            Mj = W.a[0] / h * I + _p(eps, mu, n - j, d) + h * w[j] * kern(j, j)
            y[j] = acc @ np.linalg.inv(Mj)
        jmax = n
    else:
        jmax = k
    for j in range(jmax + 1):
        G.ret[n, n - j] = y[j]


def ret_bulk_B(G, S, eps, mu, h, W, n, Mn_inv):
    """Standard VIDE single steps for 0 <= m <= n-k-1 (Eq. dyson_langreth_r, implementation (B))."""
    k, d = W.k, G.d
    for m in range(n - k):
        w = W.w(n - m)
        acc = np.zeros((d, d), complex)
        for l in range(1, k + 1):
            acc -= W.a[l] / h * G.ret[n - l, m]
        ls = np.arange(n - m)
        acc -= h * np.einsum("l,lab,lbc->ac", w[:n - m], 1j * S.ret[n, m + ls], G.ret[m + ls, m])
        G.ret[n, m] = Mn_inv @ acc


def tv_row(G, S, eps, mu, h, beta, W, n, Mn_inv):
    """Standard VIDE single step for every tau_m (Eq. dyson_langreth_tv)."""
    k, T = W.k, G.ntau
    w = W.w(n)
    js = np.arange(n)
    for m in range(T + 1):
        acc = q_tv(G, S, n, m, W, beta)
        for l in range(1, k + 1):
            acc = acc - W.a[l] / h * G.tv[n - l, m]
        acc = acc - h * np.einsum("j,jab,jbc->ac", w[:n], 1j * S.ret[n, js], G.tv[js, m])
        G.tv[n, m] = Mn_inv @ acc


def les_col_A(G, S, eps, mu, h, beta, W, n, m_from):
    """Standard VIDE along column n in the first time argument (Eq. dyson_langreth_les):
    y_m = G^<(m,n), p = i(eps - mu), kernel i Sigma^R, source -i (C^<_2 + C^<_3)[Sigma,1,G].
    m_from = 1: start-up for m = 1..k then steps to n; m_from > k: steps m_from..n only."""
    k, d = W.k, G.d
    I = np.eye(d)
    G.les[0, n] = -dag(G.tv[n, 0])
    if m_from <= k:
        M = vide_start_matrix(S, eps, mu, h, W, d)
        y0 = G.les[0, n]
        rhs = np.stack([q_les_A(G, S, m, n, W, h, beta) - M[m, 0] @ y0 for m in range(1, k + 1)])
        sol = _solve_blocks(M[1:, 1:], rhs)
        for m in range(1, k + 1):
            G.les[m, n] = sol[m - 1]
        m_from = k + 1
    for m in range(m_from, n + 1):
        w = W.w(m)
        acc = q_les_A(G, S, m, n, W, h, beta)
        for l in range(1, k + 1):
            acc = acc - W.a[l] / h * G.les[m - l, n]
        ls = np.arange(m)
        acc = acc - h * np.einsum("l,lab,lbc->ac", w[:m], 1j * S.ret[m, ls], G.les[ls, n])
        Mm = W.a[0] / h * I + _p(eps, mu, m, d) + h * w[m] * 1j * S.ret[m, m]
        G.les[m, n] = np.linalg.solve(Mm, acc)


def les_bulk_B(G, S, eps, mu, h, beta, W, n, Mn_dag_inv):
    """Conjugate VIDE single steps in the second time argument for 1 <= m <= n-k-1
    (Eq. dyson_langreth_les_cc, implementation (B)): y(t) = G^<(m,t), p = -i(eps - mu),
    kernel k_{l,n} = -i Sigma^A(l,n), source i (C^<_1 + C^<_3)[G,1,Sigma](m,n)."""
    k, d = W.k, G.d
    w = W.w(n)
    for m in range(1, n - k):
        acc = q_les_B(G, S, m, n, W, h, beta)
        for l in range(1, k + 1):
            acc = acc - W.a[l] / h * G.les[m, n - l]
        # G^<(m,l) for l < m from the hermitian conjugate, stored for l >= m (Eq. hermconjg_gtrless)
        Gml = np.concatenate([-dag(G.les[:m, m]), G.les[m, m:n]])
        Sadv = dag(S.ret[n, :n])                                          # Sigma^A(l,n), l < n
        acc = acc - h * np.einsum("l,lab,lbc->ac", w[:n], Gml, -1j * Sadv)
        G.les[m, n] = acc @ Mn_dag_inv


def dyson_timestep(n, G, S, eps, mu, beta, h, W, schedule="mixed"):
    """Compute slice n > k from slices < n: ret row, then tv row, then les column."""
    k, d = W.k, G.d
    if n <= k:
        raise ValueError("dyson_timestep needs n > k")
    Mn = step_matrix(S, eps, mu, h, W, n, d)
    Mn_inv = np.linalg.inv(Mn)
    if schedule == "serial":
        ret_row_A(G, S, eps, mu, h, W, n, full=True)
    elif schedule == "mixed":
        ret_bulk_B(G, S, eps, mu, h, W, n, Mn_inv)
        ret_row_A(G, S, eps, mu, h, W, n, full=False)
    else:
        raise ValueError(schedule)
    tv_row(G, S, eps, mu, h, beta, W, n, Mn_inv)
    if schedule == "serial" or n <= 2 * k:
        les_col_A(G, S, eps, mu, h, beta, W, n, m_from=1)
    else:
        les_bulk_B(G, S, eps, mu, h, beta, W, n, np.linalg.inv(dag(Mn)))
        G.les[0, n] = -dag(G.tv[n, 0])
        les_col_A(G, S, eps, mu, h, beta, W, n, m_from=n - k)
