"""Discrete k-th order contour convolution pieces (oracle; test infrastructure only).

Sec. "Numerical details: convolution integrals on C", Eqs. cm1, cm2, cr1, ctv1-3, cles1-3.
Each function evaluates one piece of C = A * f * B at one point, with A, B given as
hermitian pairs (X, Xcc) where Xcc = X^ddagger supplies the values outside the stored
triangles (Eq. hermconjg).  ``f`` is a single-time function (oracle.contour.Func) or None
for the identity.  W is an oracle.weights.Weights, h the real-time step, beta the inverse
temperature.  Matrix products keep the order A f B.  Inner quadrature sums are written as
one weighted sum of stacked matrix products (numpy einsum), in the order of the formula.
"""
import numpy as np

from .contour import dag


def wsum(w, X, F, Y):
    """sum_l w_l X_l F_l Y_l for stacks X, F, Y of d x d matrices (F may be one matrix)."""
    if F.ndim == 2:
        return np.einsum("l,lab,bc,lcd->ad", w, X, F, Y)
    return np.einsum("l,lab,lbc,lcd->ad", w, X, F, Y)


def fvals(f, js, d):
    """Stack of f_j for the indices js (identity when f is None)."""
    if f is None:
        return np.broadcast_to(np.eye(d, dtype=complex), (len(js), d, d))
    return np.stack([f(j) for j in js])


def fmat(f, d):
    return np.eye(d, dtype=complex) if f is None else f(-1)


# --- accessors with an explicit hermitian conjugate (Eq. hermconjg) ------------------
def retx(X, Xcc, n, j):
    """X^R(n,j); for j > n the modified retarded continuation -[Xcc^R(j,n)]^dagger."""
    return X.ret[n, j] if j <= n else -dag(Xcc.ret[j, n])


def retx_row(X, Xcc, n, js):
    return np.stack([retx(X, Xcc, n, j) for j in js])


def retx_col(X, Xcc, js, m):
    return np.stack([retx(X, Xcc, j, m) for j in js])


def lesx(X, Xcc, j, n):
    """X^<(j,n); for j > n from the conjugate: -[Xcc^<(n,j)]^dagger."""
    return X.les[j, n] if j <= n else -dag(Xcc.les[n, j])


def advx(X, Xcc, j, n):
    """X^A(j,n) = [Xcc^R(n,j)]^dagger, continued to j > n."""
    return dag(retx(Xcc, X, n, j))


def vt(X, Xcc, m, n):
    """X^vt(tau_m, t_n) = -xi [Xcc^tv(t_n, beta - tau_m)]^dagger (Eq. hermconjg_vt)."""
    return -X.sig * dag(Xcc.tv[n, X.ntau - m])


# --- Matsubara (Eqs. cm1, cm2) -------------------------------------------------------
def cmat1(A, f, B, m, W, beta):
    k, T, d = W.k, A.ntau, A.d
    ht = beta / T
    fm = fmat(f, d)
    if m <= k:
        Rm = W.R(m)
        out = np.zeros((d, d), complex)
        for j in range(k + 1):
            for l in range(k + 1):
                out += Rm[j, l] * A.mat[j] @ fm @ B.mat[l]
        return ht * out
    ls = np.arange(m + 1)
    return ht * wsum(W.w(m), A.mat[m - ls], fm, B.mat[ls])


def cmat2(A, f, B, m, W, beta):
    k, T, d, xi = W.k, A.ntau, A.d, A.sig
    ht = beta / T
    fm = fmat(f, d)
    if m >= T - k:
        Rm = W.R(T - m)
        out = np.zeros((d, d), complex)
        for j in range(k + 1):
            for l in range(k + 1):
                out += Rm[j, l] * xi * A.mat[T - j] @ fm @ B.mat[T - l]
        return ht * out
    ls = np.arange(T - m + 1)
    return ht * xi * wsum(W.w(T - m), A.mat[T - ls], fm, B.mat[m + ls])


# --- retarded (Eq. cr1) -------------------------------------------------------------
def cret(A, Acc, f, B, Bcc, n, m, W, h):
    k, d = W.k, A.d
    if n > k and n - m > k:
        js = np.arange(m, n + 1)
        return h * wsum(W.w(n - m), A.ret[n, js], fvals(f, js, d), B.ret[js, m])
    if n > k:
        js = np.arange(k + 1)
        return h * wsum(W.w(n - m)[:k + 1], A.ret[n, n - js], fvals(f, n - js, d),
                        retx_col(B, Bcc, n - js, m))
    js = np.arange(k + 1)
    return h * wsum(W.I[m, n], retx_row(A, Acc, n, js), fvals(f, js, d), retx_col(B, Bcc, js, m))


# --- left-mixing (Eqs. ctv1, ctv2, ctv3) ---------------------------------------------
def ctv1(A, Acc, f, B, n, m, W, h):
    d = A.d
    js = np.arange(max(n, W.k) + 1)
    return h * wsum(W.w(n), retx_row(A, Acc, n, js), fvals(f, js, d), B.tv[js, m])


def ctv2(A, f, B, n, m, W, beta):
    k, T, d, xi = W.k, A.ntau, A.d, A.sig
    ht = beta / T
    fm = fmat(f, d)
    if m <= k:
        Rm = W.R(m)
        out = np.zeros((d, d), complex)
        for j in range(k + 1):
            for l in range(k + 1):
                out += Rm[j, l] * A.tv[n, l] @ fm @ (xi * B.mat[T - j])
        return ht * out
    ls = np.arange(m + 1)
    return ht * xi * wsum(W.w(m), A.tv[n, m - ls], fm, B.mat[T - ls])


def ctv3(A, f, B, n, m, W, beta):
    k, T, d = W.k, A.ntau, A.d
    ht = beta / T
    fm = fmat(f, d)
    if m >= T - k:
        Rm = W.R(T - m)
        out = np.zeros((d, d), complex)
        for j in range(k + 1):
            for l in range(k + 1):
                out += Rm[j, l] * A.tv[n, T - l] @ fm @ B.mat[j]
        return ht * out
    ls = np.arange(T - m + 1)
    return ht * wsum(W.w(T - m), A.tv[n, m + ls], fm, B.mat[ls])


# --- lesser, first index <= second (Eqs. cles1, cles2, cles3) ---------------------------
def cles1(A, Acc, f, B, Bcc, n, m, W, h):
    """int_0^{t_n} A^R(t_n, s) f(s) B^<(s, t_m) ds."""
    d = A.d
    js = np.arange(max(n, W.k) + 1)
    Bl = np.stack([lesx(B, Bcc, j, m) for j in js])
    return h * wsum(W.w(n), retx_row(A, Acc, n, js), fvals(f, js, d), Bl)


def cles2(A, Acc, f, B, Bcc, n, m, W, h):
    """int_0^{t_m} A^<(t_n, s) f(s) B^A(s, t_m) ds."""
    d = A.d
    js = np.arange(max(m, W.k) + 1)
    Al = np.stack([lesx(A, Acc, n, j) for j in js])
    Ba = np.stack([advx(B, Bcc, j, m) for j in js])
    return h * wsum(W.w(m), Al, fvals(f, js, d), Ba)


def cles3(A, Acc, f, B, Bcc, n, m, W, beta):
    """-i int_0^beta A^tv(t_n, tau) f(0^-) B^vt(tau, t_m) dtau."""
    T, d = A.ntau, A.d
    ht = beta / T
    js = np.arange(T + 1)
    Bv = -B.sig * dag(Bcc.tv[m, T - js])
    return -1j * ht * wsum(W.w(T), A.tv[n, js], fmat(f, d), Bv)


# --- full convolution time slice (Sec. "Implementation: convolution") ------------------
def convolution_timestep(n, C, A, Acc, f, B, Bcc, W, beta, h):
    """Fill slice n of C = A * f * B (n = -1: Matsubara only)."""
    if n == -1:
        for m in range(A.ntau + 1):
            C.mat[m] = cmat1(A, f, B, m, W, beta) + cmat2(A, f, B, m, W, beta)
        return
    for m in range(n + 1):
        C.ret[n, m] = cret(A, Acc, f, B, Bcc, n, m, W, h)
    for m in range(A.ntau + 1):
        C.tv[n, m] = (ctv1(A, Acc, f, B, n, m, W, h) + ctv2(A, f, B, n, m, W, beta)
                      + ctv3(A, f, B, n, m, W, beta))
    for m in range(n + 1):
        C.les[m, n] = (cles1(A, Acc, f, B, Bcc, m, n, W, h) + cles2(A, Acc, f, B, Bcc, m, n, W, h)
                       + cles3(A, Acc, f, B, Bcc, m, n, W, beta))
