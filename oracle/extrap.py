"""Polynomial extrapolation of a time slice and the slice distance (oracle).

Appendix "Contour function utilities":
  * extrapolate_timestep (Eq. polyextrap): y_{n+1} = sum_l C_l y_{n-l}, applied
      - to G^tv(t, tau_m) for every m,
      - to G~^R(t, jh) (modified retarded continuation) for columns j = 0..k, and along
        diagonals y(t) = G^R(t, t - jh) for the remaining points,
      - to G^<(jh, t) (hermitian continuation for t < jh) for rows j = 0..k, and along
        diagonals y(t) = G^<(t - (n+1-j)h, t) for j = k+1..n+1.
  * distance_norm2 (Eq. distancenorm): sum of absolute differences of one slice.
"""
import numpy as np

from .contour import dag


def extrapolate_timestep(n, G, W):
    """Fill slice n+1 of G from slices n-k..n (requires n >= k)."""
    k, C = W.k, W.C
    N1 = n + 1
    G.tv[N1] = sum(C[l] * G.tv[n - l] for l in range(k + 1))
    for j in range(k + 1):
        G.ret[N1, j] = sum(C[l] * (G.ret[n - l, j] if j <= n - l else -dag(G.ret[j, n - l]))
                           for l in range(k + 1))
        G.les[j, N1] = sum(C[l] * (G.les[j, n - l] if j <= n - l else -dag(G.les[n - l, j]))
                           for l in range(k + 1))
    for jd in range(0, N1 - k):           # G^R(n+1, n+1-jd) along the diagonal t - t' = jd h
        G.ret[N1, N1 - jd] = sum(C[l] * G.ret[n - l, n - l - jd] for l in range(k + 1))
    for j in range(k + 1, N1 + 1):        # G^<(j, n+1) along the diagonal t' - t = (n+1-j) h
        off = N1 - j
        G.les[j, N1] = sum(C[l] * G.les[n - l - off, n - l] for l in range(k + 1))


def distance_norm2(n, A, B):
    """||A - B||_n of Eq. distancenorm (n = -1: Matsubara)."""
    if n == -1:
        return float(np.abs(A.mat - B.mat).sum())
    return float(np.abs(A.tv[n] - B.tv[n]).sum() + np.abs(A.ret[n, :n + 1] - B.ret[n, :n + 1]).sum()
                 + np.abs(A.les[:n + 1, n] - B.les[:n + 1, n]).sum())
