"""Small oracle problems shared by the CPU pin tests (test helpers; no CUDA)."""
import numpy as np

from oracle import drivers
from oracle.contour import Func, Herm
from oracle.freegf import green_from_H
from oracle.weights import Weights


def embedded_level(N, T, beta, h, k=5, e1=0.5, V=0.3, eb=-0.2, schedule="mixed"):
    """One level e1 coupled to a bath level eb by V, the bath folded in as Sigma = V^2 g0(eb)
    (Sec. "Test of accuracy and scaling analysis", downfolding).  Returns (G, exact G_11, Sigma)."""
    W = Weights(k)
    ex = green_from_H(N, T, np.array([[e1, V], [V, eb]]), 0.0, beta, h)
    S = green_from_H(N, T, np.array([[eb]]), 0.0, beta, h)
    for c in ("mat", "ret", "les", "tv"):
        setattr(S, c, getattr(S, c) * V * V)
    G = Herm(N, T, 1)
    eps = Func(N, 1)
    eps.val[:] = e1
    drivers.solve_fixed_sigma(G, S, eps, 0.0, beta, h, W, schedule=schedule)
    return G, ex, S


def max_err(G, ref, comps=("mat", "ret", "les", "tv"), sub=(slice(0, 1), slice(0, 1))):
    N = G.nt
    out = {}
    for c in comps:
        a = getattr(G, c)
        b = getattr(ref, c)[..., sub[0], sub[1]]
        diff = np.abs(a - b)
        if c == "ret":
            diff = diff[np.tril(np.ones((N + 1, N + 1), bool))]
        if c == "les":
            diff = diff[np.triu(np.ones((N + 1, N + 1), bool))]
        out[c] = float(diff.max())
    return out


def embedded_cluster(d, nbath, N, T, beta, h, seed, k=5, schedule="mixed", vscale=0.4):
    """A d-orbital cluster coupled to an nbath-site bath by a complex d x nbath matrix V; the
    bath folded in as Sigma = V g0_bath V^dagger (downfolding, Sec. "Test of accuracy and scaling
    analysis").  The exact answer is the cluster block of the free GF of the whole
    (d + nbath)-level Hamiltonian [[h_c, V], [V^dagger, h_b]].  Returns (G, exact, Sigma)."""
    rng = np.random.default_rng(seed)

    def herm(n):
        a = rng.normal(0, 1, (n, n)) + 1j * rng.normal(0, 1, (n, n))
        return 0.5 * (a + a.conj().T)

    hc, hb = herm(d), herm(nbath)
    V = vscale * (rng.normal(0, 1, (d, nbath)) + 1j * rng.normal(0, 1, (d, nbath)))
    full = np.block([[hc, V], [V.conj().T, hb]])
    ex = green_from_H(N, T, full, 0.0, beta, h)
    bath = green_from_H(N, T, hb, 0.0, beta, h)
    S = Herm(N, T, d)
    for c in ("mat", "ret", "les", "tv"):
        setattr(S, c, np.einsum("ab,...bc,dc->...ad", V, getattr(bath, c), V.conj()))
    G = Herm(N, T, d)
    eps = Func(N, d)
    eps.val[:] = hc
    drivers.solve_fixed_sigma(G, S, eps, 0.0, beta, h, Weights(k), schedule=schedule)
    return G, ex, S, eps
