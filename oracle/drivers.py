"""Drivers: fixed-Sigma Dyson solve and self-consistent second-Born (oracle).

* solve_fixed_sigma: dyson_mat, dyson_start, then dyson_timestep for n = k+1..N
  (Sec. "Test of accuracy and scaling analysis", generic three-step procedure).
* run_2b: the self-consistent second-Born loop of Sec. "Hubbard chain", generalised to a
  batch of problems (k-points) coupled only through the local Green's function
  G_loc = (1/N_k) sum_k G_k (Sec. "GW for the translationally invariant Hubbard model"):
    1. Matsubara loop: {G_loc, eps^MF, Sigma_2B(-1), dyson_mat} until the distance of
       successive G^M (summed over k) is below mats_tol, at most mats_maxiter times;
    2. bootstrapping: {G_loc, eps^MF, Sigma_2B(0..k), dyson_start} until the summed distance
       of slices 0..k is below boot_tol and more than two iterations were made;
    3. time stepping n = k+1..N: extrapolate_timestep(n-1), then exactly ``corrector``
       iterations of {G_loc(n), eps^MF_n, Sigma_2B(n), dyson_timestep(n)}.
  A problem with N_k = 1 and d = 2 is the Hubbard dimer in real space.
* run_gw: the same loop with the GW self-energy of Sec. "Self-energy approximation: GW"
  (oracle/gw.py) in place of the second-Born one: each Sigma evaluation first builds P, K and
  K^ddagger on its slices, then solves the susceptibility (vie2_mat in the Matsubara loop,
  vie2_start over slices 0..k in the bootstrapping, vie2_timestep(n) in each corrector pass),
  then forms dW and Sigma.
  The second-Born and GW dynamics have no closed form; they are pinned by their conservation
  laws, by their pinned building blocks, and against exact diagonalisation of the Hubbard dimer
  to the order in U at which the approximations are exact (tests/test_oracle_ed.py).
"""
import numpy as np

from . import bubble, dyson, extrap, gw
from .contour import Func, Herm


def solve_fixed_sigma(G, S, eps, mu, beta, h, W, schedule="mixed", nmax=None):
    dyson.dyson_mat(G, S, eps, mu, beta, W)
    dyson.dyson_start(G, S, eps, mu, beta, h, W)
    for n in range(W.k + 1, (G.nt if nmax is None else nmax) + 1):
        dyson.dyson_timestep(n, G, S, eps, mu, beta, h, W, schedule)
    return G


class Sigma2B:
    """Second-Born self-energy slices (Eq. sigma_hubb_2b) for the driver: Matsubara, start-up
    slices 0..k, one time step."""

    def __init__(self, k):
        self.k = k

    def mat(self, Gloc, U, S):
        bubble.sigma_2b(-1, Gloc, U, S)

    def start(self, Gloc, U, S):
        for n in range(self.k + 1):
            bubble.sigma_2b(n, Gloc, U, S)

    def step(self, n, Gloc, U, S):
        bubble.sigma_2b(n, Gloc, U, S)


class TwoBState:
    def __init__(self, nk, nt, ntau, d):
        self.G = [Herm(nt, ntau, d) for _ in range(nk)]
        self.Gloc = Herm(nt, ntau, d)
        self.S = Herm(nt, ntau, d)
        self.epsmf = [Func(nt, d) for _ in range(nk)]
        self.log = {}


def _update_mf(n, st, eps0, U, nbar):
    rho = bubble.density_matrix(n, st.Gloc)
    for kk, e0 in enumerate(eps0):
        st.epsmf[kk].set(n, bubble.hartree(n, rho, e0(n), U, nbar))


def run_2b(eps0, U, nt, ntau, beta, h, W, mu=0.0, nbar=0.5, corrector=3, schedule="mixed",
           mats_tol=1e-12, mats_maxiter=200, boot_tol=1e-12, boot_maxiter=200, nmax=None,
           state=None, sigma=None):
    """Self-consistent second-Born (or, with sigma = gw.GW(...), GW) for the problems with bare
    Hamiltonians eps0[k] (Funcs)."""
    nk = len(eps0)
    d = eps0[0].d
    st = state or TwoBState(nk, nt, ntau, d)
    sig = sigma or Sigma2B(W.k)
    # a momentum-resolved self-energy (k-space GW) acts on all G_k and gives one Sigma_k per
    # problem; the local ones act on Gloc and give the shared Sigma
    if getattr(sig, "kspace", False):
        st.Sk = [Herm(nt, ntau, d) for _ in range(nk)]
        src, dst, S_of = st.G, st.Sk, (lambda kk: st.Sk[kk])
    else:
        src, dst, S_of = st.Gloc, st.S, (lambda kk: st.S)
    # ---- Matsubara -------------------------------------------------------------------
    for kk in range(nk):  # initial guess: free G^M of the bare Hamiltonian
        st.epsmf[kk].set(-1, eps0[kk](-1))
        dyson.dyson_mat(st.G[kk], S_of(kk), st.epsmf[kk], mu, beta, W)
    it_m = 0
    for it_m in range(mats_maxiter):
        bubble.kreduce(-1, st.G, st.Gloc)
        _update_mf(-1, st, eps0, U, nbar)
        sig.mat(src, U, dst)
        err = 0.0
        for kk in range(nk):
            old = st.G[kk].mat.copy()
            dyson.dyson_mat(st.G[kk], S_of(kk), st.epsmf[kk], mu, beta, W)
            err += float(np.abs(st.G[kk].mat - old).sum())
        # a summed distance cannot fall below round-off (about 1e-15 per element)
        if err < max(mats_tol, 1e-15 * nk * (ntau + 1) * d * d):
            break
    st.log["mats_iter"] = it_m + 1
    st.log["mats_err"] = err
    bubble.kreduce(-1, st.G, st.Gloc)
    _update_mf(-1, st, eps0, U, nbar)
    sig.mat(src, U, dst)
    # ---- bootstrapping ---------------------------------------------------------------
    k = W.k
    for n in range(k + 1):  # initial guess for slices 0..k: the equilibrium Matsubara state
        for kk in range(nk):
            st.epsmf[kk].set(n, st.epsmf[kk](-1) - eps0[kk](-1) + eps0[kk](n))
    for kk in range(nk):
        dyson.dyson_start(st.G[kk], S_of(kk), st.epsmf[kk], mu, beta, h, W)
    it_b = 0
    for it_b in range(boot_maxiter):
        for n in range(k + 1):
            bubble.kreduce(n, st.G, st.Gloc)
            _update_mf(n, st, eps0, U, nbar)
        sig.start(src, U, dst)
        err = 0.0
        for kk in range(nk):
            old = st.G[kk].copy()
            dyson.dyson_start(st.G[kk], S_of(kk), st.epsmf[kk], mu, beta, h, W)
            err += sum(extrap.distance_norm2(n, st.G[kk], old) for n in range(k + 1))
        nel_boot = nk * d * d * ((k + 1) * (k + 2) + (k + 1) * (ntau + 1))
        if err < max(boot_tol, 1e-15 * nel_boot) and it_b > 2:
            break
    st.log["boot_iter"] = it_b + 1
    st.log["boot_err"] = err
    # ---- time stepping ---------------------------------------------------------------
    for n in range(k + 1, (nt if nmax is None else nmax) + 1):
        for kk in range(nk):
            extrap.extrapolate_timestep(n - 1, st.G[kk], W)
        for _ in range(corrector):
            bubble.kreduce(n, st.G, st.Gloc)
            _update_mf(n, st, eps0, U, nbar)
            sig.step(n, src, U, dst)
            for kk in range(nk):
                dyson.dyson_timestep(n, st.G[kk], S_of(kk), st.epsmf[kk], mu, beta, h, W, schedule)
    bubble.kreduce(-1, st.G, st.Gloc)
    return st


def run_gw(eps0, U, nt, ntau, beta, h, W, **kw):
    """Self-consistent GW (Eq. SigmaGW, Eq. dyson_chi) for the problems eps0[k]; returns the
    driver state and the GW chain (P, K, K^ddagger, chi, dW of the last evaluation)."""
    chain = gw.GW(nt, ntau, eps0[0].d, beta, h, W)
    st = run_2b(eps0, U, nt, ntau, beta, h, W, sigma=chain, **kw)
    return st, chain


def run_gw_kspace(eps0, U, nt, ntau, beta, h, W, add, neg, **kw):
    """Self-consistent k-space GW (Eqs. Sigmak, Pol) for the one-band problems eps0[k] on the
    momentum group given by the tables add, neg; Sigma_k per k-point (st.Sk)."""
    chain = gw.GWk(nt, ntau, len(eps0), beta, h, W, add, neg)
    st = run_2b(eps0, U, nt, ntau, beta, h, W, sigma=chain, **kw)
    return st, chain
