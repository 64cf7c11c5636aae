"""Seeded synthetic workloads: model Hamiltonians, interactions and grid parameters.

This module holds inputs only (grid sizes, dispersions, field pulses, interaction
profiles, random draws); none of the solver's arithmetic.  Both the CUDA path and the
CPU oracle take their inputs from here.

Workloads (the paper's example models, Secs. "Test of accuracy and scaling analysis",
"Hubbard chain", "GW for the translationally invariant Hubbard model"):
  embedded_level  one level eps = 0.5 coupled by V = 0.3 to a bath level eps_b = -0.2 folded
                  in as Sigma = V^2 g0(eps_b); beta = 10, ntau = 200, nt = 200, h = 0.025, k = 5
  hubbard_dimer   two sites, hopping J = 1, second-Born, quench U: 1 -> 2 at t = 0;
                  beta = 20, ntau = 400, nt = 1000, h = 0.02, k = 5, 3 corrector iterations
  chain_kspace    1D Hubbard chain in momentum space, nk = 512, eps_k(t) = -2 cos(k - A(t)),
                  A(t) = 0.5 exp(-(t-5)^2 / (2 1.5^2)) sin(2t), local second-Born U = 2;
                  beta = 10, ntau = 800, nt = 2000, h = 0.01, k = 5, 3 corrector iterations
  square_kspace   2D 16 x 16 square lattice, eps_k = -2 cos(kx - A(t)) - 2 cos(ky), U = 1.5;
                  beta = 10, ntau = 400, nt = 1000, h = 0.02, k = 5
Every workload takes size overrides so tests can run the same model on small grids.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    nt: int
    ntau: int
    nf: int
    nbatch: int
    korder: int
    h: float
    beta: float
    mu: float = 0.0
    corrector: int = 3
    nbar: float = 0.5
    eps0: np.ndarray = None       # [nt+2, nf, nf, nbatch] complex, index n+1 holds eps_n
    U: np.ndarray = None          # [nt+2] real, index n+1 holds U_n
    extra: dict = field(default_factory=dict)


def pulse_A(t, A0=0.5, omega=2.0, t0=5.0, sigma=1.5):
    """Vector potential of the Peierls pulse A(t) = A0 exp(-(t-t0)^2/(2 sigma^2)) sin(omega t)."""
    return A0 * np.exp(-((t - t0) ** 2) / (2 * sigma ** 2)) * np.sin(omega * t)


def embedded_level(nt=200, ntau=200, beta=10.0, h=0.025, korder=5, e1=0.5, V=0.3, eb=-0.2):
    eps0 = np.full((nt + 2, 1, 1, 1), e1, dtype=complex)
    w = Workload("embedded_level", nt, ntau, 1, 1, korder, h, beta, corrector=0, eps0=eps0,
                 U=np.zeros(nt + 2))
    w.extra = {"V": V, "eb": eb, "e1": e1}
    return w


def hubbard_dimer(nt=1000, ntau=400, beta=20.0, h=0.02, korder=5, J=1.0, U0=1.0, U1=2.0, corrector=3):
    eps = np.array([[0.0, -J], [-J, 0.0]], dtype=complex)
    eps0 = np.broadcast_to(eps[None, :, :, None], (nt + 2, 2, 2, 1)).copy()
    U = np.full(nt + 2, U1)
    U[0] = U0
    return Workload("hubbard_dimer", nt, ntau, 2, 1, korder, h, beta, corrector=corrector, eps0=eps0, U=U)


def hubbard_chain(M=4, nt=1000, ntau=400, beta=20.0, h=0.02, korder=5, J=1.0, U=1.5, w0=5.0, mu=0.0, nbar=0.5,
                  corrector=3):
    """Open Hubbard chain of M sites in real space (nf = M, one problem), hopping -J between
    neighbours, excited at t = 0 by the quench of the first site's on-site energy to w0
    (eps0_n = eps + w0 |1><1| for n >= 0, eps0_{-1} = eps)."""
    eps = np.zeros((M, M), dtype=complex)
    for i in range(M - 1):
        eps[i, i + 1] = eps[i + 1, i] = -J
    eps0 = np.broadcast_to(eps[None, :, :, None], (nt + 2, M, M, 1)).copy()
    eps0[1:, 0, 0, 0] += w0
    return Workload("hubbard_chain", nt, ntau, M, 1, korder, h, beta, corrector=corrector, eps0=eps0,
                    U=np.full(nt + 2, U), mu=mu, nbar=nbar)


def chain_kspace(nk=512, nt=2000, ntau=800, beta=10.0, h=0.01, korder=5, U=2.0, corrector=3,
                 A0=0.5, omega=2.0, t0=5.0, sigma=1.5):
    k = 2 * np.pi * np.arange(nk) / nk
    t = np.concatenate([[0.0], h * np.arange(nt + 1)])
    A = pulse_A(t, A0, omega, t0, sigma)
    A[0] = 0.0                                  # A(0^-) = 0: equilibrium before the pulse
    eps = -2.0 * np.cos(k[None, :] - A[:, None])  # [nt+2, nk]
    eps0 = eps[:, None, None, :].astype(complex)
    return Workload("chain_kspace", nt, ntau, 1, nk, korder, h, beta, corrector=corrector, eps0=eps0,
                    U=np.full(nt + 2, U), extra={"A": A, "k": k})


def square_kspace(L=16, nt=1000, ntau=400, beta=10.0, h=0.02, korder=5, U=1.5, corrector=3, A=None):
    kx, ky = np.meshgrid(2 * np.pi * np.arange(L) / L, 2 * np.pi * np.arange(L) / L, indexing="ij")
    kx, ky = kx.ravel(), ky.ravel()
    t = np.concatenate([[0.0], h * np.arange(nt + 1)])
    if A is None:
        A = pulse_A(t)
        A[0] = 0.0
    eps = -2.0 * np.cos(kx[None, :] - A[:, None]) - 2.0 * np.cos(ky[None, :])
    eps0 = eps[:, None, None, :].astype(complex)
    return Workload("square_kspace", nt, ntau, 1, L * L, korder, h, beta, corrector=corrector, eps0=eps0,
                    U=np.full(nt + 2, U), extra={"A": A})


def uneven_clusters(nprob=64, seed=191101211, nt_range=(500, 3000), ntau=300, h=0.02, beta_range=(5.0, 30.0),
                    dims=(1, 2, 4, 8), nbath=4, vscale=0.3, korder=5):
    """Independent embedded clusters: per problem nf ~ U(dims), nt ~ U{nt_range}, beta ~ U(beta_range),
    cluster Hamiltonian h (nf x nf hermitian, N(0,1) entries), a bath of nbath levels with its own
    hermitian Hamiltonian h_b and a real coupling V (nf x nbath, N(0, vscale^2)); the embedding
    self-energy is V g0(h_b) V^dagger.  Returns a list of dicts with these inputs."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nprob):
        d = int(rng.choice(dims))
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        beta = float(rng.uniform(*beta_range))
        hs = random_hermitian(rng, d)
        hb = random_hermitian(rng, nbath)
        V = rng.normal(0.0, vscale, (d, nbath))
        out.append({"nf": d, "nt": nt, "ntau": ntau, "beta": beta, "h": h, "korder": korder, "hs": hs, "hb": hb,
                    "V": V})
    return out


def random_hermitian(rng, d, scale=1.0):
    """d x d hermitian: diagonal N(0, scale^2), off-diagonal re, im ~ N(0, scale^2/2)."""
    a = rng.normal(0.0, scale, (d, d))
    b = rng.normal(0.0, scale, (d, d))
    m = np.triu(a, 1) / np.sqrt(2) + 1j * np.triu(b, 1) / np.sqrt(2)
    return m + m.conj().T + np.diag(rng.normal(0.0, scale, d))
