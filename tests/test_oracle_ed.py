"""Pins for the oracle's self-consistent dynamics (drivers.run_2b, drivers.run_gw) against exact
diagonalisation of the Hubbard dimer (tests/ed_hubbard.py).

The second-Born self-energy (Eq. sigma_hubb_2b) with the Hartree term is the exact self-energy
to second order in U, and so is GW (Eq. SigmaGW: its second-order term is the same bubble).
With U scaled as s U, the deviation of the self-consistent solution from the exact one is
therefore O(s^3): it falls by 8 when s halves.  At particle-hole symmetry (mu = 0, nbar = 1/2)
the odd orders of the exact self-energy vanish and the Hartree shift is zero, so second Born is
exact through third order there and its deviation falls by 16; GW keeps third-order terms of
its own, and its deviation falls by 8.  A dropped or mis-signed term of Sigma leaves an O(s^2)
deviation (ratio 4), a wrong mean-field term an O(s) one (ratio 2): both fail the windows.

Dimer eps = [[0, -1], [-1, 0]], U_{-1} = 0.5 s (the initial equilibrium), U_n = s for n >= 0
(the quench), beta = 2, ntau = 60, h = 0.05, 30 steps, k = 5, 3 corrector passes.  The
discretisation floor (the U = 0 run against the exact free evolution) is below 1e-6, two orders
under the smallest deviation used.  The 4-site ring (hopping -1, periodic; ntau = 40, 20 steps)
pins the multi-orbital real-space GW and the k-space GW (nk = 4) the same way.
"""
import numpy as np
import pytest

from oracle import bubble, drivers, observables
from oracle.contour import Func
from oracle.weights import Weights
from tests.ed_hubbard import HubbardED

EPS = np.array([[0.0, -1.0], [-1.0, 0.0]])
BETA, NTAU, NT, H = 2.0, 60, 30, 0.05


def _deviation(kind, s, mu=0.0):
    """max |G^M - G^M_exact| over tau in [0, beta) and max |rho(t) - rho_exact(t)| over the steps."""
    W = Weights(5)
    e0 = Func(NT, 2)
    e0.val[:] = EPS
    U = Func(NT, 1)
    U.val[:] = s
    U.set(-1, np.array([[0.5 * s]]))
    if kind == "2b":
        st = drivers.run_2b([e0], U, NT, NTAU, BETA, H, W, mu=mu, corrector=3)
    else:
        st, _ = drivers.run_gw([e0], U, NT, NTAU, BETA, H, W, mu=mu, corrector=3)
    G = st.G[0]
    ed = HubbardED(EPS, mu=mu, nbar=0.5)
    taus = np.arange(NTAU) * BETA / NTAU
    em = np.abs(G.mat[:NTAU] - ed.gmat(0.5 * s, BETA, taus)).max()
    rho = ed.density(0.5 * s, s, BETA, np.arange(NT + 1) * H)
    er = max(np.abs(observables.density_matrix(n, G) - rho[n]).max() for n in range(NT + 1))
    return em, er


def test_ed_reference_hubbard_atom():
    """The reference itself, in the atomic limit (one site, eps = 0, mu = 0): with
    H = U (n_up - 1/2)(n_dn - 1/2) the states |0>, |up,dn> have energy U/4 and |up>, |dn> -U/4,
    so G^M(tau) = -[exp(-beta U/4 + tau U/2) + exp(beta U/4 - tau U/2)] / Z,
    Z = 2 exp(-beta U/4) + 2 exp(beta U/4)."""
    U, beta = 1.3, 2.0
    taus = np.linspace(0.0, beta, 9)[:-1]
    ed = HubbardED(np.zeros((1, 1)), mu=0.0, nbar=0.5)
    z = 2 * np.exp(-beta * U / 4) + 2 * np.exp(beta * U / 4)
    exact = -(np.exp(-beta * U / 4 + taus * U / 2) + np.exp(beta * U / 4 - taus * U / 2)) / z
    assert np.allclose(ed.gmat(U, beta, taus)[:, 0, 0], exact, atol=1e-14, rtol=0)
    rho = ed.density(U, 2 * U, beta, np.array([0.0, 0.7]))
    assert np.allclose(rho[:, 0, 0], 0.5, atol=1e-14)


def test_ed_reference_is_the_free_solution_at_zero_u():
    """U = 0: the oracle's free dimer equals the exact one (Matsubara exactly, real time to the
    discretisation)."""
    em, er = _deviation("2b", 0.0)
    assert em < 1e-14 and er < 1e-6, (em, er)


def test_second_born_exact_through_third_order_at_half_filling():
    a, b = _deviation("2b", 0.5), _deviation("2b", 0.25)
    rm, rr = a[0] / b[0], a[1] / b[1]
    assert 12.0 < rm < 20.0 and 12.0 < rr < 20.0, (a, b, rm, rr)
    assert b[1] < 5e-5, b


def test_second_born_exact_to_second_order_off_half_filling():
    a, b = _deviation("2b", 0.5, mu=0.3), _deviation("2b", 0.25, mu=0.3)
    rm = a[0] / b[0]
    assert 6.0 < rm < 10.5, (a, b, rm)
    assert b[1] < 5e-5, b


def test_gw_exact_to_second_order():
    a, b = _deviation("gw", 0.5), _deviation("gw", 0.25)
    rm, rr = a[0] / b[0], a[1] / b[1]
    assert 6.0 < rm < 10.5 and 6.0 < rr < 10.5, (a, b, rm, rr)


def _energy_deviation(kind, s):
    """max_t |2 E(t) - <H(U_1)>| for t >= 0: E is the oracle's energy per spin, the one-body
    and mean-field part (1/2) Tr rho (eps + eps^MF) plus the Galitskii-Migdal correlation energy
    (Eq. Total_ener); the exact energy after the quench is Tr rho_0 H(U_1), constant in time.
    At half filling the mean-field reference nbar = 1/2 adds nothing to either side."""
    W = Weights(5)
    e0 = Func(NT, 2)
    e0.val[:] = EPS
    U = Func(NT, 1)
    U.val[:] = s
    U.set(-1, np.array([[0.5 * s]]))
    if kind == "2b":
        st = drivers.run_2b([e0], U, NT, NTAU, BETA, H, W, corrector=3)
    else:
        st, _ = drivers.run_gw([e0], U, NT, NTAU, BETA, H, W, corrector=3)
    G, S = st.G[0], st.S
    ed = HubbardED(EPS, mu=0.0, nbar=0.5)
    _, V0, p0 = ed.thermal(0.5 * s, BETA)
    e_exact = np.real(np.trace(((V0 * p0) @ V0.conj().T) @ (ed.h0 + s * ed.vint)))
    dev = 0.0
    for n in range(NT + 1):
        rho = observables.density_matrix(n, G)
        e = 0.5 * np.real(np.trace(rho @ (e0(n) + st.epsmf[0](n)))) + observables.correlation_energy(n, G, S, W, BETA, H)
        dev = max(dev, abs(2.0 * e - e_exact))
    return dev


@pytest.mark.parametrize("kind,lo,hi", [("2b", 12.0, 20.0), ("gw", 6.0, 10.5)])
def test_total_energy_exact_to_the_order_of_the_self_energy(kind, lo, hi):
    a, b = _energy_deviation(kind, 0.5), _energy_deviation(kind, 0.25)
    assert lo < a / b < hi, (a, b, a / b)


def test_pin_detects_a_wrong_correlation_energy(monkeypatch):
    """Planted: the Galitskii-Migdal term twice too large, an O(U^2) error."""
    orig = observables.correlation_energy
    monkeypatch.setattr(observables, "correlation_energy", lambda *a, **k: 2.0 * orig(*a, **k))
    a, b = _energy_deviation("2b", 0.5), _energy_deviation("2b", 0.25)
    assert a / b < 6.0, (a, b)


# ---- the 4-site ring: the multi-orbital real-space GW (d = 4) and the k-space GW (nk = 4) ----
RING_NTAU, RING_NT = 40, 20


def _ring_eps(M=4):
    eps = np.zeros((M, M))
    for i in range(M):
        eps[i, (i + 1) % M] = eps[(i + 1) % M, i] = -1.0
    return eps


def _ring_deviation(s, kspace, kind="gw"):
    """Deviation of G^M_ij(tau) and rho_ij(t) from the exact ring (256-state Fock space; at
    half filling rho_ii stays 1/2, the bond densities rho_{i,i+1} carry the dynamics): the
    real-space run (one problem, d = 4 sites) or the k-space run (nk = 4 one-band problems,
    eps_k = -2 cos k, Sigma_k by Eqs. Sigmak, Pol), taken to sites by
    X_ij = (1/N_k) sum_k exp(i k (r_i - r_j)) X_k."""
    from oracle import gw
    M, N, T = 4, RING_NT, RING_NTAU
    W = Weights(5)
    U = Func(N, 1)
    U.val[:] = s
    U.set(-1, np.array([[0.5 * s]]))
    if kspace:
        e0 = []
        for kk in range(M):
            f = Func(N, 1)
            f.val[:] = -2.0 * np.cos(2 * np.pi * kk / M)
            e0.append(f)
        st, _ = drivers.run_gw_kspace(e0, U, N, T, BETA, H, W, *gw.ring_tables(M), corrector=3)
        r = np.arange(M)
        ph = np.exp(2j * np.pi * np.arange(M)[None, None, :] * (r[:, None, None] - r[None, :, None]) / M) / M
        gm = np.einsum("tk,ijk->tij", np.stack([g.mat[:T, 0, 0] for g in st.G], axis=-1), ph)
        rho = [np.einsum("k,ijk->ij", np.array([observables.density_matrix(n, g)[0, 0] for g in st.G]), ph)
               for n in range(N + 1)]
    else:
        e0 = Func(N, M)
        e0.val[:] = _ring_eps(M)
        if kind == "2b":
            st = drivers.run_2b([e0], U, N, T, BETA, H, W, corrector=3)
        else:
            st, _ = drivers.run_gw([e0], U, N, T, BETA, H, W, corrector=3)
        gm = st.G[0].mat[:T]
        rho = [observables.density_matrix(n, st.G[0]) for n in range(N + 1)]
    ed = HubbardED(_ring_eps(M), mu=0.0, nbar=0.5)
    em = np.abs(gm - ed.gmat(0.5 * s, BETA, np.arange(T) * BETA / T)).max()
    ex = ed.density(0.5 * s, s, BETA, np.arange(N + 1) * H)
    return em, max(np.abs(rho[n] - ex[n]).max() for n in range(N + 1))


@pytest.mark.parametrize("kspace", [False, True], ids=["real_space_d4", "kspace_nk4"])
def test_ring_gw_exact_to_second_order(kspace):
    a, b = _ring_deviation(0.5, kspace), _ring_deviation(0.25, kspace)
    rm, rr = a[0] / b[0], a[1] / b[1]
    assert 6.0 < rm < 10.5 and 6.0 < rr < 10.5, (a, b, rm, rr)


def test_ring_second_born_exact_through_third_order():
    """The multi-orbital second Born (d = 4) of the half-filled ring: O(U^4) deviation.  U is
    taken twice as large as for GW so that the smaller deviation (2e-5) stays well above the
    time-stepping floor of this grid (1.4e-6 at U = 0)."""
    a, b = _ring_deviation(1.0, False, "2b"), _ring_deviation(0.5, False, "2b")
    rm, rr = a[0] / b[0], a[1] / b[1]
    assert 12.0 < rm < 20.0 and 12.0 < rr < 20.0, (a, b, rm, rr)


def test_pin_detects_a_mis_signed_self_energy(monkeypatch):
    """Planted on the CPU, in the oracle: Sigma_2B with the wrong overall sign.  The deviation
    becomes O(U^2), and the half-filling window of the second-Born pin rejects it."""
    orig = bubble.sigma_2b

    def flipped(n, G, U, S):
        orig(n, G, U, S)
        if n == -1:
            S.mat[...] = -S.mat
            return
        S.ret[n, :n + 1] = -S.ret[n, :n + 1]
        S.les[:n + 1, n] = -S.les[:n + 1, n]
        S.tv[n] = -S.tv[n]

    monkeypatch.setattr(bubble, "sigma_2b", flipped)
    a, b = _deviation("2b", 0.5), _deviation("2b", 0.25)
    rm, rr = a[0] / b[0], a[1] / b[1]
    assert not (12.0 < rm < 20.0 and 12.0 < rr < 20.0), (rm, rr)
    assert rm < 6.0, rm


def test_pin_detects_a_wrong_mean_field_reference(monkeypatch):
    """Planted: the mean-field term taken about nbar = 0.4 instead of the Hamiltonian's 0.5, an
    O(U) error: the deviation falls only by about 2 when U halves."""
    orig = bubble.hartree
    monkeypatch.setattr(bubble, "hartree", lambda n, rho, e0, U, nbar: orig(n, rho, e0, U, 0.4))
    a, b = _deviation("2b", 0.5), _deviation("2b", 0.25)
    assert a[0] / b[0] < 4.0, (a, b)
