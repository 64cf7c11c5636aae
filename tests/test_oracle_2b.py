"""Pins for the oracle's second-Born self-energy, k-reduction, extrapolation and the
self-consistent driver (conservation laws)."""
import numpy as np
import pytest

from oracle import bubble, drivers, extrap, observables
from oracle.contour import Func, Herm, dag
from oracle.freegf import green_from_H
from oracle.weights import Weights


def _free2(N=8, T=12, beta=4.0, h=0.1):
    eps = np.array([[0.2, -0.6 + 0.1j], [-0.6 - 0.1j, -0.3]])
    return green_from_H(N, T, eps, 0.05, beta, h)


def _U(N, v=1.3, v0=0.8):
    U = Func(N, 1)
    U.val[:] = v
    U.set(-1, np.array([[v0]]))
    return U


def test_sigma_kms_and_hermitian_relations():
    """Sigma built from a KMS-consistent G obeys Sigma^tv(0,tau) = i xi Sigma^M(beta - tau) and
    Sigma^<(0,n) = -[Sigma^tv(n,0)]^dagger; this fixes the relative sign of the Matsubara
    component (U(0)U(0^-) = U_{-1}^2 at n = 0 on the imaginary branch is taken equal here)."""
    G = _free2()
    N, T = G.nt, G.ntau
    U = _U(N, 0.8, 0.8)
    S = Herm(N, T, 2)
    for n in range(-1, N + 1):
        bubble.sigma_2b(n, G, U, S)
    for m in range(T + 1):
        assert np.allclose(S.tv[0, m], 1j * G.sig * S.mat[T - m], atol=1e-14)
    for n in range(N + 1):
        assert np.allclose(S.les[0, n], -dag(S.tv[n, 0]), atol=1e-14)
        assert np.allclose(S.les[n, n], -dag(S.les[n, n]), atol=1e-14)


def test_sigma_matches_two_bubble_route():
    """Real-time components agree with the paper's two-step route: P = -Bubble1[G,G],
    P -> U P U, Sigma = Bubble2[G, P] (Eqs. def_bubble1, def_bubble2)."""
    G = _free2()
    N, T = G.nt, G.ntau
    U = _U(N)
    u = lambda t: U(t)[0, 0]
    S = Herm(N, T, 2)
    for n in range(N + 1):
        bubble.sigma_2b(n, G, U, S)
    for n in range(N + 1):
        for j in range(n + 1):
            gtr = lambda a, b: G.ret[a, b] + (-dag(G.les[b, a])) if a >= b else -dag(G.ret[b, a] - dag(G.les[a, b]))
            les = lambda a, b: G.les[a, b] if a <= b else -dag(G.les[b, a])
            # Bubble1: C^>(t,t') = i A^>(t,t') B^<(t',t), C^<(t,t') = i A^<(t,t') B^>(t',t)
            P_gtr = -(1j * gtr(n, j) * les(j, n).T) * u(n) * u(j)
            P_les = -(1j * les(n, j) * gtr(j, n).T) * u(n) * u(j)
            P_les_jn = -(1j * les(j, n) * gtr(n, j).T) * u(n) * u(j)
            # Bubble2: C^> = i A^> B^>, C^< = i A^< B^<
            s_gtr = 1j * gtr(n, j) * P_gtr
            s_les = 1j * les(n, j) * P_les
            assert np.allclose(S.ret[n, j], s_gtr - s_les, atol=1e-14)
            assert np.allclose(S.les[j, n], 1j * les(j, n) * P_les_jn, atol=1e-14)


def test_zero_interaction_gives_free_solution():
    """U = 0: Sigma vanishes and the self-consistent run reproduces the free GF."""
    N, T, beta, h = 16, 20, 3.0, 0.05
    W = Weights(5)
    e0 = Func(N, 2)
    e0.val[:] = np.array([[0.0, -1.0], [-1.0, 0.0]])
    U = Func(N, 1)
    st = drivers.run_2b([e0], U, N, T, beta, h, W, corrector=2)
    ex = green_from_H(N, T, e0(0), 0.0, beta, h)
    assert np.abs(st.S.ret).max() == 0 and np.abs(st.S.mat).max() == 0
    assert np.abs(st.G[0].mat - ex.mat).max() < 1e-12
    assert np.abs(st.G[0].tv - ex.tv).max() < 1e-7   # BDF truncation at h = 0.05


def test_kreduce_is_the_mean():
    Gs = [_free2(), _free2(beta=3.0)]
    L = Herm(Gs[0].nt, Gs[0].ntau, 2)
    for n in range(-1, Gs[0].nt + 1):
        bubble.kreduce(n, Gs, L)
    assert np.allclose(L.tv, 0.5 * (Gs[0].tv + Gs[1].tv))
    assert np.allclose(np.tril(L.ret[..., 0, 0]), np.tril(0.5 * (Gs[0].ret + Gs[1].ret)[..., 0, 0]))


def test_extrapolation_exact_on_polynomials():
    """extrapolate_timestep reproduces data that are polynomials of degree <= k in both
    time arguments (Eq. polyextrap along columns, rows and diagonals)."""
    k, N, T = 4, 14, 3
    W = Weights(k)
    G = Herm(N, T, 1)
    p = lambda t, s: 0.3 + 0.1j * t - 0.02 * s + 0.003 * (t - s) ** 2 + 1e-4j * t ** 3 * s
    for n in range(N + 1):
        for j in range(n + 1):
            G.ret[n, j] = p(n, j)
            G.les[j, n] = p(j, n) - np.conj(p(n, j))        # anti-hermitian pair structure
        G.tv[n] = (0.5 + 0.01j * n ** 2)
    # make ret consistent with its continuation for t < t': G~^R(j,n) = -conj(G^R(n,j))
    ref = G.copy()
    for n in range(k, N):
        H = ref.copy()
        H.ret[n + 1] = 0
        H.les[:, n + 1] = 0
        H.tv[n + 1] = 0
        extrap.extrapolate_timestep(n, H, W)
        assert np.allclose(H.tv[n + 1], ref.tv[n + 1], atol=1e-10)
        for j in range(k + 1, n + 2):
            assert np.allclose(H.ret[n + 1, j], ref.ret[n + 1, j], atol=1e-9)
            assert np.allclose(H.les[j, n + 1], ref.les[j, n + 1], atol=1e-9)


@pytest.mark.slow
def test_dimer_quench_conservation():
    """Self-consistent second-Born Hubbard dimer after the quench U: 1 -> 2: the total
    (Galitskii-Migdal) energy and the particle number are conserved for t > 0 up to the
    discretisation, and the drift falls under halving of h (Eq. Total_ener)."""
    drifts, ndrift = [], []
    for N, h in ((40, 0.1), (80, 0.05)):
        W = Weights(5)
        e0 = Func(N, 2)
        e0.val[:] = np.array([[0.0, -1.0], [-1.0, 0.0]])
        U = _U(N, 2.0, 1.0)
        st = drivers.run_2b([e0], U, N, 30, 5.0, h, W, corrector=3)
        G, S = st.G[0], st.S
        E, Nn = [], []
        for n in range(N + 1):
            rho = observables.density_matrix(n, G)
            E.append(0.5 * np.real(np.trace(rho @ (e0(n) + st.epsmf[0](n))))
                     + observables.correlation_energy(n, G, S, W, 5.0, h))
            Nn.append(np.real(np.trace(rho)))
        drifts.append(np.ptp(E[1:]))
        ndrift.append(np.ptp(Nn))
    assert drifts[1] < drifts[0] / 8 and drifts[1] < 1e-3, drifts
    assert ndrift[1] < 1e-4, ndrift
