"""Pins for the oracle's Dyson solver: closed forms, downfolding brute force, convergence
rates, schedule agreement and the contour identities."""
import numpy as np
import pytest

from oracle import conv, drivers, dyson
from oracle.contour import Func, Herm, dag
from oracle.freegf import green_from_H
from oracle.weights import Weights
from tests.oracle_cases import embedded_level, max_err


def test_free_closed_form_identities():
    """Jump G^M(0+) - xi G^M(beta-) = -1, KMS (Eq. kmsbound_keld), G^R(t,t) = -i (Eq. gretdiag)
    and the equation of motion i dG^R/dt = (eps - mu) G^R by central differences."""
    eps = np.array([[0.4, 0.2 - 0.1j], [0.2 + 0.1j, -0.7]])
    N, T, beta, h = 12, 16, 3.0, 0.01
    G = green_from_H(N, T, eps, 0.1, beta, h)
    assert np.allclose(G.mat[0] - G.sig * G.mat[T], -np.eye(2), atol=1e-14)
    for m in range(T + 1):
        assert np.allclose(G.tv[0, m], 1j * G.sig * G.mat[T - m], atol=1e-14)
    for n in range(N + 1):
        assert np.allclose(G.ret[n, n], -1j * np.eye(2), atol=1e-14)
        assert np.allclose(G.les[0, n], -dag(G.tv[n, 0]), atol=1e-14)
    for n in range(1, N):
        dG = (G.ret[n + 1, 0] - G.ret[n - 1, 0]) / (2 * h)
        assert np.allclose(1j * dG, (eps - 0.1 * np.eye(2)) @ G.ret[n, 0], atol=1e-4)


def test_sigma_zero_gives_free_gf():
    """With Sigma = 0 the solver reproduces the closed-form free GF to BDF accuracy."""
    N, T, beta, h = 30, 30, 5.0, 0.05
    ex = green_from_H(N, T, np.array([[0.3]]), 0.0, beta, h)
    G, S = Herm(N, T, 1), Herm(N, T, 1)
    eps = Func(N, 1)
    eps.val[:] = 0.3
    drivers.solve_fixed_sigma(G, S, eps, 0.0, beta, h, Weights(5))
    e = max_err(G, ex)
    assert e["mat"] < 1e-13 and max(e.values()) < 1e-9, e


def test_downfolding_brute_force_and_rate():
    """Embedded level vs the exact 2x2 eigen-evolution; the error falls ~2^k per halving of h
    (k = 5; the paper's average error is O(h^(k+1)))."""
    errs = []
    for N in (20, 40, 80):
        G, ex, _ = embedded_level(N, 40, 2.0, 2.0 / N)
        e = max_err(G, ex)
        assert e["mat"] < 1e-12
        errs.append(max(e["ret"], e["les"], e["tv"]))
    assert errs[-1] < 3e-10
    for a, b in zip(errs, errs[1:]):
        assert a / b > 2 ** 5 * 0.7, errs


def test_matsubara_converges_fast_in_htau():
    """Matsubara downfolding error falls roughly as h_tau^(k+2) (Fig. test_eq), k = 3."""
    W = Weights(3)
    errs = []
    beta = 20.0
    e1, lam, e2 = -1.0, 0.5, 1.0
    for T in (50, 100, 200):
        ex = green_from_H(0, T, np.array([[e1, 1j * lam], [-1j * lam, e2]]), 0.0, beta, 0.1)
        S = green_from_H(0, T, np.array([[e2]]), 0.0, beta, 0.1)
        S.mat *= lam ** 2
        G = Herm(0, T, 1)
        eps = Func(0, 1)
        eps.val[:] = e1
        dyson.dyson_mat(G, S, eps, 0.0, beta, W)
        errs.append(np.abs(G.mat[:, 0, 0] - ex.mat[:, 0, 0]).mean())
    rate = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert min(rate) > 3.5, (errs, rate)


def test_serial_and_mixed_schedules_agree_to_discretisation():
    """Implementations (A) and (B) differ only at the discretisation level."""
    Gm, ex, _ = embedded_level(40, 30, 2.0, 0.05, schedule="mixed")
    Gs, _, _ = embedded_level(40, 30, 2.0, 0.05, schedule="serial")
    d = max_err(Gm, Gs, sub=(slice(None), slice(None)))
    e = max_err(Gm, ex)
    assert 0 < max(d.values()) < 10 * max(e.values())


def test_contour_identities_of_solution():
    """Solution satisfies G^R(t,t) = -i, KMS for tv and les, hermitian density matrix."""
    G, _, _ = embedded_level(25, 20, 2.0, 0.05)
    T = G.ntau
    for n in range(G.nt + 1):
        assert abs(G.ret[n, n, 0, 0] + 1j) < 1e-13
        assert np.allclose(G.les[0, n], -dag(G.tv[n, 0]), atol=1e-13)
        assert abs(np.real(G.les[n, n, 0, 0])) < 1e-10     # rho = -iG^< real up to discretisation
    for m in range(T + 1):
        assert np.allclose(G.tv[0, m], 1j * G.sig * G.mat[T - m], atol=1e-13)


def _d_eps_free(N, T, e, beta, h, de=1e-5):
    """dG0/de by central difference of the closed form; equals [G0 * G0] (G0 = (i d_t - e)^-1)."""
    gp = green_from_H(N, T, np.array([[e + de]]), 0.0, beta, h)
    gm = green_from_H(N, T, np.array([[e - de]]), 0.0, beta, h)
    out = Herm(N, T, 1)
    for c in ("mat", "ret", "les", "tv"):
        setattr(out, c, (getattr(gp, c) - getattr(gm, c)) / (2 * de))
    return out


def test_convolution_timestep_equals_energy_derivative():
    """[G0 * G0] = dG0/de for a free GF: pins every piece C^M, C^R, C^tv_1..3, C^<_1..3."""
    N, T, beta, h, e = 24, 60, 3.0, 0.05, 0.35
    W = Weights(5)
    g = green_from_H(N, T, np.array([[e]]), 0.0, beta, h)
    C = Herm(N, T, 1)
    for n in range(-1, N + 1):
        conv.convolution_timestep(n, C, g, g, None, g, g, W, beta, h)
    ref = _d_eps_free(N, T, e, beta, h)
    err = max_err(C, ref)
    assert max(err.values()) < 2e-7, err


def test_planted_kernel_sign_error_is_caught(monkeypatch):
    """Planting a wrong sign in the tv history kernel breaks the downfolding pin."""
    orig = dyson.tv_row

    def broken(G, S, eps, mu, h, beta, W, n, Mn_inv):
        S2 = S.copy()
        S2.ret = -S2.ret
        return orig(G, S2, eps, mu, h, beta, W, n, Mn_inv)

    monkeypatch.setattr(dyson, "tv_row", broken)
    G, ex, _ = embedded_level(20, 20, 2.0, 0.1)
    assert max_err(G, ex)["tv"] > 1e-4


def test_equilibrium_time_translation_invariance():
    """A time-independent problem in equilibrium (the embedded level, Sigma = V^2 g0) has
    G(t, t') depending on t - t' only and a constant density: the discrete solution keeps
    this to discretisation accuracy, and the deviation falls with h like the solver's error."""
    devs = []
    for N in (20, 40):
        h = 2.0 / N
        G, _, _ = embedded_level(N, 40, 2.0, h)
        R, L = G.ret[..., 0, 0], G.les[..., 0, 0]
        d = 0.0
        for lag in range(0, N // 2):
            r = np.array([R[n, n - lag] for n in range(lag, N + 1)])
            l = np.array([L[n - lag, n] for n in range(lag, N + 1)])
            d = max(d, np.abs(r - r[0]).max(), np.abs(l - l[0]).max())
        dens = np.array([L[n, n] for n in range(N + 1)])
        d = max(d, np.abs(dens - dens[0]).max())
        devs.append(d)
    assert devs[-1] < 1e-8, devs
    assert devs[0] / devs[1] > 2 ** 5 * 0.7, devs


# ---- multi-orbital pins: non-commuting matrices everywhere ------------------------------
from tests.oracle_cases import embedded_cluster  # noqa: E402


def _cluster_errs(d, nbath, Ns, seed, schedule="mixed"):
    out = []
    for N in Ns:
        G, ex, _, _ = embedded_cluster(d, nbath, N, 64, 1.0, 1.0 / N, seed=seed, schedule=schedule)
        out.append(max_err(G, ex, sub=(slice(0, d), slice(0, d))))
    return out


@pytest.mark.parametrize("d,nbath,seed", [(2, 2, 7), (4, 3, 9)])
def test_multiorbital_downfolding_brute_force(d, nbath, seed):
    """A d-orbital cluster with a complex hermitian h_c, coupled by a complex V to an nbath-site
    bath folded in as Sigma = V g0_b V^dagger: every component of the solution matches the cluster
    block of the exact (d + nbath)-level eigen-evolution, and the real-time error falls by
    about 2^k (k = 5) per halving of h (Sec. "Test of accuracy and scaling analysis")."""
    errs = _cluster_errs(d, nbath, (20, 40, 80), seed)
    assert max(e["mat"] for e in errs) < 1e-10, errs
    for c in ("ret", "les", "tv"):
        seq = [e[c] for e in errs]
        for a, b in zip(seq, seq[1:]):
            assert a / b > 0.7 * 2 ** 5, (c, seq)
    assert max(errs[-1].values()) < (3e-9 if d == 2 else 3e-7), errs[-1]


def test_multiorbital_downfolding_serial_schedule():
    """The serial schedule (implementation (A) along the whole row and column) converges to the
    same exact d = 2 cluster solution at the same rate."""
    errs = _cluster_errs(2, 2, (20, 40), 7, schedule="serial")
    for c in ("ret", "les", "tv"):
        assert errs[0][c] / errs[1][c] > 0.7 * 2 ** 5, (c, errs)
    assert max(errs[-1].values()) < 1e-7, errs


def _free(N, T, eps, beta, h):
    return green_from_H(N, T, eps, 0.0, beta, h)


def _conv_all(N, A, f, B, W, beta, h):
    C = Herm(N, A.ntau, A.d)
    for n in range(-1, N + 1):
        conv.convolution_timestep(n, C, A, A, f, B, B, W, beta, h)
    return C


def _const_func(N, F):
    f = Func(N, F.shape[0])
    f.val[:] = F
    return f


def _two_hamiltonians():
    rng = np.random.default_rng(31)
    a = rng.normal(0, 1, (2, 2)) + 1j * rng.normal(0, 1, (2, 2))
    e1 = 0.5 * (a + a.conj().T)
    b = rng.normal(0, 1, (2, 2)) + 1j * rng.normal(0, 1, (2, 2))
    dE = 0.3 * (b + b.conj().T)
    assert np.abs(e1 @ dE - dE @ e1).max() > 0.1         # they do not commute
    return e1, e1 + dE


def test_convolution_resolvent_identity_noncommuting():
    """For free GFs G_i = (i d_t - eps_i)^-1 of two non-commuting d = 2 Hamiltonians at the same
    beta and mu, the contour identity G_1 - G_2 = G_1 * (eps_1 - eps_2) * G_2 holds on every
    branch.  With a constant middle function f = eps_1 - eps_2 the discrete convolution
    reproduces it to quadrature accuracy in C^M, C^R, C^tv_1..3 and C^<_1..3 (Eqs. cm1-cles3),
    and the error falls with h like the k = 5 Gregory rule (>= 2^6 per halving)."""
    e1, e2 = _two_hamiltonians()
    W = Weights(5)
    errs = []
    for N, T in ((12, 40), (24, 80)):
        beta, h = 2.0, 0.6 / N
        G1, G2 = _free(N, T, e1, beta, h), _free(N, T, e2, beta, h)
        C = _conv_all(N, G1, _const_func(N, e1 - e2), G2, W, beta, h)
        ref = Herm(N, T, 2)
        for c in ("mat", "ret", "les", "tv"):
            setattr(ref, c, getattr(G1, c) - getattr(G2, c))
        errs.append(max_err(C, ref, sub=(slice(None), slice(None))))
    assert max(errs[-1].values()) < 1e-9, errs
    for c in ("ret", "les", "tv", "mat"):
        assert errs[0][c] / errs[1][c] > 2 ** 6 * 0.7, (c, errs)


def test_convolution_energy_derivative_noncommuting():
    """[G0 * F * G0] = d G0(eps + lam F)/d lam at lam = 0 for a d = 2 free GF and a constant F
    that does not commute with eps: pins the order A f B of every piece with f between the
    two factors (a product A B f or f A B fails)."""
    e1, e2 = _two_hamiltonians()
    F = e2 - e1
    N, T, beta, h, dl = 16, 60, 2.0, 0.04, 1e-5
    W = Weights(5)
    g = _free(N, T, e1, beta, h)
    C = _conv_all(N, g, _const_func(N, F), g, W, beta, h)
    gp, gm = _free(N, T, e1 + dl * F, beta, h), _free(N, T, e1 - dl * F, beta, h)
    ref = Herm(N, T, 2)
    for c in ("mat", "ret", "les", "tv"):
        setattr(ref, c, (getattr(gp, c) - getattr(gm, c)) / (2 * dl))
    err = max_err(C, ref, sub=(slice(None), slice(None)))
    assert max(err.values()) < 1e-7, err


def test_planted_transposition_in_les_bulk_is_caught(monkeypatch):
    """Multiplying the (B) lesser step by (M_n^dagger)^-1 from the left instead of the right
    breaks the d = 2 brute-force pin (the d = 1 pins cannot see it)."""
    def broken(G, S, eps, mu, h, beta, W, n, Mn_dag_inv):
        k, d = W.k, G.d
        w = W.w(n)
        for m in range(1, n - k):
            acc = dyson.q_les_B(G, S, m, n, W, h, beta)
            for l in range(1, k + 1):
                acc = acc - W.a[l] / h * G.les[m, n - l]
            Gml = np.concatenate([-dag(G.les[:m, m]), G.les[m, m:n]])
            acc = acc - h * np.einsum("l,lab,lbc->ac", w[:n], Gml, -1j * dag(S.ret[n, :n]))
            G.les[m, n] = Mn_dag_inv @ acc
    ok = _cluster_errs(2, 2, (20,), 7)[0]
    monkeypatch.setattr(dyson, "les_bulk_B", broken)
    bad = _cluster_errs(2, 2, (20,), 7)[0]
    assert bad["les"] > 100 * ok["les"], (ok, bad)


def test_planted_solve_side_in_ret_startup_is_caught(monkeypatch):
    """Solving the conjugate (right-multiplied) retarded start-up system as a left-multiplied one
    breaks the d = 2 brute-force pin."""
    ok = _cluster_errs(2, 2, (20,), 7)[0]
    monkeypatch.setattr(dyson, "_solve_blocks_right", dyson._solve_blocks)
    bad = _cluster_errs(2, 2, (20,), 7)[0]
    assert bad["ret"] > 100 * ok["ret"], (ok, bad)


def test_planted_product_order_in_convolution_is_caught(monkeypatch):
    """Evaluating the quadrature sums as A B f instead of A f B breaks the non-commuting
    energy-derivative pin."""
    def broken(w, X, F, Y):
        if F.ndim == 2:
            return np.einsum("l,lab,lbc,cd->ad", w, X, Y, F)
        return np.einsum("l,lab,lbc,lcd->ad", w, X, Y, F)
    monkeypatch.setattr(conv, "wsum", broken)
    with pytest.raises(AssertionError):
        test_convolution_energy_derivative_noncommuting()
