"""Pins for the oracle's reference gradient (fourth-order finite differences of the plain
forward algorithm): the stencil is exact on quartics, its result does not depend on the step,
and for a free system (U = 0) the gradient of the final kinetic energy converges under step
halving to the continuum values: dE_kin(t_N)/dA(t_N) = (1/N_k) sum_k n_k d eps_k/dA (the
occupations n_k = f(eps_k(0^-)) are conserved) and, for a uniform energy shift c of
eps_k(t), t >= 0 (a gauge transformation), dE_kin(t_N)/dc = (1/N_k) sum_k n_k(t_N)."""
import numpy as np
import pytest

from oracle import drivers, gradient
from oracle.contour import Func
from oracle.weights import Weights
from paper_1911_01211_gb300 import workloads as wl


def _funcs(w, shift=0.0):
    out = []
    for kk in range(w.nbatch):
        f = Func(w.nt, 1)
        f.val[:, 0, 0] = w.eps0[:, 0, 0, kk]
        f.val[1:] += shift          # t_n, n >= 0; eps(0^-) (index 0) unchanged
        out.append(f)
    return out


def _U(w):
    U = Func(w.nt, 1)
    U.val[:, 0, 0] = w.U
    return U


def _loss(L, nt, ntau, beta, h, U):
    W = Weights(5)

    def f(A, shift=0.0):
        w = wl.square_kspace(L=L, nt=nt, ntau=ntau, beta=beta, h=h, U=U, A=A)
        return gradient.kinetic_energy(_funcs(w, shift), _U(w), nt, ntau, beta, h, W)
    return f


def _smooth_A(nt, h):
    t = np.concatenate([[0.0], h * np.arange(nt + 1)])
    A = wl.pulse_A(t, A0=0.5, omega=2.0, t0=0.7, sigma=0.5)
    A[:2] = 0.0                       # A(0^-) = A(0) = 0
    return A


def test_fd_stencil_exact_on_quartic():
    f = lambda x: x[0] ** 4 - 3.0 * x[0] ** 3 + 0.5 * x[0] * x[1] - x[1] ** 2
    x0 = np.array([0.7, -1.3])
    exact0 = 4 * 0.7 ** 3 - 9 * 0.7 ** 2 + 0.5 * (-1.3)
    exact1 = 0.5 * 0.7 + 2.6
    assert abs(gradient.fd_derivative(f, x0, 0, 0.1) - exact0) < 1e-12
    assert abs(gradient.fd_derivative(f, x0, 1, 0.1) - exact1) < 1e-12


@pytest.mark.slow
def test_reference_gradient_free_limit_converges():
    L, beta, ntau = 2, 2.0, 12
    kx = np.repeat(2 * np.pi * np.arange(L) / L, L)
    errs = []
    for h, nt in ((0.1, 14), (0.05, 28)):
        A = _smooth_A(nt, h)
        f = _loss(L, nt, ntau, beta, h, 0.0)
        gN = gradient.fd_derivative(f, A, nt + 1)
        w = wl.square_kspace(L=L, nt=nt, ntau=ntau, beta=beta, h=h, U=0.0, A=A)
        nk = 1.0 / (np.exp(beta * w.eps0[0, 0, 0, :].real) + 1.0)
        closed = np.mean(nk * (-2.0 * np.sin(kx - A[nt + 1])))
        gc = gradient.fd_derivative(lambda x: f(A, x[0]), np.zeros(1), 0)
        st = drivers.run_2b(_funcs(w), _U(w), nt, ntau, beta, h, Weights(5), mats_tol=1e-14, boot_tol=1e-14)
        dens = np.mean([np.imag(G.les[nt, nt, 0, 0]) for G in st.G])
        errs.append((abs(gN - closed) / abs(closed), abs(gc - dens) / abs(dens)))
    (a1, b1), (a2, b2) = errs
    assert a2 < 0.03 and b2 < 0.03, errs
    assert a1 / a2 > 3.0 and b1 / b2 > 3.0, errs


@pytest.mark.slow
def test_reference_gradient_step_independent():
    """Interacting run, non-smooth field: the derivative of the discrete algorithm is resolved
    (two stencil steps agree far below the adjoint tolerance)."""
    L, nt, ntau, beta, h = 2, 14, 12, 2.0, 0.1
    rng = np.random.default_rng(11)
    A = np.zeros(nt + 2)
    A[2:] = 0.4 * rng.standard_normal(nt)
    f = _loss(L, nt, ntau, beta, h, 1.0)
    for i in (3, nt - 2):
        g1 = gradient.fd_derivative(f, A, i, 1e-3)
        g2 = gradient.fd_derivative(f, A, i, 2e-3)
        assert abs(g1 - g2) < 1e-9 * max(1.0, abs(g1)), (i, g1, g2)
