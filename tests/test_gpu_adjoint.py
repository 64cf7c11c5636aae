"""Hand-written discrete adjoint (ng_adjoint_2b behind torch.autograd) against the oracle's
reference gradient (fourth-order finite differences of the FP64 CPU forward algorithm) and
against central finite differences of the GPU forward (delta = 1e-6)."""
import multiprocessing as mp

import numpy as np
import pytest
import torch

from paper_1911_01211_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ng():
    import paper_1911_01211_gb300 as ng
    ng.load_library()
    return ng


def _kgrid(L):
    kx, ky = np.meshgrid(2 * np.pi * np.arange(L) / L, 2 * np.pi * np.arange(L) / L, indexing="ij")
    return kx.ravel(), ky.ravel()


def _eps0(A, L):
    """eps0_k(t_n) = -2 cos(kx - A_n) - 2 cos(ky) as a differentiable torch expression [nt+2, L^2]."""
    kx, ky = _kgrid(L)
    kx = torch.as_tensor(kx, device=A.device)
    ky = torch.as_tensor(ky, device=A.device)
    return -2.0 * torch.cos(kx[None, :] - A[:, None]) - 2.0 * torch.cos(ky[None, :])


class _Problem:
    def __init__(self, ng, L, nt, ntau, beta, h, U, corrector=3):
        self.ng, self.L, self.U, self.corrector = ng, L, U, corrector
        self.g = ng.Grid(nt=nt, ntau=ntau, nf=1, nbatch=L * L, korder=5, h=h, beta=beta)
        self.ctx = ng.Context(5)
        self.Ut = torch.full((nt + 2,), U, dtype=torch.float64, device="cuda")

    def loss(self, A, kind="ekin", segment=0, state=None):
        from paper_1911_01211_gb300.adjoint import densities
        e0 = _eps0(A, self.L)
        rho = densities(e0, self.ctx, self.g, self.Ut, corrector=self.corrector, segment=segment, state=state)
        N = self.g.nt
        if kind == "ekin":   # E_kin(t_N) = (1/N_k) sum_k Re rho_k(t_N) eps0_k(t_N)
            return (rho[N].real * e0[N + 1]).mean()
        # occupation of the k-point (pi/2, 0): changed by the field (the k-summed occupation
        # is conserved, so its gradient vanishes to discretisation level)
        return rho[N, self.L].real

    def grad(self, A, kind="ekin", segment=0):
        At = torch.tensor(A, dtype=torch.float64, device="cuda", requires_grad=True)
        L = self.loss(At, kind, segment)
        L.backward()
        return L.item(), At.grad.cpu().numpy()

    def value(self, A, kind="ekin"):
        with torch.no_grad():
            return float(self.loss(torch.tensor(A, dtype=torch.float64, device="cuda"), kind))


# ---- oracle reference gradient, evaluated in spawned worker processes -----------------
def _oracle_fd(args):
    L, nt, ntau, beta, h, U, A, i = args
    from oracle import gradient
    from oracle.contour import Func
    from oracle.weights import Weights
    W = Weights(5)

    def f(Ax):
        w = wl.square_kspace(L=L, nt=nt, ntau=ntau, beta=beta, h=h, U=U, A=Ax)
        eps = []
        for kk in range(w.nbatch):
            e = Func(nt, 1)
            e.val[:, 0, 0] = w.eps0[:, 0, 0, kk]
            eps.append(e)
        Uf = Func(nt, 1)
        Uf.val[:, 0, 0] = w.U
        return gradient.kinetic_energy(eps, Uf, nt, ntau, beta, h, W)
    return gradient.fd_derivative(f, A, i)


def test_adjoint_matches_oracle_reference_gradient(ng):
    L, nt, ntau, beta, h, U = 2, 18, 12, 2.0, 0.1, 1.0
    rng = np.random.default_rng(1911)
    A = np.zeros(nt + 2)
    A[2:] = 0.4 * rng.standard_normal(nt)
    p = _Problem(ng, L, nt, ntau, beta, h, U)
    _, g = p.grad(A)
    # slices: bootstrap (1..5), whole-column (A) region (6..10), (B) region and the last
    idx = [n + 1 for n in (1, 3, 5, 6, 8, 10, 11, 14, 17, 18)]
    with mp.get_context("spawn").Pool(min(len(idx), 10)) as pool:
        ref = np.array(pool.map(_oracle_fd, [(L, nt, ntau, beta, h, U, A, i) for i in idx]))
    got = g[idx]
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 1e-8, (err, got, ref)


def test_adjoint_matches_gpu_finite_differences(ng):
    L, nt, ntau, beta, h, U = 4, 80, 40, 5.0, 0.05, 1.5
    t = np.concatenate([[0.0], h * np.arange(nt + 1)])
    A = wl.pulse_A(t, A0=0.5, omega=2.0, t0=2.0, sigma=0.8)
    A[:2] = 0.0
    p = _Problem(ng, L, nt, ntau, beta, h, U)
    rng = np.random.default_rng(191101211)
    idx = sorted(set([3] + list(rng.choice(np.arange(6, nt + 2), 5, replace=False)) + [nt + 1]))
    delta = 1e-6
    for kind in ("ekin", "nk"):
        _, g = p.grad(A, kind)
        fd = []
        for i in idx:
            Ap, Am = A.copy(), A.copy()
            Ap[i] += delta
            Am[i] -= delta
            fd.append((p.value(Ap, kind) - p.value(Am, kind)) / (2 * delta))
        fd = np.array(fd)
        err = np.abs(g[idx] - fd).max() / np.abs(fd).max()
        assert err < 1e-6, (kind, err, g[idx], fd)


def test_adjoint_segment_length_does_not_change_the_gradient(ng):
    L, nt, ntau, beta, h, U = 2, 40, 16, 3.0, 0.05, 1.0
    t = np.concatenate([[0.0], h * np.arange(nt + 1)])
    A = wl.pulse_A(t, A0=0.5, omega=2.0, t0=1.0, sigma=0.5)
    A[:2] = 0.0
    p = _Problem(ng, L, nt, ntau, beta, h, U)
    _, g0 = p.grad(A, segment=0)       # ceil(sqrt(nt - k)) steps per segment
    _, g1 = p.grad(A, segment=1)
    _, g2 = p.grad(A, segment=nt)
    _, g3 = p.grad(A, segment=ng.NG_ADJ_RECORDED)   # iterates kept by the forward, none recomputed
    scale = np.abs(g0).max()
    assert np.abs(g1 - g0).max() <= 1e-13 * scale
    assert np.abs(g2 - g0).max() <= 1e-13 * scale
    assert np.abs(g3 - g0).max() <= 1e-13 * scale
    # a checkpointed backward reuses the store and releases the record: a recorded backward
    # after it is refused
    p.grad(A, segment=0)
    with pytest.raises(ng.NgError):
        p.ctx.adjoint_2b(p.g, ng.Herm(p.g), ng.Herm(p.g, ldk=1), ng.Herm(p.g, ldk=1), ng.Func(p.g), ng.Func(p.g),
                         ng.Func(p.g, scalar=True), torch.zeros((nt + 1, L * L), dtype=torch.complex128,
                                                                device="cuda"),
                         ng.Herm(p.g), ng.Herm(p.g, ldk=1), torch.zeros((nt + 2, L * L), dtype=torch.float64,
                                                                        device="cuda"),
                         segment=ng.NG_ADJ_RECORDED)
