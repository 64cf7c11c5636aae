"""Gradients of final-time observables through the second-Born time stepping.

``Dyson2B`` is a ``torch.autograd.Function`` whose forward is ng_run_2b (FP64, nf = 1) and
whose backward is ng_adjoint_2b, the hand-written discrete adjoint of the same algorithm.
Input: the bare dispersion eps0 [nt+2, nbatch] (float64, index n+1 holds eps0(t_n)); output:
the densities rho_kb(t_n) = -i G^<_kb(t_n, t_n) [nt+1, nbatch] (complex128).  Any real loss
built from rho with torch operations back-propagates to eps0 and, through torch, to whatever
produced eps0 (a field A(t), a hopping h(t)).  This module only marshals tensors; both
directions run in the CUDA kernels of libng.so.
"""
import torch

from . import NG_ADJ_RECORDED, NG_FP64, Func, Herm, tri


class Dyson2B(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps0, ngctx, grid, U, corrector, nbar, segment, state):
        """eps0: [nt+2, nbatch] float64 on the GPU; U: [nt+2] float64; state: dict that
        receives the forward buffers (G, Gloc, S, eps_mf) for inspection."""
        g = grid
        e0 = Func(g, values=eps0.detach().to(torch.complex128).reshape(g.nt + 2, 1, 1, g.nbatch))
        uf = Func(g, scalar=True)
        uf.val[:, 0, 0, 0] = U.to(torch.complex128)
        G = Herm(g, zero=False)
        Gl, S = Herm(g, ldk=1), Herm(g, ldk=1)
        mf = Func(g)
        if segment == NG_ADJ_RECORDED:   # keep every corrector iterate: no recomputation backwards
            ngctx.adjoint_forward(g, G, Gl, S, e0, mf, uf, corrector=corrector, nbar=nbar)
        else:
            ngctx.run_2b(g, G, Gl, S, e0, mf, uf, corrector=corrector, nbar=nbar, mats_tol=1e-14, boot_tol=1e-14,
                         precision=NG_FP64)
        diag = torch.tensor([tri(n) + n for n in range(g.nt + 1)], device=eps0.device)
        rho = -1j * G.les[diag, 0, 0, :]
        ctx.saved = (ngctx, g, G, Gl, S, e0, mf, uf, corrector, nbar, segment)
        if state is not None:
            state.update(G=G, Gloc=Gl, S=S, eps_mf=mf)
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        ngctx, g, G, Gl, S, e0, mf, uf, corrector, nbar, segment = ctx.saved
        # rho = -i G^<  =>  c(G^<) = conj(-i) c(rho) = i c(rho)
        seed = (1j * grad_rho).to(torch.complex128).contiguous()
        cG = Herm(g, zero=False)
        cS = Herm(g, ldk=1, zero=False)
        grad = torch.zeros((g.nt + 2, g.nbatch), dtype=torch.float64, device=seed.device)
        ngctx.adjoint_2b(g, G, Gl, S, e0, mf, uf, seed, cG, cS, grad, corrector=corrector, nbar=nbar,
                         segment=segment)
        return grad, None, None, None, None, None, None, None


def densities(eps0, ngctx, grid, U, corrector=3, nbar=0.5, segment=0, state=None):
    """rho_kb(t_n) for n = 0..nt, differentiable with respect to eps0.  segment: steps per
    recomputed segment of the backward pass (0: ceil(sqrt(nt - k))), or NG_ADJ_RECORDED to keep
    every corrector iterate of the forward in device memory instead."""
    return Dyson2B.apply(eps0, ngctx, grid, U, corrector, nbar, segment, state)
