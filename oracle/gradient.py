"""Reference gradients of the self-consistent second-Born run (oracle; test infrastructure only).

The paper has no adjoint.  The gradient that a discrete adjoint must reproduce is the
derivative of the executed discrete algorithm (Sec. "Hubbard chain" driver: Matsubara loop,
bootstrapping, predictor and fixed corrector passes per time step) with respect to its
inputs.  The oracle obtains it numerically from the plain forward algorithm:

  * fd_derivative: the fourth-order central difference
        f'(x) ~ [f(x - 2d) - 8 f(x - d) + 8 f(x + d) - f(x + 2d)] / (12 d),
    exact for polynomials of degree <= 4; its truncation error is d^4 f^(5)/30 and its
    rounding error about 1.5 eps |f| / d, so d = 1e-3 resolves the derivative of a smooth
    O(1) loss to about 1e-11 absolute (the converged setup loops add their stopping error / d);
  * kinetic_energy: the loss E_kin(t_N) = (1/N_k) sum_k Re Tr[rho_k(t_N) eps0_k(t_N)],
    rho_k = -i G_k^<(t_N, t_N) (Sec. "GW for the translationally invariant Hubbard model",
    observables), from oracle.drivers.run_2b.
"""
import numpy as np

from . import drivers, observables


def fd_derivative(f, x0, i, delta=1e-3):
    """d f / d x_i at x0 by the fourth-order central difference (x0 is not modified)."""
    vals = []
    for s in (-2, -1, 1, 2):
        x = np.array(x0, dtype=float, copy=True)
        x[i] += s * delta
        vals.append(f(x))
    return (vals[0] - 8.0 * vals[1] + 8.0 * vals[2] - vals[3]) / (12.0 * delta)


def kinetic_energy(eps0, U, nt, ntau, beta, h, W, corrector=3, mu=0.0, nbar=0.5, tol=1e-14):
    """E_kin(t_nt) of the self-consistent second-Born run with bare dispersions eps0 (list of
    oracle Funcs, one per k-point) and interaction U (scalar Func); setup loops converged to tol."""
    st = drivers.run_2b(eps0, U, nt, ntau, beta, h, W, mu=mu, nbar=nbar, corrector=corrector, mats_tol=tol,
                        boot_tol=tol)
    return observables.kinetic_energy(nt, st.G, eps0)
