"""Plain, slow FP64 CPU oracle for the contour Dyson time-stepper (NESSi, arXiv:1911.01211).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.  It shares no code with the CUDA path.

Every function follows the paper's definitions in the paper's order and notation,
written out with plain numpy loops and library primitives (dot products, dense
solves).  There is no blocking, fusion or reordering beyond the definitions.

Modules
-------
weights      integration weights P, D, I, BDF a, Gregory w, boundary-convolution R,
             extrapolation C (Sec. "Basic integration and differentiation rules")
contour      full-storage contour functions with the hermitian-conjugate accessors
             (Eqs. hermconjg, Cretmod, kmsbound_keld)
freegf       closed-form free Green's functions for a constant Hamiltonian
             (Sec. "Implementation: Free Green's functions", Eq. G0_free)
conv         the discrete convolution pieces C^M_1,2, C^R, C^tv_1,2,3, C^<_1,2,3
             (Sec. "Numerical details: convolution integrals", Eqs. cm1-cles3)
dyson        dyson_mat / dyson_start / dyson_timestep (serial and mixed schedules)
             (Sec. "Implementation: dyson", Eqs. vdiff_start, MBCVSAMx_t, MBCVSAMx_cc_*)
bubble       second-Born self-energy, Hartree mean field, k-point reduction
             (Eq. sigma_hubb_2b, Eqs. def_bubble1/2)
extrap       extrapolate_timestep and distance_norm2 (Appendix "Contour function utilities")
drivers      fixed-Sigma Dyson solve and the self-consistent second-Born loop
             (Sec. "Hubbard chain": Matsubara loop, bootstrapping, predictor-corrector)
observables  density matrix, particle number, kinetic and Galitskii-Migdal energies

Parity pins: every function is pinned by tests under ``tests/test_oracle_*.py``
against values the paper prints, closed forms, invariants or brute force.
The second-Born dynamics of a self-consistent run has no exact solution: it is
pinned only through invariants (conservation laws, KMS, hermiticity) and through
its building blocks; see the header of ``drivers``.
"""
