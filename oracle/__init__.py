"""FP64 CPU oracle for the explicit local space-time adaptive monodomain step.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it: every formula here is restated from
the paper (Ogiermann, Balzani, Perotti, "An Explicit Local Space-Time Adaptive
Framework for Monodomain Models in Cardiac Electrophysiology") in plain numpy,
in the order and notation of the paper, without blocking or fusion.

Modules
  basis    Gauss-Legendre nodes, Lagrange basis (Sec. 2.1, GL-collocated ansatz)
  forest   forest-of-trees h-refinement on a box slab, 2:1 balance, AMR (Sec. 2.2, Alg. 1)
  sipg     SIPG operator by quadrature assembly and by a matrix-free apply
           (Eq. monodomain-primal-formulation, Eq. monodomain-numerical-flux),
           Gershgorin CFL (Eq. cfl-monodomain), Kelly-type indicator (Eq. dg-error-estimate)
  ionic    Aliev-Panfilov cell model (not in the paper; published two-variable model)
  lts      forward Euler / exponential update, Algorithm 1 (A-MQ-S-LTS),
           RV-T temporal indicator (Eq. ratti-veroni-temporal), substeps (Eq. num-substeps),
           local activation times (Sec. 3.3)

Parity status: every function is pinned by the tests in ``tests/test_oracle_*.py``
(closed forms, symbolic brute force, invariants).  The two indicator *readings*
(where W_F sits in Eq. dg-error-estimate; the Bochner norm's quadrature) are pinned
to their stated definitions, not to a value printed in the paper, which prints none.
"""
