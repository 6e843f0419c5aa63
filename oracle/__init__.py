"""Plain FP64 CPU oracle for the Stokes Krylov/AMG solve phase.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library may import,
call or execute this package; only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with
the CUDA path: it reads the same seeded inputs (``stokes_inputs``) and
nothing else.

Every step follows the paper (Demidov, Mu, Wang, "Accelerating linear
solvers for Stokes problems with C++ metaprogramming") in the order its
text gives, written for readability, not speed:

* ``bsr``     -- CSR / block-CSR containers and products (Section 4,
                 the CSR vs block-valued worked example).
* ``amg``     -- smoothed-aggregation AMG with SPAI0 relaxation and the
                 V-cycle (Section 2.1, Listing "composition"; Section 4).
* ``krylov``  -- right-preconditioned BiCGStab and GMRES(m).
* ``schur``   -- Schur pressure correction, Eq. SchurPC with the
                 approximation Eq. SchurApprox.
* ``adjoint`` -- adjoint solve and sampled outer-product gradient.

Parity status: every function is pinned by a closed form, an invariant
or a brute-force/dense check in ``tests/test_oracle_*.py`` except the
mixed-precision forms, which the oracle does not model (it is FP64 only):
their parity is judged by the FP64 true residual alone.
"""
