"""CPU FP64 oracle for FD-preconditioned MINRES on isogeometric Stokes.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow, obviously correct restatement of the paper
(Montardini, Sangalli, Tani, "Robust isogeometric preconditioners for the
Stokes system based on the Fast Diagonalization method", arXiv 1712.00403):

* ``splines``     - knot vectors, Cox-de Boor recursion, Gauss quadrature (Sec. 2.1)
* ``univariate``  - univariate mass / stiffness / mixed / Nitsche matrices (Sec. 5, Appendix)
* ``kron``        - Kronecker identities and the FD solve (Sec. 2.3, Sec. 5.2, Algorithm 1)
* ``stokes``      - Taylor-Hood / Raviart-Thomas Stokes operator, P_V, P_Q (Sec. 3-5)
* ``minres``      - preconditioned MINRES (Paige-Saunders; cited in Sec. 4)
* ``gmres``       - left-preconditioned GMRES (Saad-Schultz; cited in Sec. 4) for P_T and P_C
* ``geometry``    - mapped geometry, separable approximation, P_D^G (Sec. 6, Appendix)

It shares no code with the CUDA path; the only module both sides use is the
seeded input generator ``synth``, which holds none of the method's arithmetic.

Parity status per function is stated in each module header; every function
that has no independent pin says "parity unpinned" there.
"""
