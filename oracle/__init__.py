"""Plain FP64 CPU oracle of additive-multigrid MPCG (test infrastructure).

This package is the slow, obviously-correct reference that the CUDA path is
checked against.  It is test infrastructure only: ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it; the library never does, and the two share
no code (only the seeded input generators of
``paper_2402_12833_gb300.problems``, which hold none of the method's
arithmetic).

Modules
  operators  - stencil -> CSR, prolongations (Section 2.1), Galerkin products
  mg         - the additive MG level corrections (Eq. 2, Eq. 3) as columns
  mpcg       - Algorithm 1 with the truncated window, pseudo-inverse, drop rule
  pcg        - textbook additive-MG PCG, used only as an independent pin
  ssor       - multicoloured SSOR and the multiplicative V-cycle (Section 3's comparison)
  amg        - an algebraic hierarchy by smoothed aggregation (Section 2.1's agglomeration)
"""
