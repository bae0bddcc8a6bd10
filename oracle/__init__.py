"""Plain, slow, obviously correct FP64 CPU oracle of the Neuberger-Dirac hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or run anything in this package.  The GPU library
(``paper_1010_5636_gb300``) never imports it and shares no code with it; the two meet
only through the seeded input generators in ``synth``.

Modules (each function cites the part of the paper it follows):
  wilson     -- Q = gamma5 D_W and the pseudofermion force (plain C, scalar loops), Sec. 2.1
  geometry   -- lexicographic / even-odd site tables and neighbour tables
  zolotarev  -- Zolotarev rational approximation of sign(x) (mpmath, 40 digits)
  mscg       -- multi-shift conjugate gradient with error-controlled stopping
  lowmodes   -- lowest modes of Q^2, Rayleigh-Ritz of Q, residues, kappa_+- (Sec. 2.3)
  overlap    -- deflated sign(Q) and the Neuberger-Dirac operator (Sec. 2.2, 2.3)
  force      -- the force of phi^dagger (Q^2)^{-1} phi and finite-difference helpers

Parity pins: every function is checked in tests/test_oracle_*.py against something
other than itself (closed forms, invariants, dense diagonalisation, brute force).
Functions without such a pin say "parity unpinned" in their docstring.
"""
