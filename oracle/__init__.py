"""CPU FP64 oracle for the unrolled COSMO iteration -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import or run this package.  The product path (the C-ABI
library and its Python binding) never calls it and shares no code with it;
the only shared module is ``synth`` (seeded problem data, no solver maths).

Contents
  linalg.py  dense LDL' (direct-mode KKT solve, Sec. 2.3) and a Householder +
             implicit-QR symmetric eigensolver (used by Eq. psd-proj)
  cones.py   zero / nonneg / box / SOC / PSD projections and their VJPs,
             including the Daleckii-Krein rule, Eqs. (psd-cotangent-dk, lowner)
  cosmo.py   Sec. 2.2 iteration (Eq. cosmo_linear_system .. cosmo_projection)
             unrolled K times, residuals (App. E), loss, and the hand-written
             reverse pass through the formed KKT system.

Pins (tests/test_oracle_*.py): closed-form SDP values (max-cut and Lovasz
theta of cycles, complete and empty graphs), brute-force max-cut bounds,
projection invariants (idempotence, Moreau decomposition, orthogonality,
nonnegative spectrum), LAPACK comparisons (numpy eigh / solve), DK special
cases and DK against torch's eigh autograd on separated spectra, the implicit
rule of Eq. (grad_rho) against the KKT route and finite differences, central
finite differences of the whole unrolled map, and fixed points at planted
optimal solutions.  Parity unpinned: nothing (every function above has at
least one pin that does not re-use its own formula).
"""
from . import linalg, cones, cosmo  # noqa: F401
