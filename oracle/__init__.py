"""CPU oracle for the locally compressed MFS (test infrastructure only).

A plain, slow, FP64 numpy implementation of what the GPU library computes,
written from the paper's equations and algorithms, each function citing the
passage it follows.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import it; the library never does, and this package
imports nothing from the library.  The two share only the seeded workload
generators in `workloads.py` (geometry and random draws, no method
arithmetic).

Pins (see tests/test_oracle_*.py): closed-form single-disk resistance and
mobility (Stokeslet + potential dipole for translation, rotlet for rotation),
kernel symmetry, exact identity matvec for an isolated pair (Algorithm 3,
Step 2b), reduction to one-body preconditioning without contacts (eqs.
(resistance) and (2esysprec)),
symmetric positive-definite two-disk resistance matrices, mirror-symmetry
zeros, two-way resistance/mobility consistency (Sec. 6.1), a dense direct
solve of the same square system, and convergence toward a fine brute-force
MFS on two and three disks.

Parity unpinned: polydisperse pair geometry (limiting points for unequal
radii, rolling radius of the peanut) has no counterpart in the paper; it is
pinned only by the radius-a closed forms and by brute force.  GMRES iteration
counts are not pinned (the paper's 47 iterations are context only).
"""
