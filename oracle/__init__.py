"""CPU FP64 oracle for the condensed H(div)-HDG hp-multigrid solver.

TEST INFRASTRUCTURE ONLY.  This package is the parity reference for the CUDA
library: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it.  The product path never calls
it, and it shares no code with the CUDA library (``paper_2303_06762_gb300``):
the two are separate implementations of the same published method, in
different languages and along different computational routes, and neither
imports the other.  Only the seeded input generators in ``workloads`` serve
both.

What it computes (G. Fu & W. Kuang, "hp-multigrid preconditioner for a
divergence-conforming HDG scheme for the incompressible flow problems"):

* ``topology``   — facets, orientations, interior-facet numbering (Section 2).
* ``quadrature`` — collapsed Gauss–Jacobi rules on triangles, Gauss–Legendre
  on facets.
* ``spaces``     — W_h^k, the Raviart–Thomas space RT_k, the facet space and
  its orthonormal Legendre basis, built in physical coordinates (Section 2).
* ``hdg``        — the local system of eq. stWeak, static condensation onto the
  skeleton unknowns (Section 3.2), the augmented-Lagrangian operator A^ε
  (eq. stALform), global assembly, the exact discrete solution by a sparse
  direct solve of the condensed saddle point (eq. stOptForm), recovery,
  error norms and the post-processing of eq. stPost.
* ``cr``         — an independent Crouzeix–Raviart assembly of eq. equivCRstWeak
  with the RT0 reconstruction Π^RT (eq. CR_2RT0) and the interpolation Π^CR
  (eq. RT0N1_2CR), for Theorem 3.1 and Lemma 3.2.
* ``mg``         — vertex patches and block Gauss–Seidel smoothing
  (eq. bjac, Section 5 settings), the averaging transfer (eq. avgOpt) with the
  harmonic-extension correction (eqs. div-transfer, harmonic-ex), the
  h-multigrid of Algorithm 1 and the hp-multigrid of Algorithm 2.
* ``krylov``     — flexible GMRES and the augmented-Lagrangian Uzawa iteration
  (eq. stOpEq-ALU).

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
property the paper or the mathematics fixes (see tests/test_oracle_*.py); the
paper's own error tables are missing from its text, so numeric error values
are pinned through convergence slopes, not printed values.
"""
