"""Plain FP64 CPU oracle of the implicit truncated LISL Scheme 2 with Howard policy iteration.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that the CUDA library
is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import it; the library itself never imports, links or calls anything in here, and this
package shares no code with the library (its inputs come from the `workloads` generators,
which hold none of the scheme's arithmetic).

Modules:
  lisl       - Scheme 2 stencils with boundary truncation, row assembly, policy improvement,
               Howard policy iteration with a sparse direct solve, implicit time stepping.
  multigrid  - bilinear prolongation, full-weighting restriction, Galerkin hierarchy,
               damped-Jacobi V-cycle, grid/algebraic complexities.
"""
