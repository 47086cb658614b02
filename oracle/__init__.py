"""Plain, slow, FP64 CPU oracle for the parallel-in-time KKT solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA library (``paper_2405_18964_gb300``): it
assembles sparse matrices from a generic Lagrange-basis element loop and
follows the paper's formulas step by step.

Modules
  fem      Q2-Q1 Taylor-Hood operators on a uniform square grid (Sec. 2.2),
           the winds (recirculating, the Sec. 5.2 two-vortex wind, nodal)
  kkt      all-at-once KKT matrix (Eq. FinalA), right-hand sides (zero and
           prescribed boundary velocity, Sec. 5), the block-circulant P_C and
           its exact FFT-diagonalised inverse (Sec. 3.1), FGMRES (Sec. 3.4)
  inexact  Chebyshev semi-iteration, geometric multigrid with multicolour
           SOR, the Stokes transform G_j = T^l Z_j T^r (Eq. GJTransformation),
           the commutator preconditioner P~_j, inexact Uzawa and Algorithm 3
           (Sec. 4), inner GMRES and Algorithms 1 and 2
  layout   maps between the library's full-grid storage and the reduced
           (Dirichlet-eliminated, pressure-pinned) vectors used here

Parity status: every function is pinned by a `-m "not gpu"` test against a
closed form (among them the Sec. 5.1 exact solution), an invariant, a
brute-force solve or a bound printed in the paper, except the inexact
nested preconditioners (Chebyshev / MG / Uzawa combinations), whose
intermediate values the paper never prints: those are pinned only through
convergence to their exact counterparts as iteration counts grow ("parity
unpinned" for the exact iterate values; see ``inexact``'s header).
"""
