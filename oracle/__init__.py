"""FP64 CPU oracle of the staggered-grid real-valued P_N system.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that the
CUDA library is checked against.  Only the test-suite (tests/), the smoke
check in __graft_entry__.py and the CPU-baseline leg of bench.py may import,
call or execute anything here.  The CUDA library and its Python binding never
import it and share no code, table or helper with it.

Contents (each module cites the passages of Koerner, Portsmouth and Jakob,
"P_N-Method for Multiple Scattering in Participating Media", EGSR 2018, that it
follows):

* sh.py       -- SH bases and the angular coupling matrices by quadrature
* printed.py  -- the appendix's final real P_N equations, term by term
* grid.py     -- staggered (parity) placement of the unknowns, interpolation
* pn.py       -- explicit CSR assembly, matrix-free FP64 apply, direct solve,
                 CG on the normal equations (CGLS), residuals
* gmres.py    -- restarted GMRES in FP64 (a plain Krylov solve of A u = Q)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, library routines, invariants or brute force.
"""
