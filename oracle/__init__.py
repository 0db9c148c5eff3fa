"""FP64 CPU oracle for the moist compressible-Euler DG method with implicit
condensation (Hittmeir, Lederer, Schoeberl, von Wahl, arXiv 2305.13847).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The product path (``paper_2305_13847_gb300``) never imports, calls or links
anything here, and nothing here imports the product package: the two share no
code.  Inputs that both sides consume come only from the seeded generator
``paper_2305_13847_gb300.inputs``, which holds random draws and workload sizes
and none of the method's arithmetic.

Everything is float64 numpy.  Each function cites the section / equation of
the paper it follows.  Where the paper is silent or ambiguous the reading taken
is stated in the docstring.

Modules
-------
constants  Table 1 and the microphysics constants of Section 2.1.
thermo     Eq. (2.2), (2.3), (2.4), (2.6), (2.8), Eq. (3.4) sound speed, v_r.
basis      Gauss-Legendre rule and Lagrange basis on [-1, 1] (Section 3.1).
mesh       Structured quad/hex mesh, node and face geometry (Section 3.1).
dg         Flux, Lax-Friedrichs flux, semi-discrete operator Eq. (3.2)/(3.3),
           SSPRK(4,3) (Remark 3.1).
initial    Hydrostatic base state and warm-bubble initial state (Appendix B
           style set-ups restated for the synthetic workloads).

Parity status: every function is pinned by tests in tests/test_oracle_*.py
(closed forms, invariants, brute force, convergence rates).  The full time
step has no printed solution to compare with; beyond the invariants it is
"parity unpinned" in the sense that no external number fixes it.
"""
