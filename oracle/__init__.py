"""Plain, slow FP64 CPU oracle for the tent-pitched Trefftz-DG method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never calls it, and it
shares no code with that path: it is written directly from the paper
(Perugia, Schoberl, Stocker, Wintersteiger, "Tent pitching and Trefftz-DG
method for the acoustic wave equation") with numpy primitives.

Modules and the passages they follow:
  quadrature  - Gauss-Jacobi rules by the Golub-Welsch eigenproblem and the
                collapsed (conical-product) rule on the reference n-simplex
                (Section 4.1: one spatial rule mapped onto the tent faces).
  basis       - exact-rational coefficients of the second-order Trefftz
                space U^p from the recursion eq. (3.1), monomial initial data
                (Section 3, Section 6.3).
  pitching    - tent pitching with the edge-slope limit (Section 2.2,
                Section 6 setup); the algorithm itself is only cited by the
                paper, the exact rule implemented is stated in the module.
  tdg         - the tent-by-tent sweep: local system eq. (4.1) plus the
                recovery terms of Section 5, Dirichlet faces from eq. (2.5),
                LU solve, outflow written at the top points (Section 4.1).
  energy      - energy E (Section 6.5), the error functional e (Section 6)
                and each tent's energy loss from eq. (2.5)/(4.1) tested with
                its own solution.
  adjoint     - the transposed tent maps, the whole space-time system and
                the wave-speed gradient through it and by differences.
  parallel    - the sweep over the independent tents of a level on several
                processes (the paper's parallel loop over a layer, Section 6).

Parity status: the pins in tests/test_oracle_*.py cover every function;
"parity unpinned" items are listed in each module header.
"""
