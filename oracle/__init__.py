"""FP64 CPU oracle for the discrete-DtN absorbing boundary condition (Wu & Li).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path; the only common module is the seeded input
generator ``paper_1908_02456_gb300.inputs``, which holds no arithmetic of the
method.

The oracle is plain, slow and follows the paper's own formulas in the paper's
order, in float64 / complex128:

* ``lattice``     -- grid, stencil, index sets I, Gamma (eq:25), Sigma (App. A),
                     the blocks H_{I,I}, H_{Gamma,Sigma} (Sec. 2, eq:22/eq:32).
* ``dtn``         -- the DtN map K(s) of eq:17, two independent routes: the
                     definition itself on a truncated exterior (brute-force Schur
                     complement) and the App. A formula eq:eval with the free
                     lattice Green's function (App. D) from a periodic FFT lattice;
                     plus the 1D closed form.
* ``coefficients``-- order-0 (M = K(s0), Thm 3.1) and order-1 (A, B, Q of Thm 3.2)
                     ABC matrices.
* ``propagate``   -- the reduced dynamics eq:dynamics0 / eq:dynamics1, the
                     degree-4 Taylor propagator (eq:21 with its signs read as
                     sum_k (dt L)^k / k!), the density-dependent mean field, its
                     energy functional (whose rho-derivative is the potential) and
                     the norm / Lyapunov / energy diagnostics.
* ``adjoint``     -- reverse-mode gradient of the absorbed probability with
                     respect to the potential, written from the same Taylor form.
* ``exact``       -- the free Gaussian packet of eq:15 (the reference solution of
                     the paper's 3D experiment).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants proved in the paper, brute force on tiny inputs or the
paper's printed values; the internal building blocks (names with a leading
underscore, and small pieces such as ``Box.diag_weight``, ``order2_end`` or
``all_offsets``) through the pinned functions that call them.  No function here
is "parity unpinned".
"""
