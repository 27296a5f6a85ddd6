"""FP64 CPU oracle for the FlashMP subdomain-transform preconditioner.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and
its Python binding) imports or calls this package; only the tests, the
``smoke()`` self-check and the CPU-baseline leg of ``bench.py`` do.

It is a plain, slow, direct restatement of the method in float64:

* ``yee``        sparse incidence matrices (gradient, curl, divergence), the
                 double-curl operator and the system matrix (Eq. 5, Eq. 7).
* ``transforms`` the 1-D DCT-II / DST-I tables from the SVD of the difference
                 operator (Eq. 8) and the tensor-product axis transforms
                 TrX/TrY/TrZ (Eq. 9).
* ``box``        the subdomain exact solve: transform G, per-mode 3x3 solve
                 (Eq. 12) by a dense linear solve, inverse transform
                 (Algorithm 1, exact_solve).
* ``ras``        restricted additive Schwarz over overlapping boxes (Sec. II-B).
* ``krylov``     restarted flexible GMRES and BiCGSTAB (Sec. IV-A).
* ``cn``         the Crank-Nicolson step (Eqs. 2-4).
* ``complexity`` the operation and memory counts of Sec. III-B / Table 2.

Every function cites the paper passage it follows. The oracle shares no code
with the CUDA path; both take their inputs from
``paper_2508_07193_b300.workloads`` (random draws only).
"""
