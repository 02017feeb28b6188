"""FP64 CPU oracle for the hybrid-mesh acoustic DG method (arxiv 1507.02557).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (the two meet only through the seeded inputs of
``paper_1507_02557_b300.inputs``).

It is a plain, slow restatement of the paper's discretisation in numpy, in
float64, each step citing the section / equation / algorithm it follows:

* ``jacobi``   Jacobi polynomials and Gauss-Jacobi / Gauss-Lobatto rules.
* ``rules``    cubature rules on the reference elements (Sec. 2.1, 2.3).
* ``elements`` reference elements: bases of Sec. 2.1 and their operators.
* ``mesh``     vertex maps, geometric factors, face matching.
* ``dg``       right-hand side of Eq. (skewform) / strong form, LSRK(5,4),
               energy, local time steps (Eq. dtK), multi-rate levels.
* ``constants`` trace and Markov constants of Appendix B.

Functions whose result has no independent pin say "parity unpinned" in their
docstring.
"""
