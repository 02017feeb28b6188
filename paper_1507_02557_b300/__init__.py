"""Hybrid-mesh acoustic discontinuous Galerkin on B300 (sm_103a).

The compute path lives in the ``libdg`` shared library (C ABI, CUDA kernels);
``paper_1507_02557_b300.dg`` is its thin Python binding.  This package
initialiser deliberately imports nothing, so that ``paper_1507_02557_b300.inputs``
(seeded synthetic inputs) can be used without loading the library.
"""
