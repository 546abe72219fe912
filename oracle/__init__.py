"""Plain, slow CPU FP64 oracle of the RBF-FD surface Laplacian path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (no kernels, headers, helpers, tables or
pre/post-processing); the only common module is the seeded input generator
``paper_1404_0812_gb300.workloads``, which holds none of the method's
arithmetic.

Each function follows the paper (Shankar, Wright, Kirby, Fogelson, "A Radial
Basis Function (RBF)-Finite Difference (FD) Method for Diffusion and
Reaction-Diffusion Equations on Surfaces") step by step, in float64, with
numpy / LAPACK calls as the only library primitives (an eigenvalue routine, a
dense solve, a sort).  Parity status per function is stated in its module
docstring; the pins live in ``tests/test_oracle_*.py``.
"""
