"""CPU FP64 oracle for the vielbein LB + Cahn-Hilliard step (arXiv:1904.10070).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The CUDA library and
its Python binding never import it and never fall back to it.

Pinned functions (each checked by a ``-m "not gpu"`` test against what the paper or the
mathematics fixes, never against itself): velocities, weights, kernel_K, kernel_Kt, feq,
moments, laplace_beltrami, face_values/flux_difference, rhs, step, totals,
interface_length, and the closed forms in ``closed_forms``.
"""
