"""PDHCG-II for convex QP on B300 (sm_103a): C-ABI CUDA library + thin Python binding.

The solver itself lives in ``csrc/`` (hand-written CUDA behind the C ABI of
``include/pdhcg.h``); ``pdhcg.py`` marshals arguments to it with ctypes.
``workloads.py`` holds the seeded synthetic problem generators.
"""
__all__ = ["pdhcg", "workloads"]
