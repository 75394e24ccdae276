"""GB300-native nonhydrostatic Boussinesq RK3 substep (arXiv 2502.14148).

The compute path is the CUDA library ``libocn.so`` built from ``csrc/`` and
reached through the C ABI declared in ``include/ocn.h``; ``ocn.py`` is the thin
ctypes binding.  ``inputs.py`` holds the seeded synthetic workloads.
"""
__all__ = ["ocn", "inputs"]
