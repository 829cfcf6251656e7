"""GB300 library for batched implicit-Euler time stepping of the 2D eddy-current
FE model across MLMC samples and Parareal slices (Hahn & Schoeps, arXiv
2507.19246).

The compute path is the CUDA library ``_lib/libmqs.so`` behind the C ABI of
``include/mqs.h``; ``paper_2507_19246_gb300.mqs`` is its ctypes binding.
There is no CPU fallback: using the binding without the built library raises.
"""
__all__ = ["build", "mqs"]
