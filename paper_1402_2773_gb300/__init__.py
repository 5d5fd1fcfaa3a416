"""GB300 (sm_103a) Noisy Gradient Descent Bit-Flip LDPC decoding.

The decoder itself is the CUDA library ``libngdbf.so`` behind the C ABI of
``include/ngdbf.h``; ``paper_1402_2773_gb300.ngdbf`` is its ctypes binding.
``paper_1402_2773_gb300.workload`` draws seeded synthetic codes and frames.
"""
from ._build import build_all, build_cuda  # noqa: F401

__all__ = ["build_all", "build_cuda"]
