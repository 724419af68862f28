"""GB300 (sm_103a) matrix-based visibility simulator after arXiv:2312.09763.

The computation runs in the CUDA library ``libmatvis_gb300.so`` behind the
C-ABI of ``include/matvis.h``; :mod:`.binding` marshals arguments into it
(PyTorch supplies device memory through its caching allocator, and streams).
There is no CPU fallback: importing :class:`Simulator` without the built
library raises.
"""
from .binding import Simulator, MatvisError, load_library, perturb_sky, redundancy_plan  # noqa: F401

__all__ = ["Simulator", "MatvisError", "load_library", "perturb_sky", "redundancy_plan"]
