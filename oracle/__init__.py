"""FP64 CPU oracle for inexact spectral deferred corrections (arXiv:1401.7824).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import or run this package.
The CUDA product path never imports it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
