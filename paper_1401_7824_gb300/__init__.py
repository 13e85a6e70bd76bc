"""GB300 (sm_103a) implementation of inexact spectral deferred corrections
(arXiv:1401.7824): a C-ABI CUDA library (include/isdc.h, libisdc.so) and a
thin Python binding with the same entry-point names."""
from .isdc import *  # noqa: F401,F403
from .isdc import Isdc, IsdcError, load, library_path  # noqa: F401
