"""B300-native (sm_103a) per-voxel visibility histograms and TGV primal-dual solver.

The compute path is the CUDA library ``libtgv.so`` (C-ABI in include/tgv.h);
``paper_2107_14790_b300.tgv`` is its ctypes binding.  Importing this package
does not load the library; the first ``tgv_*`` call does, and raises ImportError
if it has not been built.
"""
from . import tgv  # noqa: F401
from .tgv import Domain, TgvError  # noqa: F401

__all__ = ["tgv", "Domain", "TgvError"]
