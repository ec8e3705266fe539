"""GB300-native Chebyshev-Jacobi (CJM) solver: C-ABI library libcj.so + ctypes binding.

The library is loaded on first use by the functions in :mod:`.cj`; building it is
``paper_1705_00103_gb300.build.build()``.
"""
from . import build  # noqa: F401
from .cj import *  # noqa: F401,F403
