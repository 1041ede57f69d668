"""GB300 (sm_103a) hot path of GOCP ADAPT-VQE (arxiv 2607.15906).

The compute path is the CUDA library under ``csrc/`` behind the C ABI of
``include/gocp.h``; this package marshals arguments to it (ctypes) and uses
PyTorch only for device memory and streams.  There is no CPU fallback:
``load()`` raises when the library is missing.
"""

from ._lib import GocpError, load, launch_count, library_path  # noqa: F401
from .problem import Problem, exact_sum  # noqa: F401

__all__ = ["GocpError", "Problem", "exact_sum", "load", "launch_count", "library_path"]
