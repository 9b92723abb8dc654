"""GB300 (sm_103a) exact frequent-episode counting and level-wise mining.

The compute path is libfem.so (CUDA kernels behind the C ABI in
include/fem.h); ``binding`` marshals arguments to it with ctypes.  Importing
``binding`` raises ImportError when the library has not been built: there is
no CPU fallback.
"""
from . import build  # noqa: F401  (nvcc build of libfem.so)


def load():
    """Imports and returns the ctypes binding (builds nothing)."""
    from . import binding
    return binding
