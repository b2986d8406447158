"""GB300 (sm_103a) tree gravity for SMBHs in galactic nuclei.

The compute path is librv (CUDA kernels behind the C ABI in include/rv.h);
``rv`` is its Python binding.
"""
from . import rv  # noqa: F401
from .rv import Context, System, RvError  # noqa: F401
