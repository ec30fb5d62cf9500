"""CROM (arXiv 2206.02607) online latent-space time step for GB300 (sm_103a).

The compute lives in libcrom.so (CUDA kernels behind the C ABI of include/crom.h);
``paper_2206_02607_gb300.crom`` is the ctypes binding and ``build()`` compiles the
library in-tree with nvcc.
"""
from .build import build  # noqa: F401
