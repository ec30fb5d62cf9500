"""FP64 CPU oracle of the CROM latent-space step.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never calls it and shares no code with it.
"""
from .crom_oracle import *  # noqa: F401,F403
