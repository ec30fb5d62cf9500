"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the bench.

This package draws random numbers, builds grids and packs arrays.  It holds none of
the CROM method's arithmetic: no decoder evaluation, no PDE update, no projection.
"""
from .gen import *  # noqa: F401,F403
