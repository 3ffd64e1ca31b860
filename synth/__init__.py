"""Seeded synthetic inputs shared by the FP64 oracle tests and the GPU path.

Only random draws and workload descriptions live here; no step of the
assimilation method is computed in this package.
"""
from . import philox, configs  # noqa: F401
