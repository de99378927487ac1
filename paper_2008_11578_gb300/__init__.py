"""GB300-native (sm_103a) ORCA step for pedestrians and autonomous vehicles.

The hot path (grid binning, k-nearest neighbours, ORCA half-planes with
responsibility factors, per-agent velocity LP with least-penetration
fallback, integration) lives in liborca (``csrc/``), a C-ABI CUDA library.
This package builds it (``build()``) and binds it (``api``).
"""
from . import scenes  # noqa: F401
from ._lib import LIB_PATH, OrcaError, build, load  # noqa: F401

__all__ = ["scenes", "build", "load", "OrcaError", "LIB_PATH"]
