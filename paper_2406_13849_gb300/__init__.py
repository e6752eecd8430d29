"""GB300-native nested-geometry particle tracking (arXiv 2406.13849 hot path).

The compute path is the C-ABI library built from ``csrc/`` (declared in
``include/trk.h``); ``native`` is its thin Python binding and ``inputs``
generates seeded synthetic geometry descriptions and ray sets.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "native", "build"]
