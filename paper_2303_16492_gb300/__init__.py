"""GB300-native block-randomized stochastic tensor-ring solver (TR-BRSGD /
TR-ScaledBRSGD of arXiv 2303.16492).

The compute path is libtrsgd.so (hand-written sm_103a CUDA behind the C-ABI in
include/trsgd.h); ``api`` is its Python binding and ``synth`` the seeded
synthetic input generators.
"""
from . import _abi  # noqa: F401

__all__ = ["api", "synth", "build"]
