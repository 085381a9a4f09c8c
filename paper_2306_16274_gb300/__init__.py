"""GB300-native fused non-orthogonal MRT pseudopotential lattice Boltzmann step.

The compute path is liblbm.so (hand-written CUDA for sm_103a behind the C ABI in
include/lbm.h); ``lbm`` is its Python binding.
"""
from .lbm import CONTACT_FIELDS, Batch, LBMError, Params, Simulation, estimate_bytes, lib  # noqa: F401

__all__ = ["CONTACT_FIELDS", "Batch", "LBMError", "Params", "Simulation", "estimate_bytes", "lib"]
