"""GB300 (sm_103a) Valence-Bond quantum Monte Carlo hot path.

Jastrow-Valence-Bond wave functions (arXiv:2207.14715, Sec. 2) evaluated over walker
populations by hand-written CUDA kernels behind the C ABI of include/vbqmc.h.
"""
from . import systems  # noqa: F401

__all__ = ["systems", "vbqmc"]
