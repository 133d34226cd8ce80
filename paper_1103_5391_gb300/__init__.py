"""GB300 hot path of time-step-targeting DMRG with Krylov time evolution (arXiv:1103.5391).

The compute lives in the C-ABI library libtdmrg.so (hand-written sm_103a CUDA,
declared in include/tdmrg.h); `tdmrg` is its argument-marshalling binding.
"""
from . import tdmrg  # noqa: F401
