"""Seeded synthetic inputs for the superblock hot path.

This package holds no arithmetic of the method: it only draws random sector
tables, random operator blocks and random wave functions with the shapes,
sparsity (which sector blocks exist) and value scales of time-step-targeting
DMRG superblocks.  Both the CUDA path and the CPU oracle consume it.
"""
from .sectors import SyntheticSuperblock, gaussian_block_sectors, make_synthetic, chain_config, ladder_config  # noqa: F401
