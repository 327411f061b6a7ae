"""GB300-native high-order gas-kinetic scheme (HGKS), arXiv 2207.01173.

The solver is the CUDA library libhgks.so behind the C-ABI in include/hgks.h;
`paper_2207_01173_gb300.hgks` is its thin Python binding.
"""
from .hgks import (BC_EXTERNAL, BC_PERIODIC, BC_WALL, FP64, MIXED, MIXED_T64, VISC_CONSTANT, VISC_POWER, Batch, HgksError, Solver,  # noqa: F401
                   flop_model, footprint_bytes, fp64_probe, lib, library_path)
