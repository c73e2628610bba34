"""GB300 (sm_103a) Schur-complement Low-Rank preconditioner and SLR-PCG.

Li, Xi & Saad, "Schur complement based domain decomposition preconditioners
with low-rank corrections" (arXiv 1505.04340).  The compute path is the CUDA
library built from ``csrc/`` (C ABI in ``include/slr.h``); ``slr`` is its
Python binding.
"""
from .slr import SLR, SLRError, dd_order, load  # noqa: F401
