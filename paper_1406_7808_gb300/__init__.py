"""Segmental-refinement full multigrid (SR-FMG) for the 3D Poisson problem on GB300.

The solver runs as hand-written sm_103a CUDA kernels behind a C ABI
(``include/srfmg.h``); ``paper_1406_7808_gb300.srfmg`` is the thin Python
binding over that library.  Importing this package loads nothing; the CUDA
library is opened on first use of the binding, which raises if it is missing.
"""
__all__ = ["inputs", "srfmg"]
