"""AERO-MPPI planning step on GB300 (sm_103a): CUDA kernels behind a C-ABI.

Importing the package loads nothing; ``paper_2509_17340_gb300.aero`` loads the
CUDA library (``libaero_mppi.so``) and fails loudly if it is missing.
"""
