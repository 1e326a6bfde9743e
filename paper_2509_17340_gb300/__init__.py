"""AERO-MPPI planning step on GB300 (sm_103a): CUDA kernels behind a C-ABI.

Importing the package loads nothing; ``paper_2509_17340_gb300.aero`` loads the
CUDA library (``libaero_mppi.so``) and fails loudly if it is missing.
``use_checked_build()`` before that import selects the checked build
(``libaero_mppi_checked.so``: the kernels check the indices they rely on and
``sync_status`` reports a failed check).
"""
import sys

_library = "libaero_mppi.so"


def use_checked_build() -> None:
    """Make ``.aero`` load ``libaero_mppi_checked.so``; call before importing it."""
    global _library
    if __name__ + ".aero" in sys.modules:
        raise RuntimeError("paper_2509_17340_gb300.aero is already loaded with " + _library)
    _library = "libaero_mppi_checked.so"


def library_name() -> str:
    return _library
