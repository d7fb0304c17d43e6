"""GB300 (sm_103a) kernel ridge regression with random-feature preconditioning.

The compute path is the C ABI in ``include/krr.h`` implemented by the CUDA
library ``libkrr_gb300.so`` built from ``csrc/``; ``_krr`` is its ctypes
binding.  Importing this package does not load the library; importing
``paper_1611_03220_gb300.api`` (or calling ``load()``) does, and fails
loudly if it has not been built.
"""

__all__ = ["load", "build"]


def load():
    """Import the ctypes binding (raises ImportError if the library is missing)."""
    from . import _krr
    return _krr


def build(force: bool = False, verbose: bool = False) -> str:
    from .builder import build as _b
    return _b(force=force, verbose=verbose)
