"""GB300 (sm_103a) library for the openQ*D Dirac operator with C* boundaries.

The compute path is the CUDA library ``libqxd.so`` behind the C ABI of
``include/qxd.h``; ``qxd`` is its thin Python binding.
"""
from . import build, qxd  # noqa: F401
from .qxd import Lattice, QxdError  # noqa: F401

__all__ = ["build", "qxd", "Lattice", "QxdError"]
