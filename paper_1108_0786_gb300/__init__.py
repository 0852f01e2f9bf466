"""GB300-native coupled D3Q19 lattice Boltzmann / rigid-body swimmer step.

The compute path lives in ``csrc/`` (CUDA for sm_103a plus a C ABI declared
in ``include/lbm.h``); ``lbm`` is the thin ctypes binding over that library.
Importing the package does not load the CUDA library: ``Lattice`` (and
``load_library``) load it on first use and raise if it is missing.
"""
from .workloads import Scenario  # noqa: F401

__all__ = ["Scenario", "Lattice", "load_library", "build"]


def __getattr__(name):
    if name in ("Lattice", "load_library", "LbmError"):
        from . import lbm
        return getattr(lbm, name)
    if name == "build":
        from ._build import build
        return build
    raise AttributeError(name)
