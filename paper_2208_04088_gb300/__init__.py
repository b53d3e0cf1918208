"""GB300 (sm_103a) solver for the solid lattice Boltzmann method with local
Dirichlet and Neumann boundary rules (Faust, Schlueter, Mueller, Mueller 2022).

The computation lives in the C-ABI library ``liblbm.so`` (``include/lbm.h``,
sources in ``csrc/``); ``_native`` is its ctypes binding and ``workloads``
states the synthetic benchmark problems.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "native"]


def __getattr__(name):
    if name == "native":
        from . import _native
        return _native
    raise AttributeError(name)
