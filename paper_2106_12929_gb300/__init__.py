"""GB300-native lattice Boltzmann stream-and-collide (arXiv 2106.12929's hot path).

The compute lives in ``liblb.so`` (CUDA C-ABI, ``include/lb.h``); this package is
the Python binding over it. Importing it does not load the library; the first
``Lattice`` does, and raises if the library was not built.
"""
from ._lib import LBError, load  # noqa: F401
from .lattice import Lattice, adam_update  # noqa: F401
from .autograd import lb_run  # noqa: F401

__all__ = ["Lattice", "LBError", "adam_update", "lb_run", "load"]
