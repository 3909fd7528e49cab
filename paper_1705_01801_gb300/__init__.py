"""GB300 (sm_103a) implementation of the curvilinear wave lattice-Boltzmann method of
Velasco, Munoz and Mendoza (arXiv:1705.01801): a C-ABI CUDA library (csrc/, include/lbw.h)
and its thin ctypes binding (lbw.py)."""
from . import lbw  # noqa: F401

__all__ = ["lbw"]
