"""GB300 (sm_103a) MLS transfer functions for immersed-boundary markers.

Exact-MLS and fast-MLS shape functions (Spandan et al., arXiv:1805.01113,
Section 2), Euler-to-Lagrange interpolation and Lagrange-to-Euler spreading,
behind the C ABI in include/mls.h.  ``binding`` is the ctypes layer with the
same names; ``api`` wraps it for PyTorch tensors.
"""

from . import binding
from .build_ext import build, LIB

__all__ = ["binding", "build", "LIB"]
