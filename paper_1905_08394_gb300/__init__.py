"""GB300 (sm_103a) engine for exact output amplitudes of random 2D-lattice
circuits held as an untruncated PEPS (arXiv:1905.08394, Guo et al.).

`binding` holds the one-to-one ctypes functions of the C ABI;
`Simulator` is a convenience wrapper that owns the context and a
torch-allocated device workspace.  Importing the package does not load the
shared library; the first call does, and fails loudly if it is missing.
"""
from .engine import Simulator  # noqa: F401

__all__ = ["Simulator"]
