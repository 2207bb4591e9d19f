"""GB300 (sm_103a) engine for exact output amplitudes of random 2D-lattice
circuits held as an untruncated PEPS (arXiv:1905.08394, Guo et al.).

`binding` holds the one-to-one ctypes functions of the C ABI;
`Simulator` is a convenience wrapper that owns the context and a
torch-allocated device workspace.  Importing the package does not load the
shared library; the first call does, and fails loudly if it is missing.

Batches of amplitudes: `Simulator.amplitudes(bits, precision="fp16x3",
scheme="quadrants", prefix_cols=..., prefix_group=...)`; `autotune.tune`
picks the contraction order and tile options for a batch.

One amplitude too large for one contraction (7x7 (1+40+1)): slice it.

    ss = slicing.choose_quadrants(sim.h, circ, ws_budget, x=x)   # cut CZs
    ids = slicing.consistent_slice_ids(circ, ss.sliced_cz, x)     # slices that can be nonzero
    amp = sim.amplitudes([x], scheme="quadrants", precision="fp16x3",
                         sliced_cz=ss.sliced_cz, slice_ids=ids)   # FP64 sum over them

Across ranks, `distributed.rank_slice_ids` splits `ids` and
`distributed.allreduce_sum_c128` adds the partial amplitudes.
"""
from .engine import Simulator  # noqa: F401

__all__ = ["Simulator"]
