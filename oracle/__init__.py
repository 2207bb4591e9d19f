"""CPU FP64 oracle for the PEPS amplitude path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs
of `bench.py` may import anything from here.  The product path (the CUDA
library under `paper_1905_08394_gb300/` and its Python binding) never imports,
links or runs this package, and this package never imports the product.  The
two share nothing but the seeded input generators in `rqc_inputs`.

Two independent computations of the same definition, a_x = <x| C |0...0>
(the overlap of the paper's main-text equation for <tau|psi>):

* `statevector` (O2): a dense complex128 state vector, gates applied one by
  one in circuit order.  Practical up to 5x5 (2^25 amplitudes, 512 MiB).
* `peps` (O3): a PEPS of rank-5 site tensors built gate by gate exactly as the
  paper's single-qubit absorption and two-qubit split-and-bundle equations say,
  projected on the bitstring, and contracted exactly site by site in the order
  of the supplementary "exact computation of the overlap" equations (row
  sweep), or the same sweep transposed (column sweep).  All FP64, no
  renormalisation, no truncation.

Parity status: both are pinned by the CPU tests in `tests/test_oracle.py`
(closed forms, brute force, invariants, planted mistakes) and
`tests/test_complexity.py` (the paper's memory figures); the tie rule that the
held-bit contraction relies on is checked against O2/O3 in `tests/test_ties.py`
and `tests/test_slicing.py`.  Nothing here is "parity unpinned".
"""
