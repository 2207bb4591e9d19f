"""Writes the FP64 oracle amplitudes that the full-size GPU tests compare
against (the oracle is too slow to run inside every test at these sizes).
Calls only oracle/ and the seeded input generators.

    python tests/golden/make_oracle_values.py 6x6_d32
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import peps as op  # noqa: E402
from rqc_inputs import workload  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def six_by_six_d32():
    """8 of the 512 bitstrings of the 6x6 (1+32+1) batch: members 0, 21, 42, 63
    of group 0 and of group 5 (prefix = columns 0-2)."""
    circ, bits = workload("6x6_d32")
    idx = [0, 21, 42, 63, 320, 341, 362, 383]
    p = op.build(circ.R, circ.C, circ.gates)
    t = time.time()
    amps = op.amplitudes_with_prefix(p, bits[idx], prefix_cols=3)
    return {"workload": "6x6_d32", "indices": idx,
            "bitstrings": [int(b) for b in bits[idx]],
            "amplitudes": [[float(a.real), float(a.imag)] for a in amps],
            "oracle": "oracle.peps column sweep with prefix reuse (FP64)",
            "seconds": time.time() - t}


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "6x6_d32"
    if which == "6x6_d32":
        d = six_by_six_d32()
    else:
        raise SystemExit(f"unknown set {which}")
    path = os.path.join(HERE, f"oracle_{which}.json")
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
    print(f"wrote {path} in {d['seconds']:.0f} s")
