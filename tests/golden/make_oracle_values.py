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


def seven_by_seven_d40_subslices():
    """4 sub-slices of the 7x7 (1+40+1) amplitude: the second and the fourth
    CZ gate of every horizontal edge have their Schmidt bit held fixed (84
    bits; every running tensor of the column sweep then has at most 2^26
    entries).  The oracle applies each held CZ as its single Schmidt term
    P_s (x) Z^s.  Many sub-slices of these circuits vanish exactly (held
    projectors leave a qubit in a basis state through runs of diagonal gates);
    candidates k = 0, 1, ... are evaluated in turn and the first four with a
    nonzero amplitude are kept.

    Bit values: two projectors P_s, P_s' on the same qubit with only diagonal
    gates (T, CZ) between them vanish unless s = s', so the values are drawn
    along each qubit's gate sequence: a held CZ reuses the value of the
    previous held projector on its lower qubit unless a non-diagonal gate
    (H, sqrt X, sqrt Y) acted since; otherwise it takes a fresh bit from
    SplitMix64(5 ^ 0x5AB + k) for sub-slice k."""
    from rqc_inputs import SplitMix64

    circ, bits = workload("7x7_d40")
    C = circ.C
    per_edge, k = {}, 0
    for g in circ.gates:
        if g.kind != "cz":
            continue
        a, b = g.qubits
        if b == a + 1 and b // C == a // C:
            per_edge.setdefault((a, b), []).append(k)
        k += 1
    fixed = sorted(o for ords in per_edge.values() for o in (ords[1], ords[3]))
    fixed_set = set(fixed)
    subs = []
    t = time.time()
    for sub in range(4):
        rng = SplitMix64((5 ^ 0x5AB) + sub)
        last = {}
        value = {}
        k = 0
        for g in circ.gates:
            if g.kind == "1q":
                if g.name in ("H", "SX", "SY"):
                    last.pop(g.qubits[0], None)
                continue
            if k in fixed_set:
                q0 = g.qubits[0]
                v = last[q0] if q0 in last else (rng.next() & 1)
                last[q0] = v
                value[k] = v
            k += 1
        vals = [value[o] for o in fixed]
        sid = sum(v << j for j, v in enumerate(vals))
        p = op.build(circ.R, circ.C, circ.gates, sliced=fixed, slice_id=sid)
        amp = op.amplitude(p, int(bits[0]))
        print(f"sub-slice {sub}: {amp} ({time.time() - t:.0f} s)", flush=True)
        subs.append({"fixed_s": vals, "amplitude": [amp.real, amp.imag]})
    return {"workload": "7x7_d40", "bitstring": int(bits[0]), "fixed_cz": fixed,
            "subslices": subs, "oracle": "oracle.peps column sweep, held CZ bits applied "
            "as single Schmidt terms (FP64)", "seconds": time.time() - t}


def seven_by_seven_d24():
    """The 7x7 lattice at depth (1+24+1) (bond dimension 8; largest running
    tensor 2^24 entries, within reach of the oracle): amplitudes of the first
    two bitstrings drawn with seed 5."""
    from rqc_inputs import make_circuit, uniform_bitstrings

    circ = make_circuit(7, 7, 24, 5)
    bits = uniform_bitstrings(49, 2, 5)
    t = time.time()
    p = op.build(7, 7, circ.gates)
    amps = op.amplitudes(p, bits)
    return {"workload": "7x7 (1+24+1), seed 5", "bitstrings": [int(b) for b in bits],
            "amplitudes": [[a.real, a.imag] for a in amps], "oracle": "oracle.peps column sweep (FP64)",
            "seconds": time.time() - t}


def eight_by_eight_d25():
    """The 8x8 lattice at depth (1+25+1) (the paper's workstation experiment;
    bond dimension 8 on every edge cut by the square partition, 16 on some
    others): the first 8 of the workload's 10000 bitstrings, by the oracle's
    square partition (its column sweep would hold 2^30-entry tensors)."""
    circ, bits = workload("8x8_d25")
    idx = list(range(8))
    t = time.time()
    p = op.build(8, 8, circ.gates)
    amps = op.amplitudes_quadrant(p, bits[idx])
    return {"workload": "8x8_d25", "indices": idx, "bitstrings": [int(b) for b in bits[idx]],
            "amplitudes": [[float(a.real), float(a.imag)] for a in amps],
            "oracle": "oracle.peps square partition (FP64)", "seconds": time.time() - t}


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "6x6_d32"
    if which == "6x6_d32":
        d = six_by_six_d32()
    elif which == "7x7_d24":
        d = seven_by_seven_d24()
    elif which == "7x7_d40":
        d = seven_by_seven_d40_subslices()
    elif which == "8x8_d25":
        d = eight_by_eight_d25()
    else:
        raise SystemExit(f"unknown set {which}")
    path = os.path.join(HERE, f"oracle_{which}.json")
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
    print(f"wrote {path} in {d['seconds']:.0f} s")
