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


def _consistent_values(circ, held, x, seed):
    """Values for the held CZ bits that no tie forces to zero (input recipe).

    A held CZ puts P_s on its lower-index qubit and Z^s on the other; on one
    qubit every CZ factor is diagonal, so when each run of single-qubit gates
    between two held projectors is monomial (diagonal or anti-diagonal) the
    second value is the first (or its flip), and after the last held projector
    of a qubit the same holds with the measured bit x_q.  The values are a
    solution of these ties: each class of tied bits takes one seeded draw
    (SplitMix64), or the value the output bit forces."""
    import numpy as np

    from rqc_inputs import SplitMix64

    def mono(U):
        m = np.abs(U)
        t = 1e-12 * m.max()
        if m[0, 1] <= t and m[1, 0] <= t:
            return 0
        if m[0, 0] <= t and m[1, 1] <= t:
            return 1
        return None

    n = circ.R * circ.C
    index = {o: j for j, o in enumerate(held)}
    run = [np.eye(2, dtype=complex) for _ in range(n)]
    link = [None] * n            # (previous held bit on the qubit, parity) or None
    prev = [-1] * n
    par = [0] * n
    ties = []                    # (j, i, c): v_j = v_i ^ c; i = -1: v_j = c

    def close(q):
        if par[q] is not None:
            m = mono(run[q])
            par[q] = None if m is None else par[q] ^ m
        run[q] = np.eye(2, dtype=complex)

    k = 0
    for g in circ.gates:
        if g.kind == "1q":
            q = g.qubits[0]
            run[q] = np.asarray(g.U).reshape(2, 2) @ run[q]
            continue
        a, b = sorted(g.qubits)
        close(a)
        close(b)
        if k in index:
            j = index[k]
            if par[a] is not None:   # tied to the previous held bit, or to |0>
                ties.append((j, prev[a], par[a]))
            prev[a], par[a] = j, 0
        k += 1
    for q in range(n):
        close(q)
        if prev[q] >= 0 and par[q] is not None:
            ties.append((prev[q], -1, ((x >> q) & 1) ^ par[q]))
    # union-find with parities; node len(held) is the constant 0
    N = len(held)
    up, pp = list(range(N + 1)), [0] * (N + 1)

    def find(u):
        p = 0
        while up[u] != u:
            p ^= pp[u]
            u = up[u]
        return u, p

    for j, i, c in ties:
        ra, pa = find(j)
        rb, pb = find(N if i < 0 else i)
        if ra != rb:
            up[ra], pp[ra] = rb, pa ^ pb ^ c
        elif pa ^ pb != c:
            raise ValueError("the held bits' ties contradict one another")
    rng = SplitMix64(seed)
    root_val = {find(N)[0]: 0}
    vals = []
    for j in range(N):
        r, p = find(j)
        if r not in root_val:
            root_val[r] = rng.next() & 1
        vals.append(root_val[r] ^ p)
    return vals


def seven_by_seven_d40_subslices():
    """4 sub-slices of the 7x7 (1+40+1) amplitude: the second and the fourth
    CZ gate of every horizontal edge have their Schmidt bit held fixed (84
    bits; every running tensor of the column sweep then has at most 2^26
    entries).  The oracle applies each held CZ as its single Schmidt term
    P_s (x) Z^s.  Values that break a tie between held projectors (or between
    the last one on a qubit and the output bit) give an exactly vanishing
    sub-slice, so candidate k takes the values of _consistent_values with seed
    5 ^ 0x5AB + k.  Some candidates still vanish (a cancellation over several
    qubits: on 4x4 (1+40+1) four held CZs around a 2x2 block of qubits do it);
    their value is roundoff, 1e-16 below the 1e-20 of a sub-slice that does
    not vanish.  The first four candidates whose magnitude is above 1e-30 are
    kept, with their candidate numbers."""
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
    x = int(bits[0])
    subs = []
    t = time.time()
    for cand in range(32):
        vals = _consistent_values(circ, fixed, x, (5 ^ 0x5AB) + cand)
        sid = sum(v << j for j, v in enumerate(vals))
        p = op.build(circ.R, circ.C, circ.gates, sliced=fixed, slice_id=sid)
        amp = op.amplitude(p, x)
        print(f"candidate {cand}: {amp} ({time.time() - t:.0f} s)", flush=True)
        if abs(amp) > 1e-30:
            subs.append({"candidate": cand, "fixed_s": vals, "amplitude": [amp.real, amp.imag]})
            if len(subs) == 4:
                break
    return {"workload": "7x7_d40", "bitstring": x, "fixed_cz": fixed,
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
