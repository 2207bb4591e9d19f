"""Seeded synthetic inputs for the PEPS amplitude path: random quantum circuits
on an R x C lattice and the output bitstrings whose amplitudes are wanted.

This module is the single source of inputs shared by the CUDA path, the CPU
oracle, the tests and the benchmark.  It holds none of the simulation
arithmetic: it only decides *which* gates are applied, in which order, and
which bitstrings are asked for.  Gate matrices are emitted as explicit 2x2
complex128 arrays so that neither consumer has to agree on names.

Circuit rules (random quantum circuits of the paper's supplementary section
"Introduction to Random Quantum Circuits"; the CZ layer order and the
single-qubit-gate rule are the ones this project fixes, because the paper only
sketches them):

* initial state |0...0>;
* cycle 0: H on every qubit;
* cycles t = 1..D: the CZ layer (t-1) mod 8 from the order
  H00, V00, H10, V10, H01, V01, H11, V11.  Layer Hab holds the horizontal edges
  (r,c)-(r,c+1) with c%2 == a and r%2 == b; layer Vab holds the vertical edges
  (r,c)-(r+1,c) with r%2 == a and c%2 == b;
* in the same cycle t, every qubit that was in a CZ in cycle t-1 and is not in
  one in cycle t gets a single-qubit gate: T if it has had no T yet, otherwise
  sqrt(X) or sqrt(Y), different from its previous single-qubit gate.  After T
  the choice is a fair draw (low bit of one SplitMix64 output: 0 -> sqrt(X),
  1 -> sqrt(Y)); after sqrt(X) it is sqrt(Y) and vice versa, with no draw;
* cycle D+1: H on every qubit (and nothing else).

Qubit numbering: q = r*C + c.  Bit q of a uint64 bitstring is the output bit of
qubit q (so at most 64 qubits).

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written here from its published definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1

# ---------------------------------------------------------------------------
# SplitMix64
# ---------------------------------------------------------------------------


class SplitMix64:
    """SplitMix64 generator: a Weyl sequence (golden-ratio increment) passed
    through a 64-bit variant of the MurmurHash3 finaliser."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + self.GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


# ---------------------------------------------------------------------------
# Gate matrices (fixed here; the paper does not print them)
# ---------------------------------------------------------------------------

_S2 = 1.0 / math.sqrt(2.0)
GATES = {
    "H": np.array([[_S2, _S2], [_S2, -_S2]], dtype=np.complex128),
    "T": np.array([[1.0, 0.0], [0.0, complex(_S2, _S2)]], dtype=np.complex128),
    "SX": 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128),
    "SY": 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128),
}

CZ_LAYER_ORDER = ("H00", "V00", "H10", "V10", "H01", "V01", "H11", "V11")


@dataclass(frozen=True)
class Gate:
    """One gate of the circuit.  kind is "1q" (qubits=(q,), U = 2x2 matrix,
    row index = output basis state), "cz" (qubits=(q0, q1) with q0 < q1,
    nearest neighbours on the lattice, U = None) or "2q" (qubits=(q0, q1)
    nearest neighbours in either order, U = 4x4 matrix with row index
    2*tau0 + tau1 and column index 2*sigma0 + sigma1, qubit q0 first)."""

    kind: str
    qubits: tuple
    name: str
    U: np.ndarray | None = None
    cycle: int = 0


@dataclass
class Circuit:
    R: int
    C: int
    depth: int
    seed: int
    gates: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return self.R * self.C

    def cz_count(self, q0: int, q1: int) -> int:
        a, b = min(q0, q1), max(q0, q1)
        return sum(1 for g in self.gates if g.kind == "cz" and g.qubits == (a, b))


def cz_layer_edges(R: int, C: int, layer: int) -> list:
    """Edges (q0, q1), q0 < q1, of CZ layer `layer` (0..7) in the order
    H00,V00,H10,V10,H01,V01,H11,V11, listed in ascending q0."""
    name = CZ_LAYER_ORDER[layer % 8]
    a, b = int(name[1]), int(name[2])
    edges = []
    if name[0] == "H":
        for r in range(R):
            for c in range(C - 1):
                if c % 2 == a and r % 2 == b:
                    edges.append((r * C + c, r * C + c + 1))
    else:
        for r in range(R - 1):
            for c in range(C):
                if r % 2 == a and c % 2 == b:
                    edges.append((r * C + c, (r + 1) * C + c))
    edges.sort()
    return edges


def make_circuit(R: int, C: int, depth: int, seed: int) -> Circuit:
    """Random circuit of depth (1+depth+1) on an R x C lattice (rules above)."""
    if R < 1 or C < 1 or R * C > 64:
        raise ValueError("lattice must have 1..64 qubits")
    n = R * C
    rng = SplitMix64(seed)
    circ = Circuit(R, C, depth, seed)
    for q in range(n):
        circ.gates.append(Gate("1q", (q,), "H", GATES["H"], 0))
    had_t = [False] * n
    prev = [None] * n  # previous gate from {T, SX, SY}
    in_cz_prev = [False] * n
    for t in range(1, depth + 1):
        edges = cz_layer_edges(R, C, t - 1)
        in_cz = [False] * n
        for q0, q1 in edges:
            in_cz[q0] = in_cz[q1] = True
            circ.gates.append(Gate("cz", (q0, q1), "CZ", None, t))
        for q in range(n):
            if in_cz_prev[q] and not in_cz[q]:
                if not had_t[q]:
                    name = "T"
                    had_t[q] = True
                elif prev[q] == "SX":
                    name = "SY"
                elif prev[q] == "SY":
                    name = "SX"
                else:  # previous was T: fair draw
                    name = "SX" if (rng.next() & 1) == 0 else "SY"
                prev[q] = name
                circ.gates.append(Gate("1q", (q,), name, GATES[name], t))
        in_cz_prev = in_cz
    for q in range(n):
        circ.gates.append(Gate("1q", (q,), "H", GATES["H"], depth + 1))
    return circ


# ---------------------------------------------------------------------------
# Bitstrings
# ---------------------------------------------------------------------------

BITSTRING_SALT = 0xB175


def uniform_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    """`count` uniform n-bit strings (uint64), one SplitMix64 draw each from
    the stream seeded with seed ^ 0xB175."""
    rng = SplitMix64(seed ^ BITSTRING_SALT)
    mask = (1 << n_qubits) - 1 if n_qubits < 64 else MASK64
    return np.array([rng.next() & mask for _ in range(count)], dtype=np.uint64)


def prefix_group_bitstrings(R: int, C: int, prefix_cols: int, groups: int,
                            per_group: int, seed: int) -> np.ndarray:
    """Bitstrings in `groups` groups of `per_group`; inside a group all share
    the bits of the qubits in columns < prefix_cols.  Group g draws its prefix
    bits (one draw, low bits assigned to the prefix qubits in ascending q);
    then each member draws its suffix bits likewise.  Ordered group-major."""
    rng = SplitMix64(seed ^ BITSTRING_SALT)
    pre_q = [r * C + c for r in range(R) for c in range(C) if c < prefix_cols]
    suf_q = [r * C + c for r in range(R) for c in range(C) if c >= prefix_cols]
    pre_q.sort()
    suf_q.sort()
    out = []
    for _ in range(groups):
        d = rng.next()
        base = 0
        for i, q in enumerate(pre_q):
            base |= ((d >> i) & 1) << q
        for _ in range(per_group):
            e = rng.next()
            x = base
            for i, q in enumerate(suf_q):
                x |= ((e >> i) & 1) << q
            out.append(x)
    return np.array(out, dtype=np.uint64)


def all_bitstrings(n_qubits: int) -> np.ndarray:
    return np.arange(1 << n_qubits, dtype=np.uint64)


# ---------------------------------------------------------------------------
# Named workloads (the five lattices the project measures)
# ---------------------------------------------------------------------------

WORKLOADS = {
    "4x4_d8": dict(R=4, C=4, depth=8, seed=1, bitstrings=64),
    "5x5_d16": dict(R=5, C=5, depth=16, seed=2, bitstrings=1024),
    "6x6_d24": dict(R=6, C=6, depth=24, seed=3, bitstrings=4096),
    "6x6_d32": dict(R=6, C=6, depth=32, seed=4, groups=8, per_group=64, prefix_cols=3),
    "7x7_d40": dict(R=7, C=7, depth=40, seed=5, bitstrings=1),
    # the paper's workstation experiment: 10000 amplitudes of an 8x8 (1+25+1)
    # circuit against the Porter-Thomas distribution
    "8x8_d25": dict(R=8, C=8, depth=25, seed=6, bitstrings=10000),
}


def workload(name: str):
    """(circuit, bitstrings) of a named workload."""
    w = WORKLOADS[name]
    circ = make_circuit(w["R"], w["C"], w["depth"], w["seed"])
    if "groups" in w:
        bits = prefix_group_bitstrings(w["R"], w["C"], w["prefix_cols"], w["groups"],
                                       w["per_group"], w["seed"])
    else:
        bits = uniform_bitstrings(w["R"] * w["C"], w["bitstrings"], w["seed"])
    return circ, bits


def two_qubit_test_gates(seed: int):
    """Four 4x4 gate matrices (rows 2*t0 + t1, columns 2*s0 + s1): iSWAP
    (operator-Schmidt rank 4), CNOT (rank 2), the non-unitary II + XX/2 + YY/4
    (rank 3) and a seeded random unitary (rank 4)."""
    rng = np.random.default_rng(seed)
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    iswap = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
    rank3 = np.eye(4, dtype=np.complex128) + 0.5 * np.kron(X, X) + 0.25 * np.kron(Y, Y)
    z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    q, r = np.linalg.qr(z)
    return [iswap, cnot, rank3, q * (np.diag(r) / np.abs(np.diag(r)))]


def make_circuit_general(R: int, C: int, layers: int, seed: int) -> Circuit:
    """H on all qubits, then `layers` rounds of two-qubit gates from
    two_qubit_test_gates on every third edge (rotating), each in a random
    qubit order, each round followed by a random single-qubit unitary on every
    qubit; H on all at the end.  Seeded (numpy default_rng(seed))."""
    rng = np.random.default_rng(seed)
    gs = two_qubit_test_gates(seed)
    n = R * C
    circ = Circuit(R, C, layers, seed)
    circ.gates = [Gate("1q", (q,), "H", GATES["H"]) for q in range(n)]
    edges = [(r * C + c, r * C + c + 1) for r in range(R) for c in range(C - 1)] + \
            [(r * C + c, (r + 1) * C + c) for r in range(R - 1) for c in range(C)]
    for layer in range(layers):
        for k, (a, b) in enumerate(edges):
            if (k + layer) % 3 == 0:
                G = gs[(k + layer) % len(gs)]
                qs = (a, b) if rng.random() < 0.5 else (b, a)
                if qs[0] > qs[1]:   # the matrix is given with qubit qs[0] first
                    G = G.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)
                circ.gates.append(Gate("2q", qs, "G", G))
        for q in range(n):
            z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
            u, rr = np.linalg.qr(z)
            circ.gates.append(Gate("1q", (q,), "U", u * (np.diag(rr) / np.abs(np.diag(rr)))))
    circ.gates += [Gate("1q", (q,), "H", GATES["H"]) for q in range(n)]
    return circ
