"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix
(closed forms, brute force, invariants), plus planted-mistake checks that show
the pins catch a transposed gate, a wrong sign and a wrong leg order."""
import itertools
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import peps as op
from oracle import statevector as sv
from rqc_inputs import GATES, Gate, make_circuit, uniform_bitstrings

RNG = np.random.default_rng(12345)


def rand_unitary(rng):
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def g1(q, U):
    return Gate("1q", (q,), "U", np.asarray(U, dtype=np.complex128))


def gcz(a, b):
    return Gate("cz", (min(a, b), max(a, b)), "CZ")


# ---------------------------------------------------------------------------
# Closed forms for the state vector (P5) -- helpers return the max error so
# that the planted-mistake tests can reuse them.
# ---------------------------------------------------------------------------

def err_product_state(n=5, seed=0):
    """No CZ: a_x = prod_q <x_q| U_q |0> (each U_q a product of random
    unitaries applied in order)."""
    rng = np.random.default_rng(seed)
    gates, tot = [], [np.eye(2, dtype=complex) for _ in range(n)]
    for _ in range(3):
        for q in range(n):
            U = rand_unitary(rng)
            gates.append(g1(q, U))
            tot[q] = U @ tot[q]
    a = sv.amplitudes(n, gates, np.arange(1 << n, dtype=np.uint64))
    ref = np.array([np.prod([tot[q][(x >> q) & 1, 0] for q in range(n)]) for x in range(1 << n)])
    return np.abs(a - ref).max()


def err_hcz_h(R=3, C=3, layers=(0, 1, 2, 3)):
    """H on all, some CZ layers, H on all:
    a_x = 2^-n sum_y (-1)^(x.y + sum_{(i,j) in E} y_i y_j)."""
    from rqc_inputs import cz_layer_edges
    n = R * C
    edges = [e for L in layers for e in cz_layer_edges(R, C, L)]
    gates = [g1(q, GATES["H"]) for q in range(n)] + [gcz(*e) for e in edges] + \
            [g1(q, GATES["H"]) for q in range(n)]
    a = sv.amplitudes(n, gates, np.arange(1 << n, dtype=np.uint64))
    ys = np.arange(1 << n)
    ybits = (ys[:, None] >> np.arange(n)[None, :]) & 1
    phase_e = np.zeros(1 << n, dtype=np.int64)
    for (i, j) in edges:
        phase_e += ybits[:, i] * ybits[:, j]
    ref = np.zeros(1 << n)
    for x in range(1 << n):
        xy = ((ys & x).astype(np.int64))
        par = np.array([bin(v).count("1") for v in xy]) + phase_e
        ref[x] = np.sum((-1.0) ** par) / 2 ** n
    return np.abs(a - ref).max()


def test_statevector_product_state_closed_form():
    assert err_product_state() < 1e-14


def test_statevector_hh_is_identity():
    n = 6
    gates = [g1(q, GATES["H"]) for q in range(n)] * 2
    a = sv.amplitudes(n, gates, np.arange(1 << n, dtype=np.uint64))
    ref = np.zeros(1 << n)
    ref[0] = 1
    assert np.abs(a - ref).max() < 1e-15


def test_statevector_h_cz_h_walsh_formula():
    assert err_hcz_h() < 1e-14
    assert err_hcz_h(2, 4, layers=range(8)) < 1e-14


def test_statevector_bit_order():
    # X = SX.SX on qubit q sends |0..0> to the basis state with only bit q set
    n = 5
    for q in range(n):
        gates = [g1(q, GATES["SX"]), g1(q, GATES["SX"])]
        psi = sv.run(n, gates)
        assert abs(psi[1 << q] - 1) < 1e-15


def test_statevector_norm():
    for (R, C, d, s) in [(3, 3, 8, 1), (4, 4, 16, 2), (2, 5, 13, 3)]:
        c = make_circuit(R, C, d, s)
        psi = sv.run(R * C, c.gates)
        assert abs(np.vdot(psi, psi) - 1) < 1e-12


# ---------------------------------------------------------------------------
# O3 (PEPS) against O2 (state vector): brute force (P1), norm (P2), bond
# dimensions (P3), scale covariance (P8), orientation (P9), slicing (P6),
# the SVD split (A1).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("R,C,d,seed", [(2, 2, 8, 1), (2, 3, 16, 2), (3, 3, 8, 3),
                                        (3, 3, 16, 4), (3, 4, 16, 5), (1, 4, 9, 6),
                                        (4, 1, 9, 7)])
def test_peps_equals_statevector_all_bitstrings(R, C, d, seed):
    c = make_circuit(R, C, d, seed)
    n = R * C
    allx = np.arange(1 << n, dtype=np.uint64)
    ref = sv.amplitudes(n, c.gates, allx)
    p = op.build(R, C, c.gates)
    a = op.amplitudes(p, allx)
    assert np.abs(a - ref).max() < 1e-13
    assert abs(np.sum(np.abs(a) ** 2) - 1) < 1e-12          # P2


def test_peps_equals_statevector_4x4_sampled():
    c = make_circuit(4, 4, 8, 1)
    x = uniform_bitstrings(16, 512, 1)
    ref = sv.amplitudes(16, c.gates, x)
    a = op.amplitudes(op.build(4, 4, c.gates), x)
    assert np.abs(a - ref).max() < 1e-14


def test_peps_equals_statevector_4x5_d16_sampled():
    c = make_circuit(4, 5, 16, 8)
    x = uniform_bitstrings(20, 64, 8)
    ref = sv.amplitudes(20, c.gates, x)
    a = op.amplitudes(op.build(4, 5, c.gates), x)
    assert np.abs(a - ref).max() < 1e-14


@pytest.mark.parametrize("R,C,d", [(4, 4, 8), (5, 5, 16), (6, 6, 24), (6, 6, 32), (3, 4, 20)])
def test_bond_dims_are_two_to_the_cz_count(R, C, d):
    c = make_circuit(R, C, d, 1)
    p = op.build(R, C, c.gates)
    for r in range(R):
        for col in range(C):
            q = r * C + col
            if col + 1 < C:
                assert p.bond_dim(q, q + 1) == 2 ** c.cz_count(q, q + 1)
            if r + 1 < R:
                assert p.bond_dim(q, q + C) == 2 ** c.cz_count(q, q + C)
    if d % 8 == 0:  # equality in the "chi" bound when 8 divides d
        assert max(max(t.shape[1:]) for t in p.A) == 2 ** (d // 8)


def test_scale_covariance():
    c = make_circuit(3, 3, 16, 4)
    x = uniform_bitstrings(9, 32, 4)
    p = op.build(3, 3, c.gates)
    gates2 = list(c.gates)
    k = [i for i, g in enumerate(gates2) if g.kind == "1q" and g.cycle == 5][0]
    g = gates2[k]
    gates2[k] = Gate("1q", g.qubits, g.name, 8.0 * g.U, g.cycle)
    a1 = op.amplitudes(p, x)
    a2 = op.amplitudes(op.build(3, 3, gates2), x)
    assert np.abs(a2 - 8 * a1).max() < 1e-14


def test_row_sweep_equals_column_sweep():
    c = make_circuit(4, 3, 16, 9)
    x = uniform_bitstrings(12, 64, 9)
    p = op.build(4, 3, c.gates)
    assert np.abs(op.amplitudes(p, x, "row") - op.amplitudes(p, x, "column")).max() < 1e-14


def transpose_circuit(c):
    """The same circuit on the transposed lattice: qubit (r, c) -> (c, r)."""
    R, C = c.R, c.C
    m = {r * C + col: col * R + r for r in range(R) for col in range(C)}
    gates = []
    for g in c.gates:
        if g.kind == "1q":
            gates.append(Gate("1q", (m[g.qubits[0]],), g.name, g.U, g.cycle))
        else:
            a, b = m[g.qubits[0]], m[g.qubits[1]]
            gates.append(Gate("cz", (min(a, b), max(a, b)), "CZ", None, g.cycle))
    return SimpleNamespace(R=C, C=R, gates=gates), m


def test_transposed_lattice_same_amplitudes():
    c = make_circuit(3, 4, 16, 10)
    ct, m = transpose_circuit(c)
    x = uniform_bitstrings(12, 64, 10)
    xt = np.array([sum(((int(v) >> q) & 1) << m[q] for q in range(12)) for v in x],
                  dtype=np.uint64)
    a = op.amplitudes(op.build(3, 4, c.gates), x)
    at = op.amplitudes(op.build(4, 3, ct.gates), xt)
    assert np.abs(a - at).max() < 1e-14


def test_svd_split_gives_same_amplitudes():
    c = make_circuit(3, 3, 16, 11)
    x = uniform_bitstrings(9, 64, 11)
    a = op.amplitudes(op.build(3, 3, c.gates, split="projector"), x)
    b = op.amplitudes(op.build(3, 3, c.gates, split="svd"), x)
    assert np.abs(a - b).max() < 1e-13
    U, V = op.svd_split(op.cz_matrix())
    assert U.shape[2] == 2  # chi_o = 2 for a controlled gate


@pytest.mark.parametrize("sliced", [[0], [3, 7], [1, 5, 9, 20]])
def test_slice_sum_identity(sliced):
    c = make_circuit(3, 3, 16, 12)
    x = uniform_bitstrings(9, 16, 12)
    full = op.amplitudes(op.build(3, 3, c.gates), x)
    tot = np.zeros_like(full)
    for sid in range(1 << len(sliced)):
        tot += op.amplitudes(op.build(3, 3, c.gates, sliced=sliced, slice_id=sid), x)
    assert np.abs(tot - full).max() < 1e-14


def test_prefix_reuse_equals_plain():
    from rqc_inputs import prefix_group_bitstrings
    c = make_circuit(3, 4, 16, 13)
    x = prefix_group_bitstrings(3, 4, 2, 3, 5, 13)
    p = op.build(3, 4, c.gates)
    assert np.abs(op.amplitudes_with_prefix(p, x, 2) - op.amplitudes(p, x)).max() < 1e-15


# ---------------------------------------------------------------------------
# Square partition (supplementary Fig. S2(b)): brute force against the state
# vector, equality with the column sweep, and the paper's complexity.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("R,C,d,seed", [(2, 2, 8, 1), (2, 4, 16, 2), (4, 2, 16, 3),
                                        (4, 4, 8, 4)])
def test_quadrant_equals_statevector(R, C, d, seed):
    c = make_circuit(R, C, d, seed)
    n = R * C
    x = np.arange(1 << n, dtype=np.uint64) if n <= 12 else uniform_bitstrings(n, 256, seed)
    ref = sv.amplitudes(n, c.gates, x)
    a = op.amplitudes_quadrant(op.build(R, C, c.gates), x)
    assert np.abs(a - ref).max() < 1e-13


def test_quadrant_equals_column_sweep_6x6():
    c = make_circuit(6, 6, 16, 3)
    x = uniform_bitstrings(36, 4, 3)
    p = op.build(6, 6, c.gates)
    a, b = op.amplitudes_quadrant(p, x), op.amplitudes(p, x)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_quadrant_needs_even_sides_or_an_odd_square():
    with pytest.raises(ValueError):
        op.quadrant_sites(5, 6)
    with pytest.raises(ValueError):
        op.quadrant_sites(5, 7)
    parts = op.quadrant_sites(7, 7)
    assert sorted(q for v in parts.values() for q in v) == list(range(49))
    assert [len(parts[k]) for k in ("ul", "ur", "bl", "br")] == [12, 16, 12, 9]


@pytest.mark.parametrize("L,d,seed", [(3, 8, 1), (3, 16, 2), (3, 24, 3)])
def test_odd_partition_equals_statevector(L, d, seed):
    c = make_circuit(L, L, d, seed)
    n = L * L
    x = np.arange(1 << n, dtype=np.uint64) if n <= 9 else uniform_bitstrings(n, 16, seed)
    ref = sv.amplitudes(n, c.gates, x)
    assert np.abs(op.amplitudes_quadrant(op.build(L, L, c.gates), x) - ref).max() < 1e-13


@pytest.mark.parametrize("L,d,seed", [(5, 16, 3), (7, 16, 4)])
def test_odd_partition_equals_column_sweep(L, d, seed):
    c = make_circuit(L, L, d, seed)
    x = uniform_bitstrings(L * L, 3, seed)
    p = op.build(L, L, c.gates)
    a, b = op.amplitudes_quadrant(p, x), op.amplitudes(p, x)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("L,d", [(7, 40), (9, 40), (7, 24)])
def test_odd_partition_cost_matches_the_paper(L, d):
    # Eq. (timesquareodd): (2^k + 1) 2^(k (3L - 1) / 2) for the merges;
    # Eq. (spacesquareodd): 2^(k (L + 1)) + 2^(k L): the largest part and one more
    from paper_1905_08394_gb300 import complexity as cx
    k = -(-d // 8)
    chi = 2 ** k
    dims = {}
    for r in range(L):
        for cc in range(L):
            q = r * L + cc
            if cc + 1 < L:
                dims[(q, q + 1)] = chi
            if r + 1 < L:
                dims[(q, q + L)] = chi
    cost = op.quadrant_contraction_cmacs(L, L, dims)
    # the two pair merges give the formula; the last merge adds chi^L
    assert cost["merges"] == cx.time_square_odd(L, d) + chi ** L
    assert cost["largest"] + chi ** L == cx.space_square_odd(L, d)


@pytest.mark.parametrize("L,d", [(6, 32), (8, 40), (6, 24)])
def test_quadrant_cost_matches_the_paper(L, d):
    # Eq. (timesquareeven): 2^(3 k L / 2 + 1) multiply-adds for the merges, k = ceil(d/8);
    # Eq. (spacesquareeven): 2^(k L + 1) entries, two quarter-pair tensors of chi^L
    from paper_1905_08394_gb300 import complexity as cx
    k = -(-d // 8)
    chi = 2 ** k
    dims = {}
    for r in range(L):
        for cc in range(L):
            q = r * L + cc
            if cc + 1 < L:
                dims[(q, q + 1)] = chi
            if r + 1 < L:
                dims[(q, q + L)] = chi
    cost = op.quadrant_contraction_cmacs(L, L, dims)
    # the two pair merges give the formula; the last merge adds chi^L
    assert cost["merges"] == cx.time_square_even(L, d) + chi ** L
    assert 2 * cost["largest"] == cx.space_square_even(L, d)
    # at L = 6 it also undercuts the column sweep's Eq. (time) (at L = 8, k = 5 the
    # partition saves memory, 2^41 vs 2^45 entries, but not time)
    if L == 6:
        assert cost["merges"] + cost["quarters"] < cx.time_generic(L, L, d) / 4


# ---------------------------------------------------------------------------
# General two-qubit gates (main-text "factorize": SVD split, chi_o <= 4)
# ---------------------------------------------------------------------------

PAULI = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]),
         np.diag([1.0, -1.0])]


def g2(a, b, G):
    return Gate("2q", (a, b), "G", np.asarray(G, dtype=np.complex128))


def two_qubit_gates(rng):
    iswap = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]])
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]])
    rank3 = (np.kron(PAULI[0], PAULI[0]) + 0.5 * np.kron(PAULI[1], PAULI[1])
             + 0.25 * np.kron(PAULI[2], PAULI[2]))                 # not unitary; rank 3
    z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    q, r = np.linalg.qr(z)
    return [iswap, cnot, rank3, q * (np.diag(r) / np.abs(np.diag(r)))]


def circuit_with_2q(R, C, seed):
    """H on all, then layers of random two-qubit gates on alternating edges
    (either qubit order), single-qubit gates in between, H on all."""
    rng = np.random.default_rng(seed)
    gs = two_qubit_gates(rng)
    n = R * C
    gates = [g1(q, GATES["H"]) for q in range(n)]
    edges = [(r * C + c, r * C + c + 1) for r in range(R) for c in range(C - 1)] + \
            [(r * C + c, (r + 1) * C + c) for r in range(R - 1) for c in range(C)]
    for layer in range(3):
        for k, (a, b) in enumerate(edges):
            if (k + layer) % 3 == 0:
                G = gs[(k + layer) % len(gs)]
                gates.append(g2(a, b, G) if rng.random() < 0.5 else g2(b, a, G))
        for q in range(n):
            gates.append(g1(q, rand_unitary(rng)))
    return gates


def test_statevector_2q_gate_order_and_cz():
    # CZ through the general path equals the CZ routine; swapping the qubit
    # order of a gate and permuting its matrix gives the same state
    rng = np.random.default_rng(3)
    n = 4
    base = [g1(q, rand_unitary(rng)) for q in range(n)]
    cz = np.diag([1, 1, 1, -1.0])
    a = sv.run(n, base + [gcz(1, 2)])
    b = sv.run(n, base + [g2(1, 2, cz)])
    assert np.abs(a - b).max() < 1e-15
    G = two_qubit_gates(rng)[3]
    Gs = G.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)
    assert np.abs(sv.run(n, base + [g2(0, 1, G)]) - sv.run(n, base + [g2(1, 0, Gs)])).max() < 1e-14


@pytest.mark.parametrize("R,C,seed", [(2, 2, 1), (2, 3, 2), (3, 3, 3)])
def test_peps_2q_gates_equal_statevector(R, C, seed):
    gates = circuit_with_2q(R, C, seed)
    n = R * C
    x = np.arange(1 << n, dtype=np.uint64)
    ref = sv.amplitudes(n, gates, x)
    a = op.amplitudes(op.build(R, C, gates), x)
    assert np.abs(a - ref).max() < 1e-13


# Orientation of a general gate G[(t0 t1), (s0 s1)] (qubit q0 first), pinned by
# closed forms that a shared convention mistake (G read transposed, or the two
# qubits swapped) cannot pass: every expected value below is written out by
# hand, not computed by either oracle.
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
ISWAP = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)


CYCLE = np.zeros((4, 4), dtype=complex)     # |00> -> |01> -> |11> -> |10> -> |00>
for _s, _t in ((0, 1), (1, 3), (3, 2), (2, 0)):
    CYCLE[_t, _s] = 1.0


def _orientation_cases():
    """(gate list on 2x2 (n = 4), {bitstring: amplitude}) with every other
    amplitude of the final state zero."""
    q0, q1 = 1, 3          # vertical neighbours on a 2x2 lattice (q = r*2 + c)
    rng = np.random.default_rng(77)
    U = two_qubit_gates(rng)[3]
    Us = U.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)   # qubits swapped
    bit = lambda t0, t1: (t0 << q0) | (t1 << q1)
    return [
        # CNOT, control q0: |q0=1, q1=0> -> |q0=1, q1=1>
        ([g1(q0, X), g2(q0, q1, CNOT)], {bit(1, 1): 1.0}),
        # the same gate given with q1 first: q1 is the control and is 0
        ([g1(q0, X), g2(q1, q0, CNOT)], {bit(1, 0): 1.0}),
        # iSWAP |q0=0, q1=1> = i |q0=1, q1=0>
        ([g1(q1, X), g2(q0, q1, ISWAP)], {bit(1, 0): 1j}),
        # a cyclic permutation (not symmetric): |00> -> |q0=0, q1=1>, and
        # from |q0=1, q1=0> back to |00>
        ([g2(q0, q1, CYCLE)], {bit(0, 1): 1.0}),
        ([g1(q0, X), g2(q0, q1, CYCLE)], {bit(0, 0): 1.0}),
        # the same permutation given with q1 first: |00> -> |q0=1, q1=0>
        ([g2(q1, q0, CYCLE)], {bit(1, 0): 1.0}),
        # a random U on |00>: the amplitudes are U's first column, entry
        # (2 t0 + t1) at |q0=t0, q1=t1>
        ([g2(q0, q1, U)], {bit(t0, t1): U[2 * t0 + t1, 0] for t0 in (0, 1) for t1 in (0, 1)}),
        # U then U^dagger returns the start state, also with the qubit order of
        # the second gate reversed (its matrix permuted to match)
        ([g1(0, X), g2(q0, q1, U), g2(q0, q1, U.conj().T)], {1: 1.0}),
        ([g1(0, X), g2(q0, q1, U), g2(q1, q0, Us.conj().T)], {1: 1.0}),
    ]


def _expected(amps):
    ref = np.zeros(16, dtype=complex)
    for x, a in amps.items():
        ref[x] = a
    return ref


def err_2q_orientation_statevector():
    worst = 0.0
    for gates, amps in _orientation_cases():
        psi = sv.run(4, gates)
        worst = max(worst, float(np.abs(psi - _expected(amps)).max()))
    return worst


def err_2q_orientation_peps():
    worst = 0.0
    allx = np.arange(16, dtype=np.uint64)
    for gates, amps in _orientation_cases():
        a = op.amplitudes(op.build(2, 2, gates), allx)
        worst = max(worst, float(np.abs(a - _expected(amps)).max()))
    return worst


def test_2q_orientation_closed_forms():
    assert err_2q_orientation_statevector() < 1e-14
    assert err_2q_orientation_peps() < 1e-13


def test_planted_transposed_2q_gate_is_caught(monkeypatch):
    orig_sv = sv.apply_2q
    monkeypatch.setattr(sv, "apply_2q",
                        lambda psi, n, q0, q1, G: orig_sv(psi, n, q0, q1, np.asarray(G).T))
    assert err_2q_orientation_statevector() > 1e-3
    monkeypatch.undo()
    orig_op = op.PEPS.apply_2q
    monkeypatch.setattr(op.PEPS, "apply_2q",
                        lambda self, q0, q1, G: orig_op(self, q0, q1, np.asarray(G).T))
    assert err_2q_orientation_peps() > 1e-3


def test_planted_swapped_2q_qubits_are_caught(monkeypatch):
    orig_sv = sv.apply_2q
    monkeypatch.setattr(sv, "apply_2q",
                        lambda psi, n, q0, q1, G: orig_sv(psi, n, q1, q0, G))
    assert err_2q_orientation_statevector() > 1e-3


def test_svd_split_ranks():
    rng = np.random.default_rng(4)
    iswap, cnot, rank3, rnd = two_qubit_gates(rng)
    for G, k in ((iswap, 4), (cnot, 2), (rank3, 3), (rnd, 4), (np.diag([1, 1, 1, -1.0]), 2)):
        U, V = op.svd_split(np.asarray(G, dtype=complex).reshape(2, 2, 2, 2))
        assert U.shape[2] == k


# ---------------------------------------------------------------------------
# Marginals: the double-layer contraction against the state vector's sums
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("R,C,d,seed", [(2, 3, 16, 1), (3, 3, 8, 2), (3, 4, 16, 3)])
def test_double_layer_marginals_equal_statevector_sums(R, C, d, seed):
    c = make_circuit(R, C, d, seed)
    n = R * C
    p = op.build(R, C, c.gates)
    x = uniform_bitstrings(n, 6, seed)
    for mask in (0b1, (1 << (n // 2)) - 1, 0b1010101 & ((1 << n) - 1), (1 << n) - 1):
        ref = sv.marginals(n, c.gates, x, mask)
        assert np.abs(op.marginals(p, x, mask) - ref).max() < 1e-13


def test_double_layer_square_partition():
    c = make_circuit(4, 4, 8, 5)
    p = op.build(4, 4, c.gates)
    x = uniform_bitstrings(16, 3, 5)
    ref = sv.marginals(16, c.gates, x, 0x0F0F)
    got = np.array([op.marginal_quadrant(p, int(b), 0x0F0F) for b in x])
    assert np.abs(got - ref).max() < 1e-13


def test_marginals_special_cases():
    c = make_circuit(3, 3, 16, 4)
    p = op.build(3, 3, c.gates)
    x = uniform_bitstrings(9, 4, 4)
    # nothing measured: the norm; everything measured: |amplitude|^2
    assert np.abs(op.marginals(p, x, 0) - 1).max() < 1e-13
    assert np.abs(op.marginals(p, x, (1 << 9) - 1) - np.abs(op.amplitudes(p, x)) ** 2).max() < 1e-15
    # the marginals of all settings of the measured bits sum to 1
    mask = 0b100010011
    xs = [sum(((k >> j) & 1) << q for j, q in enumerate([0, 1, 4, 8])) for k in range(16)]
    assert abs(op.marginals(p, xs, mask).sum() - 1) < 1e-13


# ---------------------------------------------------------------------------
# Planted mistakes: each must be caught by one of the pins above.
# ---------------------------------------------------------------------------

def test_planted_transposed_gate_in_statevector_is_caught(monkeypatch):
    orig = sv.apply_1q
    monkeypatch.setattr(sv, "apply_1q", lambda psi, n, q, U: orig(psi, n, q, U.T))
    assert err_product_state() > 1e-3


def test_planted_wrong_cz_sign_is_caught(monkeypatch):
    def bad_cz(psi, n, q0, q1):
        lo, hi = min(q0, q1), max(q0, q1)
        v = psi.reshape(1 << (n - hi - 1), 2, 1 << (hi - lo - 1), 2, 1 << lo)
        v[:, 0, :, 1, :] *= -1.0          # flips |01> instead of |11>
    monkeypatch.setattr(sv, "apply_cz", bad_cz)
    assert err_hcz_h() > 1e-3


def test_planted_wrong_bundling_in_peps_is_caught(monkeypatch):
    # bundling s as the *slow* index on one site only (l' = (s, l) vs r' = (r, s))
    def bad_split(self, q0, q1, U, V):
        ax0, ax1 = self._shared_axes(q0, q1)
        chi_o = U.shape[2]
        a0 = np.einsum("tos,olrud->tlruds", U, self.A[q0])
        a0 = np.moveaxis(a0, 5, ax0 + 1)
        sh = list(self.A[q0].shape)
        sh[ax0] *= chi_o
        self.A[q0] = a0.reshape(sh)
        a1 = np.einsum("sto,olrud->tlruds", V, self.A[q1])
        a1 = np.moveaxis(a1, 5, ax1)          # s before the old leg
        sh = list(self.A[q1].shape)
        sh[ax1] *= chi_o
        self.A[q1] = a1.reshape(sh)
    monkeypatch.setattr(op.PEPS, "apply_2q_split", bad_split)
    c = make_circuit(3, 3, 16, 4)
    x = uniform_bitstrings(9, 64, 4)
    ref = sv.amplitudes(9, c.gates, x)
    a = op.amplitudes(op.build(3, 3, c.gates), x)
    assert np.abs(a - ref).max() > 1e-3


def test_planted_overlapping_quarters_are_caught(monkeypatch):
    # one site counted in two quarters (and missing from its own)
    orig = op.quadrant_sites

    def bad(R, C):
        q = orig(R, C)
        q["ur"] = q["ur"][:-1] + [q["ul"][0]]
        return q
    monkeypatch.setattr(op, "quadrant_sites", bad)
    c = make_circuit(4, 4, 8, 4)
    x = uniform_bitstrings(16, 32, 4)
    ref = sv.amplitudes(16, c.gates, x)
    try:
        a = op.amplitudes_quadrant(op.build(4, 4, c.gates), x)
    except AssertionError:
        return                      # caught: open legs are left over
    assert np.abs(a - ref).max() > 1e-3


def test_planted_missing_conjugate_in_double_layer_is_caught(monkeypatch):
    def bad(peps, x, mask):
        out = []
        for q in range(peps.R * peps.C):
            A = peps.A[q]
            sig = [(int(x) >> q) & 1] if (mask >> q) & 1 else [0, 1]
            D = sum(np.einsum("lrud,LRUD->lLrRuUdD", A[s], A[s]) for s in sig)
            dl, dr, du, dd = A.shape[1:]
            out.append(D.reshape(dl * dl, dr * dr, du * du, dd * dd))
        return out
    monkeypatch.setattr(op, "double_layer", bad)
    c = make_circuit(3, 3, 16, 2)
    x = uniform_bitstrings(9, 4, 2)
    ref = sv.marginals(9, c.gates, x, 0b111)
    assert np.abs(op.marginals(op.build(3, 3, c.gates), x, 0b111) - ref).max() > 1e-3


def test_planted_transposed_peps_gate_is_caught(monkeypatch):
    orig = op.PEPS.apply_1q
    monkeypatch.setattr(op.PEPS, "apply_1q", lambda self, q, U: orig(self, q, np.asarray(U).T))
    c = make_circuit(3, 3, 8, 2)
    x = uniform_bitstrings(9, 64, 2)
    ref = sv.amplitudes(9, c.gates, x)
    a = op.amplitudes(op.build(3, 3, c.gates), x)
    assert np.abs(a - ref).max() > 1e-3
