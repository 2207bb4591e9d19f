"""Seeded input generators: RNG, gate matrices and the circuit rules.  These
are inputs to both the CUDA path and the oracle, so they are pinned on their
own (CPU)."""
import numpy as np
import pytest

from rqc_inputs import (CZ_LAYER_ORDER, GATES, SplitMix64, cz_layer_edges, make_circuit,
                        prefix_group_bitstrings, uniform_bitstrings, workload)


def test_splitmix64_published_outputs():
    # Outputs of the reference SplitMix64 implementation (Steele, Lea & Flood
    # 2014; the splitmix64.c distributed with xoshiro): seed 0 and seed 1234567.
    r = SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                            0x06C45D188009454F]
    r = SplitMix64(1234567)
    assert [r.next() for _ in range(5)] == [6457827717110365317, 3203168211198807973,
                                            9817491932198370423, 4593380528125082431,
                                            16408922859458223821]


def test_gate_matrices():
    I = np.eye(2)
    X = np.array([[0, 1], [1, 0]])
    Y = np.array([[0, -1j], [1j, 0]])
    S = np.diag([1, 1j])
    for name, U in GATES.items():
        assert np.allclose(U @ U.conj().T, I, atol=1e-15), name
    assert np.allclose(GATES["H"] @ GATES["H"], I)
    assert np.allclose(GATES["SX"] @ GATES["SX"], X)
    assert np.allclose(GATES["SY"] @ GATES["SY"], Y)
    assert np.allclose(GATES["T"] @ GATES["T"], S)


@pytest.mark.parametrize("R,C", [(2, 2), (3, 4), (5, 5), (6, 6), (7, 7), (1, 5)])
def test_cz_layers_partition_edges(R, C):
    all_edges = set()
    for r in range(R):
        for c in range(C - 1):
            all_edges.add((r * C + c, r * C + c + 1))
    for r in range(R - 1):
        for c in range(C):
            all_edges.add((r * C + c, (r + 1) * C + c))
    seen = []
    for layer in range(8):
        edges = cz_layer_edges(R, C, layer)
        qs = [q for e in edges for q in e]
        assert len(qs) == len(set(qs)), "a layer touches a qubit twice"
        name = CZ_LAYER_ORDER[layer]
        a, b = int(name[1]), int(name[2])
        for (q0, q1) in edges:
            r0, c0 = divmod(q0, C)
            if name[0] == "H":
                assert q1 == q0 + 1 and c0 % 2 == a and r0 % 2 == b
            else:
                assert q1 == q0 + C and r0 % 2 == a and c0 % 2 == b
        seen += edges
    assert len(seen) == len(set(seen)) and set(seen) == all_edges


@pytest.mark.parametrize("R,C,d,seed", [(4, 4, 8, 1), (5, 5, 16, 2), (6, 6, 24, 3),
                                        (6, 6, 32, 4), (7, 7, 40, 5), (3, 5, 13, 9)])
def test_circuit_rules(R, C, d, seed):
    circ = make_circuit(R, C, d, seed)
    n = R * C
    by_cycle = {}
    for g in circ.gates:
        by_cycle.setdefault(g.cycle, []).append(g)
    assert [g.name for g in by_cycle[0]] == ["H"] * n
    assert [g.name for g in by_cycle[d + 1]] == ["H"] * n
    in_cz = {0: set()}
    for t in range(1, d + 1):
        gs = by_cycle.get(t, [])
        czs = [g.qubits for g in gs if g.kind == "cz"]
        assert czs == cz_layer_edges(R, C, t - 1)
        in_cz[t] = {q for e in czs for q in e}
        ones = [g for g in gs if g.kind == "1q"]
        expect = sorted(q for q in range(n) if q in in_cz[t - 1] and q not in in_cz[t])
        assert [g.qubits[0] for g in ones] == expect
        assert not (set(g.qubits[0] for g in ones) & in_cz[t])
    # per-qubit sequence of non-H single-qubit gates
    for q in range(n):
        seq = [g.name for g in circ.gates if g.kind == "1q" and g.qubits == (q,)
               and 1 <= g.cycle <= d]
        if seq:
            assert seq[0] == "T"
            assert seq.count("T") == 1
            for a, b in zip(seq, seq[1:]):
                assert b in ("SX", "SY") and a != b
    # every edge gets one CZ per 8 cycles (the "chi" equation's premise)
    if d % 8 == 0:
        for (q0, q1) in set(g.qubits for g in circ.gates if g.kind == "cz"):
            assert circ.cz_count(q0, q1) == d // 8


def test_draws_are_fair_and_seeded():
    c1 = make_circuit(6, 6, 32, 4)
    c2 = make_circuit(6, 6, 32, 4)
    assert [g.name for g in c1.gates] == [g.name for g in c2.gates]
    c3 = make_circuit(6, 6, 32, 5)
    assert [g.name for g in c1.gates] != [g.name for g in c3.gates]
    names = [g.name for g in make_circuit(7, 7, 400, 11).gates]
    assert abs(names.count("SX") - names.count("SY")) < 0.1 * (names.count("SX") + names.count("SY"))


def test_bitstrings():
    b = uniform_bitstrings(25, 1000, 2)
    assert b.dtype == np.uint64 and int(b.max()) < (1 << 25)
    assert len(set(b.tolist())) > 990
    g = prefix_group_bitstrings(6, 6, 3, 8, 64, 4)
    assert len(g) == 512
    mask = sum(1 << (r * 6 + c) for r in range(6) for c in range(3))
    for k in range(8):
        grp = g[64 * k:64 * (k + 1)]
        assert len({int(x) & mask for x in grp}) == 1
        assert len({int(x) & ~mask for x in grp}) > 60
    assert len({int(x) & mask for x in g}) == 8
    circ, bits = workload("6x6_d32")
    assert (circ.R, circ.C, circ.depth) == (6, 6, 32) and np.array_equal(bits, g)
