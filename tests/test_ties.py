"""CZ Schmidt bits fixed by the output bitstring (peps_output_ties, held by
PEPS_FLAG_HOLD_TIES), on the host: the C library's list agrees with the tie
rule of the slicing module for every bit and bitstring, and the FP64 oracle
confirms the rule itself -- its PEPS with every listed bit held at its tied
value gives the state vector's amplitude, and with one held bit flipped the
amplitude is exactly zero.  No GPU needed."""
import numpy as np
import pytest

from oracle import peps as op
from oracle import statevector as sv
from paper_1905_08394_gb300 import binding as B
from paper_1905_08394_gb300 import slicing
from rqc_inputs import GATES, Circuit, Gate, make_circuit, uniform_bitstrings, workload


def ctx_for(circ):
    h = B.peps_create(circ.R, circ.C)
    C = circ.C
    for g in circ.gates:
        if g.kind == "1q":
            B.peps_apply_1q(h, g.qubits[0] // C, g.qubits[0] % C, g.U)
        elif g.kind == "2q":
            a, b = g.qubits
            B.peps_apply_2q(h, a // C, a % C, b // C, b % C, g.U)
        else:
            a, b = g.qubits
            B.peps_apply_cz(h, a // C, a % C, b // C, b % C)
    return h


def cz_lower_qubits(circ):
    return [min(g.qubits) for g in circ.gates if g.kind == "cz"]


def held_values(ties, lower, x):
    """{cz ordinal: held Schmidt bit} for output bitstring x (kinds 1 and 2;
    linked bits, kind 3, have no value of their own)."""
    out = {}
    for t in ties:
        k, kind, flip = t[:3]
        if kind == 3:
            continue
        out[k] = flip if kind == 1 else ((int(x) >> lower[k]) & 1) ^ flip
    return out


def python_tied_values(circ, x):
    """{cz ordinal: value} of every CZ bit the slicing module's tie rule fixes
    for output x (its class holds the constant node)."""
    ncz = sum(1 for g in circ.gates if g.kind == "cz")
    allcz = list(range(ncz))
    find = slicing._tie_components(circ, allcz, x)
    assert find is not None
    root, _ = find(ncz)
    out = {}
    for j in allcz:
        r, par = find(j)
        if r == root:
            out[j] = par ^ find(ncz)[1]
    return out


def circuit_with_constant_ties():
    """2x3 lattice: qubits 0 and 1 start without a Hadamard, so the first
    projector on them is tied to the initial |0> (qubit 0 gets X first: its
    bit is 1); the others get H first.  Diagonal gates between the CZs."""
    R, C = 2, 3
    n = R * C
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    g = [Gate("1q", (0,), "X", X)] + [Gate("1q", (q,), "H", GATES["H"]) for q in range(2, n)]
    cz = lambda a, b: Gate("cz", (min(a, b), max(a, b)), "CZ")
    g += [cz(0, 1), cz(1, 2), cz(0, 3), Gate("1q", (0,), "T", GATES["T"]), cz(0, 1), cz(3, 4),
          cz(4, 5), Gate("1q", (1,), "H", GATES["H"]), cz(1, 4), cz(2, 5)]
    g += [Gate("1q", (q,), "H", GATES["H"]) for q in range(n)]
    return Circuit(R, C, len(g), 0, g)


CIRCUITS = [("6x6_d32", None), ("4x4_d24", (4, 4, 24, 3)), ("4x4_d16", (4, 4, 16, 9)),
            ("3x4_d40", (3, 4, 40, 2)), ("5x5_d16", None)]


def _circ(name, spec):
    if spec is None:
        return workload(name)[0]
    return make_circuit(*spec)


def python_links(circ, x):
    """{(cz, src): flip} for every pair of bits on one edge that the slicing
    module's rule ties to each other but not to a constant, src the first
    bit of its class on that edge."""
    from paper_1905_08394_gb300.slicing import cz_edges

    edges, _ = cz_edges(circ)
    ncz = len(edges)
    find = slicing._tie_components(circ, list(range(ncz)), x)
    const = find(ncz)[0]
    first = {}
    out = {}
    for j in range(ncz):
        r, p = find(j)
        if r == const:
            continue
        key = (r, edges[j])
        if key in first:
            s, ps = first[key]
            out[(j, s)] = p ^ ps
        else:
            first[key] = (j, p)
    return out


@pytest.mark.parametrize("name,spec", CIRCUITS)
def test_c_ties_equal_the_slicing_rule(name, spec):
    circ = _circ(name, spec)
    h = ctx_for(circ)
    ties = B.peps_output_ties(h, with_src=True)
    lower = cz_lower_qubits(circ)
    assert len(ties) > 0
    links = {(k, src): flip for k, kind, flip, src in ties if kind == 3}
    for x in uniform_bitstrings(circ.R * circ.C, 4, 17):
        assert held_values(ties, lower, x) == python_tied_values(circ, int(x))
        assert links == python_links(circ, int(x))
    B.peps_destroy(h)


def test_constant_ties_from_the_initial_state():
    circ = circuit_with_constant_ties()
    h = ctx_for(circ)
    ties = {k: (kind, flip) for k, kind, flip in B.peps_output_ties(h)}
    # CZ ordinals: 0 (0,1), 1 (1,2), 2 (0,3), 3 (0,1), 4 (3,4), 5 (4,5), 6 (1,4), 7 (2,5)
    # CZ 0: projector on qubit 0, which is X|0> = |1> since the start
    assert ties[0] == (1, 1)
    # CZ 2: the next projector on qubit 0, only diagonal factors between
    assert ties[2] == (1, 1)
    # CZ 3 after T on qubit 0: still diagonal, still tied to the start
    assert ties[3] == (1, 1)
    # CZ 1: projector on qubit 1, untouched but for CZ 0's diagonal factor: |0>
    assert ties[1] == (1, 0)
    # CZ 6: qubit 1 had an H since CZ 1 and a lone H before the measurement
    assert 6 not in ties
    for x in range(1 << 6):
        assert held_values(list((k, *v) for k, v in ties.items()), cz_lower_qubits(circ), x) == \
            python_tied_values(circ, x)
    B.peps_destroy(h)


@pytest.mark.parametrize("spec", [(3, 3, 16, 4), (4, 4, 16, 9), (3, 4, 24, 5)])
def test_held_bits_give_the_amplitude_in_the_oracle(spec):
    circ = make_circuit(*spec)
    R, C, n = circ.R, circ.C, circ.R * circ.C
    h = ctx_for(circ)
    ties = [t for t in B.peps_output_ties(h) if t[1] in (1, 2)]
    B.peps_destroy(h)
    assert ties
    lower = cz_lower_qubits(circ)
    sl = [k for k, _, _ in ties]
    xs = np.arange(1 << n, dtype=np.uint64) if n <= 9 else uniform_bitstrings(n, 24, spec[3])
    ref = sv.amplitudes(n, circ.gates, xs)
    for x, a in zip(xs, ref):
        vals = held_values(ties, lower, x)
        sid = sum(vals[k] << j for j, k in enumerate(sl))
        held = op.amplitudes(op.build(R, C, circ.gates, sliced=sl, slice_id=sid), [x])[0]
        assert abs(held - a) <= 1e-12, (int(x), held, a)
        # a held bit at the other value: that term of the bond sum is exactly zero
        j = int(x) % len(sl)
        other = op.amplitudes(op.build(R, C, circ.gates, sliced=sl, slice_id=sid ^ (1 << j)),
                              [x])[0]
        assert abs(other) <= 1e-14


@pytest.mark.parametrize("spec", [(4, 4, 24, 3), (3, 4, 40, 2), (4, 4, 32, 11)])
def test_linked_bits_in_the_oracle(spec):
    # a linked bit at the other value than its source's (XOR flip) gives
    # exactly zero; with every held and linked bit restricted, the sum over
    # the sources' values is the amplitude
    circ = make_circuit(*spec)
    R, C, n = circ.R, circ.C, circ.R * circ.C
    h = ctx_for(circ)
    ties = B.peps_output_ties(h, with_src=True)
    B.peps_destroy(h)
    links = [(k, flip, src) for k, kind, flip, src in ties if kind == 3]
    assert links, "the circuit has no linked bits"
    lower = cz_lower_qubits(circ)
    held = [t for t in ties if t[1] in (1, 2)]
    srcs = sorted({s for _, _, s in links})
    sl = [k for k, _, _, _ in held] + srcs + [k for k, _, _ in links]
    for x in uniform_bitstrings(n, 3, spec[3]):
        ref = sv.amplitudes(n, circ.gates, [x])[0] if n <= 20 else None
        hv = held_values(held, lower, x)
        base = sum(hv[k] << j for j, k in enumerate(sl[:len(held)]))
        total = 0
        for t in range(1 << len(srcs)):
            sid = base
            sv_ = {s: (t >> i) & 1 for i, s in enumerate(srcs)}
            for i, s in enumerate(srcs):
                sid |= sv_[s] << (len(held) + i)
            for i, (k, flip, s) in enumerate(links):
                sid |= (sv_[s] ^ flip) << (len(held) + len(srcs) + i)
            total += op.amplitudes(op.build(R, C, circ.gates, sliced=sl, slice_id=sid), [x])[0]
            # the first link broken: exactly zero
            bad = sid ^ (1 << (len(held) + len(srcs)))
            assert abs(op.amplitudes(op.build(R, C, circ.gates, sliced=sl, slice_id=bad),
                                     [x])[0]) <= 1e-14
        full = op.amplitudes(op.build(R, C, circ.gates), [x])[0]
        assert abs(total - full) <= 1e-12 * max(1.0, abs(full) * 1e3)
        if ref is not None:
            assert abs(full - ref) <= 1e-12


def test_planted_wrong_flip_is_caught():
    # the same oracle check with one tie's flip inverted must fail
    circ = make_circuit(3, 3, 16, 4)
    h = ctx_for(circ)
    ties = [t for t in B.peps_output_ties(h) if t[1] in (1, 2)]
    B.peps_destroy(h)
    bad = [(k, kind, flip ^ (1 if i == 0 else 0)) for i, (k, kind, flip) in enumerate(ties)]
    lower = cz_lower_qubits(circ)
    sl = [k for k, _, _ in bad]
    xs = np.arange(1 << 9, dtype=np.uint64)
    ref = sv.amplitudes(9, circ.gates, xs)
    worst = 0.0
    for x, a in zip(xs[:64], ref[:64]):
        vals = held_values(bad, lower, x)
        sid = sum(vals[k] << j for j, k in enumerate(sl))
        held = op.amplitudes(op.build(3, 3, circ.gates, sliced=sl, slice_id=sid), [x])[0]
        worst = max(worst, abs(held - a))
    assert worst > 1e-3


def test_hold_ties_plan_shrinks_the_work():
    circ, _ = workload("6x6_d32")
    h = ctx_for(circ)
    for scheme in ("columns", "quadrants"):
        kw = dict(precision="fp16x3", prefix_cols=3, prefix_group=64, max_lanes=16,
                  scheme=scheme)
        o0, k0 = B.make_opts(**kw)
        o1, k1 = B.make_opts(hold_ties=True, **kw)
        f0 = B.peps_plan_info_get(h, 512, o0)["flops_call"]
        f1 = B.peps_plan_info_get(h, 512, o1)["flops_call"]
        # the same figure as holding the tied and linked bits at fixed values
        ties = B.peps_output_ties(h)
        o2, k2 = B.make_opts(fixed_cz=[t[0] for t in ties], fixed_s=[0] * len(ties), **kw)
        assert f1 == B.peps_plan_info_get(h, 512, o2)["flops_call"]
        assert f1 < f0
    o, k = B.make_opts(hold_ties=True, sliced_cz=[0], slice_ids=[0])
    with pytest.raises(B.PepsError) as e:
        B.peps_plan_info_get(h, 1, o)
    assert e.value.code == B.PEPS_EINVAL
    o, k = B.make_opts(hold_ties=True, measured_mask=1)
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 1, o)
    B.peps_destroy(h)
