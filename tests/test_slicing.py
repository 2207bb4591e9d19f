"""Slice-set chooser (host planning): budget respected, the C planner agrees on
the sizes and flops it predicts, choices are seeded."""
import numpy as np
import pytest

from paper_1905_08394_gb300 import binding as B
from paper_1905_08394_gb300 import slicing
from rqc_inputs import make_circuit, workload


def ctx_for(circ):
    h = B.peps_create(circ.R, circ.C)
    C = circ.C
    for g in circ.gates:
        if g.kind == "1q":
            B.peps_apply_1q(h, g.qubits[0] // C, g.qubits[0] % C, g.U)
        else:
            a, b = g.qubits
            B.peps_apply_cz(h, a // C, a % C, b // C, b % C)
    return h


@pytest.mark.parametrize("name,budget", [("7x7_d40", 2 ** 33), ("7x7_d40", 2 ** 30),
                                         ("6x6_d32", 2 ** 20), ("5x5_d16", 2 ** 6)])
def test_budget_and_planner_agree(name, budget):
    circ, _ = workload(name)
    ss = slicing.choose(circ, budget, seed=5)
    assert ss.max_entries <= budget
    h = ctx_for(circ)
    o, keep = B.make_opts(precision="fp16x3", sliced_cz=ss.sliced_cz, slice_ids=[0], fuse_rows=1)
    info = B.peps_plan_info_get(h, 1, o)
    assert info["max_entries"] == ss.max_entries
    assert info["flops_per_chain"] == 8 * sum(ss.step_cmacs)
    B.peps_destroy(h)


def test_sub_slice_as_slice_plus_fixed_bits():
    # a sub-slice of a 2^33 slice with 48 more bits held fixed (beyond the 62
    # bits a slice id carries)
    circ, _ = workload("7x7_d40")
    ss = slicing.choose(circ, 2 ** 33, seed=5)
    sub = slicing.choose(circ, 2 ** 25, seed=5, base=ss.sliced_cz)
    extra = [o for o in sub.sliced_cz if o not in ss.sliced_cz]
    assert len(sub.sliced_cz) > 62
    h = ctx_for(circ)
    o, keep = B.make_opts(precision="fp16x3", sliced_cz=ss.sliced_cz, slice_ids=[7],
                          fixed_cz=extra, fixed_s=[1, 0] * (len(extra) // 2) + [1] * (len(extra) % 2),
                          fuse_rows=1)
    info = B.peps_plan_info_get(h, 1, o)
    assert info["max_entries"] == sub.max_entries
    assert info["flops_per_chain"] == 8 * sum(sub.step_cmacs)
    o, keep = B.make_opts(sliced_cz=ss.sliced_cz, fixed_cz=[ss.sliced_cz[0]], fixed_s=[0])
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 1, o)   # a bit cannot be both sliced and fixed
    B.peps_destroy(h)


def test_seven_by_seven_needs_forty_cuts_for_64_gib():
    # every boundary between columns needs >= 7 cut bits for a 2^33 budget with
    # chi = 32 on 7 rows (2^40 -> 2^33), except that the last column's
    # boundary is counted once: the greedy choice finds 40
    circ, _ = workload("7x7_d40")
    ss = slicing.choose(circ, 2 ** 33, seed=5)
    assert len(ss.sliced_cz) == 40 and ss.max_entries == 2 ** 33
    assert slicing.choose(circ, 2 ** 33, seed=5).sliced_cz == ss.sliced_cz
    assert slicing.choose(circ, 2 ** 33, seed=6).sliced_cz != ss.sliced_cz


def test_sub_slices_extend_the_slice_set():
    circ, _ = workload("7x7_d40")
    ss = slicing.choose(circ, 2 ** 33, seed=5)
    sub = slicing.choose(circ, 2 ** 22, seed=5, base=ss.sliced_cz)
    assert set(ss.sliced_cz) <= set(sub.sliced_cz)
    assert sub.max_entries <= 2 ** 22


def test_seeded_slice_ids():
    ids = slicing.seeded_slice_ids(40, 5, 5)
    assert len(set(ids)) == 5 and all(0 <= i < 2 ** 40 for i in ids)
    assert ids == slicing.seeded_slice_ids(40, 5, 5)


def test_square_partition_chooser_fits_7x7_d40():
    # the square partition's slice set for 7x7 (1+40+1) under 200 GiB: a
    # dozen cut bits instead of forty, every quarter within 2^32 entries
    circ, _ = workload("7x7_d40")
    h = ctx_for(circ)
    ss = slicing.choose_quadrants(h, circ, 200 * 2 ** 30, seed=5)
    assert ss.workspace_bytes <= 200 * 2 ** 30
    assert len(ss.sliced_cz) <= 14 and ss.max_entries <= 2 ** 33
    assert ss.flops_per_slice * ss.n_slices < 2e18
    o, keep = B.make_opts(precision="fp16x3", scheme="quadrants", sliced_cz=ss.sliced_cz,
                          slice_ids=[0])
    info = B.peps_plan_info_get(h, 1, o)
    assert info["flops_per_chain"] == ss.flops_per_slice
    assert B.peps_workspace_bytes(h, 1, o) == ss.workspace_bytes
    # the unsliced plan is too large to run; the estimate flag still sizes it
    o, keep = B.make_opts(precision="fp16x3", scheme="quadrants")
    with pytest.raises(B.PepsError):
        B.peps_workspace_bytes(h, 1, o)
    o, keep = B.make_opts(precision="fp16x3", scheme="quadrants", flags=B.PEPS_FLAG_ESTIMATE)
    assert B.peps_plan_info_get(h, 1, o)["max_entries"] == 2 ** 40
    B.peps_destroy(h)


def test_lower_half_reuse_accounting():
    # odd side, one bitstring: the planner counts the lower half once per value
    # of its own bits; the chooser's closed form agrees with the planner's
    # figure for the call over every slice
    circ = make_circuit(5, 5, 16, 41)
    _, per = slicing.cz_edges(circ)
    sl = sorted([per[("h", 0, 1)][0], per[("h", 1, 1)][1], per[("v", 2, 3)][0], per[("h", 3, 2)][0]])
    h = ctx_for(circ)
    o, keep = B.make_opts(precision="fp16x3", scheme="quadrants", sliced_cz=sl, slice_ids=[0])
    one = B.peps_plan_info_get(h, 1, o)
    o, keep = B.make_opts(precision="fp16x3", scheme="quadrants", sliced_cz=sl)
    full = B.peps_plan_info_get(h, 1, o)
    mask = slicing.lower_half_mask(circ, sl)
    assert one["n_lower_bits"] == bin(mask).count("1") == 2
    assert 0 < one["flops_lower"] < one["flops_per_chain"]
    assert full["flops_call"] == pytest.approx(slicing.call_flops(one, len(sl)), rel=1e-12)
    assert full["flops_call"] < one["flops_per_chain"] * 2 ** len(sl)
    # several bitstrings: nothing is reused
    multi = B.peps_plan_info_get(h, 3, o)
    assert multi["flops_call"] == pytest.approx(3 * one["flops_per_chain"] * 2 ** len(sl), rel=1e-12)
    B.peps_destroy(h)


def test_slice_group_shares_the_lower_bits():
    mask = 0b1010011
    g = slicing.slice_group(7, mask, seed=5)
    assert len(g) == 2 ** 3 and len(set(g)) == len(g)
    assert len({x & mask for x in g}) == 1
    assert g == slicing.slice_group(7, mask, seed=5)


@pytest.mark.parametrize("R,C,depth,seed", [(4, 4, 12, 3), (3, 4, 16, 8), (4, 3, 10, 11)])
def test_vanishing_slices_against_the_oracle(R, C, depth, seed):
    # slice the last CZs of the circuit (where a run such as sqrt(Y) and the
    # final H ties a projector to the output bit): every slice the tie rule
    # rejects is zero in the oracle's sliced network, and the slices it keeps
    # sum to the amplitude
    from oracle import peps as op
    from rqc_inputs import make_circuit, uniform_bitstrings

    circ = make_circuit(R, C, depth, seed)
    ncz = sum(1 for g in circ.gates if g.kind == "cz")
    sl = list(range(ncz - 7, ncz))
    for x in uniform_bitstrings(R * C, 3, seed):
        x = int(x)
        keep = set(slicing.consistent_slice_ids(circ, sl, x))
        assert len(keep) < 2 ** len(sl)          # some tie holds for these circuits
        vals = {i: op.amplitudes(op.build(R, C, circ.gates, sliced=sl, slice_id=i), [x])[0]
                for i in range(2 ** len(sl))}
        full = op.amplitudes(op.build(R, C, circ.gates), [x])[0]
        scale = max(abs(v) for v in vals.values())
        for i, v in vals.items():
            if i not in keep:
                assert abs(v) <= 1e-12 * scale, (i, v)
        assert abs(sum(vals[i] for i in keep) - full) <= 1e-12 * abs(full)
        n_cons, n_low = slicing.slice_counts(circ, sl, x, 0)
        assert n_cons == len(keep) and n_low == 1


def test_ties_without_output_bits():
    # with no output bit only ties between projectors on one qubit (or to the
    # initial |0>) remain, and they never fix a bit to a constant after H
    from rqc_inputs import make_circuit

    circ = make_circuit(4, 4, 12, 3)
    ncz = sum(1 for g in circ.gates if g.kind == "cz")
    sl = list(range(ncz - 7, ncz))
    assert all(i >= 0 for _, i, _ in slicing.slice_constraints(circ, sl))
    assert len(slicing.consistent_slice_ids(circ, sl)) <= 2 ** len(sl)


def test_the_7x7_d40_amplitude_slice_set():
    # the set the whole-amplitude benchmark runs: chosen for the workload's
    # bitstring under 180 GB; most of its cuts are fixed by the bitstring, so
    # only ~100 slices can be nonzero, in a few runs sharing the lower half;
    # deterministic in the seed
    circ, bits = workload("7x7_d40")
    x = int(bits[0])
    h = ctx_for(circ)
    ss = slicing.choose_quadrants(h, circ, 180 * 10 ** 9, seed=5, x=x)
    ids = slicing.consistent_slice_ids(circ, ss.sliced_cz, x)
    mask = slicing.lower_half_mask(circ, ss.sliced_cz)
    assert ss.workspace_bytes <= 180 * 10 ** 9 and ss.max_entries <= 2 ** 33
    assert len(ids) <= 128 and len(ss.sliced_cz) >= 16
    assert slicing.slice_counts(circ, ss.sliced_cz, x, mask) == (len(ids), len({i & mask for i in ids}))
    # the planner's count of the call equals the chooser's total
    o, keep = B.make_opts(precision="fp16x3", scheme="quadrants", sliced_cz=ss.sliced_cz,
                          slice_ids=ids)
    assert B.peps_plan_info_get(h, 1, o)["flops_call"] == pytest.approx(ss.flops_total, rel=1e-12)
    assert ss.flops_total < 0.2 * 3.1e17     # under a fifth of the unsliced contraction
    again = slicing.choose_quadrants(h, circ, 180 * 10 ** 9, seed=5, x=x)
    assert again.sliced_cz == ss.sliced_cz
    B.peps_destroy(h)


def test_square_partition_chooser_keeps_the_cheapest_sets():
    # keep > 1: the cheapest sets found within the budget, cheapest first, each
    # within the budget; the first is the single choice
    circ, bits = workload("6x6_d32")
    h = ctx_for(circ)
    one = slicing.choose_quadrants(h, circ, 2 * 10 ** 9, seed=3)
    many = slicing.choose_quadrants(h, circ, 2 * 10 ** 9, seed=3, keep=3)
    assert 1 <= len(many) <= 3
    assert many[0].flops_total == one.flops_total
    assert all(a.flops_total <= b.flops_total for a, b in zip(many, many[1:]))
    assert all(s.workspace_bytes <= 2 * 10 ** 9 for s in many)
    B.peps_destroy(h)
