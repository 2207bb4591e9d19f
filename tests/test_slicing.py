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
