"""Parity of the square-partition contraction (supplementary Fig. S2(b)) on the
GPU, through the C ABI, with the CPU oracles: the state vector where it fits
(4x4) and the FP64 PEPS column sweep beyond (the amplitude does not depend on
the contraction order).  Tolerances as in test_gpu_parity: 1e-5 normwise for
FP32 and FP16X3, a bound from the unit roundoff for the other forms."""
import math

import numpy as np
import pytest

from oracle import peps as op
from oracle import statevector as sv
from paper_1905_08394_gb300 import binding as B
from rqc_inputs import make_circuit, prefix_group_bitstrings, uniform_bitstrings, workload

pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-5
UNIT_ROUNDOFF = {"bf16": 2.0 ** -8, "tf32": 2.0 ** -11, "fp16": 2.0 ** -11, "bf16x3": 2.0 ** -16}
QUAD = dict(scheme="quadrants")


def tol_for(prec, n_steps):
    if prec in ("fp32", "fp16x3"):
        return SPLIT_TOL
    return 8 * UNIT_ROUNDOFF[prec] * math.sqrt(n_steps)


def relerr(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def sim_factory(cuda_device):
    from paper_1905_08394_gb300 import Simulator

    made = []

    def make(circ):
        s = Simulator(circ.R, circ.C, device=cuda_device.index or 0)
        s.apply_circuit(circ)
        made.append(s)
        return s

    yield make
    for s in made:
        s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16x3", "tf32", "bf16x3"])
def test_4x4_d8_against_the_state_vector(sim_factory, prec):
    circ, bits = workload("4x4_d8")
    sim = sim_factory(circ)
    ref = sv.amplitudes(16, circ.gates, bits)
    out = sim.amplitudes(bits, precision=prec, **QUAD)
    assert relerr(out, ref) < tol_for(prec, 10)


def test_4x4_d16_against_the_state_vector(sim_factory):
    circ = make_circuit(4, 4, 16, 5)
    bits = uniform_bitstrings(16, 128, 5)
    sim = sim_factory(circ)
    ref = sv.amplitudes(16, circ.gates, bits)
    for prec in ("fp32", "fp16x3"):
        assert relerr(sim.amplitudes(bits, precision=prec, **QUAD), ref) < SPLIT_TOL


@pytest.fixture(scope="module")
def d24(sim_factory):
    circ, bits = workload("6x6_d24")
    bits = bits[:16]
    ref = op.amplitudes(op.build(6, 6, circ.gates), bits)
    return circ, bits, ref, sim_factory(circ)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "bf16x3", "fp16", "fp16x3"])
def test_6x6_d24_every_form(d24, prec):
    circ, bits, ref, sim = d24
    out = sim.amplitudes(bits, precision=prec, **QUAD)
    assert relerr(out, ref) < tol_for(prec, 38)


def test_6x6_d24_agrees_with_the_column_sweep(d24):
    circ, bits, ref, sim = d24
    a = sim.amplitudes(bits, precision="fp16x3", **QUAD)
    b = sim.amplitudes(bits, precision="fp16x3")
    assert relerr(a, b) < 2 * SPLIT_TOL


def test_6x6_d16_prefix_groups_and_lanes(sim_factory):
    circ = make_circuit(6, 6, 16, 9)
    bits = prefix_group_bitstrings(6, 6, 3, 3, 12, 9)
    sim = sim_factory(circ)
    ref = op.amplitudes(op.build(6, 6, circ.gates), bits)
    for prec in ("fp32", "fp16x3"):
        plain = sim.amplitudes(bits, precision=prec, **QUAD)
        grouped = sim.amplitudes(bits, precision=prec, prefix_cols=3, prefix_group=12,
                                 max_lanes=5, **QUAD)
        assert relerr(plain, ref) < SPLIT_TOL and relerr(grouped, ref) < SPLIT_TOL


def test_even_rectangle(sim_factory):
    circ = make_circuit(4, 6, 16, 12)
    bits = uniform_bitstrings(24, 24, 12)
    sim = sim_factory(circ)
    ref = op.amplitudes(op.build(4, 6, circ.gates), bits)
    assert relerr(sim.amplitudes(bits, precision="fp16x3", **QUAD), ref) < SPLIT_TOL


def test_slices_sum_to_the_unsliced_amplitude(sim_factory):
    circ = make_circuit(6, 6, 16, 13)
    bits = uniform_bitstrings(36, 6, 13)
    sim = sim_factory(circ)
    full = sim.amplitudes(bits, precision="fp32", **QUAD)
    sliced = [2, 30, 77]
    tot = sim.amplitudes(bits, precision="fp32", sliced_cz=sliced, **QUAD)
    assert relerr(tot, full) < 1e-6
    one = sim.amplitudes(bits, precision="fp32", sliced_cz=sliced, slice_ids=[5], **QUAD)
    ref = op.amplitudes(op.build(6, 6, circ.gates, sliced=sliced, slice_id=5), bits)
    assert relerr(one, ref) < SPLIT_TOL


def test_graph_replay_is_bit_identical(sim_factory):
    circ = make_circuit(6, 6, 16, 14)
    bits = prefix_group_bitstrings(6, 6, 3, 2, 8, 14)
    sim = sim_factory(circ)
    kw = dict(precision="fp16x3", prefix_cols=3, prefix_group=8, max_lanes=4, **QUAD)
    eager = sim.amplitudes(bits, **kw)
    g1 = sim.amplitudes(bits, flags=B.PEPS_FLAG_GRAPH, **kw)
    g2 = sim.amplitudes(bits, flags=B.PEPS_FLAG_GRAPH, **kw)
    assert np.array_equal(g1, eager) and np.array_equal(g2, eager)


def test_autotune_chooses_an_order_and_caches_it(sim_factory, tmp_path):
    import torch

    from paper_1905_08394_gb300 import autotune

    circ = make_circuit(6, 6, 16, 15)
    bits = prefix_group_bitstrings(6, 6, 3, 2, 12, 15)
    sim = sim_factory(circ)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    d_out = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
    kw = dict(precision="fp16x3", prefix_cols=3, prefix_group=12, max_lanes=4)
    cache = str(tmp_path / "tune.json")
    cands = [{"scheme": "columns"}, {"scheme": "quadrants"}]
    best = autotune.tune(sim, d_bits, d_out, kw, cands=cands, repeats=1, cache=cache)
    assert best in cands
    again = autotune.tune(sim, d_bits, d_out, kw, cands=cands, repeats=1, cache=cache)
    assert again == best
    ref = op.amplitudes(op.build(6, 6, circ.gates), bits)
    out = sim.amplitudes(bits, **kw, **best)
    assert relerr(out, ref) < SPLIT_TOL


# ---------------------------------------------------------------------------
# Odd side (Fig. S2(c)): ul (m+1) x m, ur (m+1) x (m+1) with the centre site,
# bl m x (m+1), br m x m; F_u = F_ul F_ur, F_b = F_bl F_br, amplitude F_u . F_b
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_odd_3x3_against_the_state_vector(sim_factory, prec):
    circ = make_circuit(3, 3, 16, 31)
    x = np.arange(512, dtype=np.uint64)
    ref = sv.amplitudes(9, circ.gates, x)
    sim = sim_factory(circ)
    assert relerr(sim.amplitudes(x, precision=prec, **QUAD), ref) < SPLIT_TOL


def test_odd_5x5_against_the_column_oracle(sim_factory):
    circ = make_circuit(5, 5, 16, 32)
    x = uniform_bitstrings(25, 16, 32)
    ref = op.amplitudes(op.build(5, 5, circ.gates), x)
    sim = sim_factory(circ)
    for prec in ("fp32", "fp16x3", "bf16x3"):
        assert relerr(sim.amplitudes(x, precision=prec, **QUAD), ref) < tol_for(prec, 22), prec


def test_odd_7x7_d24_against_the_golden_values(sim_factory):
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_7x7_d24.json")) as f:
        g = json.load(f)
    circ = make_circuit(7, 7, 24, 5)
    x = np.array(g["bitstrings"], dtype=np.uint64)
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])
    sim = sim_factory(circ)
    for prec in ("fp32", "fp16x3"):
        assert relerr(sim.amplitudes(x, precision=prec, **QUAD), ref) < SPLIT_TOL, prec
    # and the two schemes agree
    assert relerr(sim.amplitudes(x, precision="fp16x3", **QUAD), sim.amplitudes(x, precision="fp16x3")) < 2 * SPLIT_TOL


def test_odd_slices_sum_to_the_unsliced_amplitude(sim_factory):
    # a sliced bit on the horizontal cut (the quarters' batch legs), one on the
    # upper vertical cut and one inside ur
    circ = make_circuit(5, 5, 16, 33)
    bits = uniform_bitstrings(25, 4, 33)
    from paper_1905_08394_gb300 import slicing

    _, per = slicing.cz_edges(circ)
    sliced = sorted([per[("v", 2, 1)][0], per[("h", 1, 1)][1], per[("h", 0, 3)][0]])
    sim = sim_factory(circ)
    full = sim.amplitudes(bits, precision="fp32", **QUAD)
    tot = sim.amplitudes(bits, precision="fp32", sliced_cz=sliced, **QUAD)
    assert relerr(tot, full) < 1e-6
    for sid in (3, 6):
        one = sim.amplitudes(bits, precision="fp16x3", sliced_cz=sliced, slice_ids=[sid], **QUAD)
        ref = op.amplitudes(op.build(5, 5, circ.gates, sliced=sliced, slice_id=sid), bits)
        assert relerr(one, ref) < SPLIT_TOL, sid


def test_odd_7x7_d24_chosen_slices_against_the_golden_values(sim_factory):
    # the slice chooser of the square partition under a 64 MiB workspace budget
    # (the unsliced plan needs ~456 MiB); the slice sum is the amplitude
    import json
    import os

    from paper_1905_08394_gb300 import binding as Bn
    from paper_1905_08394_gb300 import slicing

    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_7x7_d24.json")) as f:
        g = json.load(f)
    circ = make_circuit(7, 7, 24, 5)
    x = np.array(g["bitstrings"], dtype=np.uint64)[:2]
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])[:2]
    sim = sim_factory(circ)
    ss = slicing.choose_quadrants(sim.h, circ, 64 * 2 ** 20, seed=5)
    assert 0 < len(ss.sliced_cz) <= 10 and ss.workspace_bytes <= 64 * 2 ** 20
    o, keep = Bn.make_opts(precision="fp16x3", scheme="quadrants", sliced_cz=ss.sliced_cz)
    assert Bn.peps_workspace_bytes(sim.h, len(x), o) <= 2 * 64 * 2 ** 20
    for prec in ("fp32", "fp16x3"):
        out = sim.amplitudes(x, precision=prec, sliced_cz=ss.sliced_cz, **QUAD)
        assert relerr(out, ref) < SPLIT_TOL, prec


def test_odd_one_bitstring_reuses_the_lower_half(sim_factory):
    # one bitstring: slices that share their lower-half bits keep F_b; the sum
    # over every slice is the amplitude, a sub-list of slices the oracle's
    # sum over the same slices, and a call with one slice per group agrees
    from paper_1905_08394_gb300 import slicing

    circ = make_circuit(5, 5, 16, 41)
    _, per = slicing.cz_edges(circ)
    sl = sorted([per[("h", 0, 1)][0], per[("h", 1, 1)][1], per[("v", 2, 3)][0], per[("h", 3, 2)][0]])
    x = uniform_bitstrings(25, 1, 41)
    sim = sim_factory(circ)
    full = sim.amplitudes(x, precision="fp16x3", **QUAD)
    tot = sim.amplitudes(x, precision="fp16x3", sliced_cz=sl, **QUAD)
    assert relerr(tot, full) < SPLIT_TOL
    st = sim.stats()
    assert st["launches_contract"] < 16 * sim.plan_info(1, precision="fp16x3", sliced_cz=sl,
                                                          slice_ids=[0], **QUAD)["n_launches"]
    ids = [9, 3, 12, 1, 11]
    part = sim.amplitudes(x, precision="fp16x3", sliced_cz=sl, slice_ids=ids, **QUAD)
    ref = sum(op.amplitudes(op.build(5, 5, circ.gates, sliced=sl, slice_id=i), x) for i in ids)
    assert relerr(part, ref) < SPLIT_TOL
    for i in ids:
        one = sim.amplitudes(x, precision="fp16x3", sliced_cz=sl, slice_ids=[i], **QUAD)
        r1 = op.amplitudes(op.build(5, 5, circ.gates, sliced=sl, slice_id=i), x)
        assert np.abs(one - r1).max() < SPLIT_TOL * np.abs(full).max(), i


def test_7x7_d32_sliced_square_partition_against_the_column_sweep(sim_factory):
    # the 7x7 geometry at bond dimension 16, whole: the slices the square
    # partition's chooser picks for one bitstring under 4 GiB, only those the
    # tie rule keeps, sum to the unsliced square partition, which agrees with
    # the column sweep; slices the rule rejects vanish on the GPU
    from paper_1905_08394_gb300 import slicing

    circ = make_circuit(7, 7, 32, 5)
    x = uniform_bitstrings(49, 1, 5)
    sim = sim_factory(circ)
    col = sim.amplitudes(x, precision="fp16x3")
    quad = sim.amplitudes(x, precision="fp16x3", **QUAD)
    assert relerr(quad, col) < 2 * SPLIT_TOL
    ss = slicing.choose_quadrants(sim.h, circ, 4 << 30, seed=5, x=int(x[0]))
    keep = slicing.consistent_slice_ids(circ, ss.sliced_cz, int(x[0]))
    assert 0 < len(keep) < 2 ** len(ss.sliced_cz)
    tot = sim.amplitudes(x, precision="fp16x3", sliced_cz=ss.sliced_cz, slice_ids=keep, **QUAD)
    assert relerr(tot, quad) < SPLIT_TOL
    drop = [i for i in range(min(2 ** len(ss.sliced_cz), 4096)) if i not in set(keep)][:4]
    for i in drop:
        z = sim.amplitudes(x, precision="fp16x3", sliced_cz=ss.sliced_cz, slice_ids=[i], **QUAD)
        assert abs(z[0]) <= 1e-12 * abs(quad[0]), i
