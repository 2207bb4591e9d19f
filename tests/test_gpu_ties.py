"""Held Schmidt bits (PEPS_FLAG_HOLD_TIES) on the GPU: every CZ bit that the
output bitstring fixes takes only its tied value, and each site operand has a
variant per value of the output bits it depends on.  The amplitudes must be
those of the unheld network: against the state vector and the FP64 oracle,
for both contraction schemes, with prefix groups, in the bench configuration
against the stored oracle values.  Tolerance 1e-5 normwise (FP32, FP16X3)."""
import json
import os

import numpy as np
import pytest

from oracle import peps as op
from oracle import statevector as sv
from rqc_inputs import make_circuit, uniform_bitstrings, workload

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-5


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


@pytest.mark.parametrize("R,C,d,seed", [(4, 4, 16, 9), (4, 4, 24, 3), (3, 5, 32, 2),
                                        (5, 5, 16, 2)])
@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_held_bits_against_the_state_vector(sim_factory, R, C, d, seed, prec):
    circ = make_circuit(R, C, d, seed)
    n = R * C
    x = uniform_bitstrings(n, 512, seed)
    ref = sv.amplitudes(n, circ.gates, x)
    sim = sim_factory(circ)
    assert sim.plan_info(len(x), precision=prec, hold_ties=True)["flops_call"] < \
        sim.plan_info(len(x), precision=prec)["flops_call"]
    for scheme in (("columns", "quadrants") if R % 2 == 0 and C % 2 == 0 or R == C else
                   ("columns",)):
        got = sim.amplitudes(x, precision=prec, hold_ties=True, scheme=scheme, max_lanes=32)
        assert relerr(got, ref) < TOL, scheme


@pytest.mark.parametrize("scheme", ["columns", "quadrants"])
def test_held_bits_with_prefix_groups_6x6_d24(sim_factory, scheme):
    from rqc_inputs import prefix_group_bitstrings

    circ = make_circuit(6, 6, 24, 3)
    bits = prefix_group_bitstrings(6, 6, 3, 4, 16, 3)
    ref = op.amplitudes(op.build(6, 6, circ.gates), bits[::5])
    sim = sim_factory(circ)
    for prec in ("fp32", "fp16x3"):
        got = sim.amplitudes(bits, precision=prec, hold_ties=True, prefix_cols=3, prefix_group=16,
                             max_lanes=16, scheme=scheme)
        assert relerr(got[::5], ref) < TOL, prec


def test_held_bits_with_general_gates(sim_factory):
    # a general two-qubit gate in the middle of a CZ circuit: it cuts the ties
    # through its qubits, and the CZ bits on its edge (not addressable) stay
    # unheld; the rest are held
    from rqc_inputs import Circuit, Gate, two_qubit_test_gates

    base = make_circuit(4, 4, 24, 9)
    k = len(base.gates) // 2
    G = two_qubit_test_gates(9)[0]
    gates = base.gates[:k] + [Gate("2q", (5, 6), "G", G), Gate("2q", (10, 14), "G", G)] + \
        base.gates[k:]
    circ = Circuit(4, 4, 24, 9, gates)
    x = uniform_bitstrings(16, 256, 3)
    ref = sv.amplitudes(16, circ.gates, x)
    sim = sim_factory(circ)
    for prec in ("fp32", "fp16x3"):
        got = sim.amplitudes(x, precision=prec, hold_ties=True)
        assert relerr(got, ref) < TOL, prec


def test_bench_configuration_held(sim_factory):
    with open(os.path.join(HERE, "golden", "oracle_6x6_d32.json")) as f:
        g = json.load(f)
    circ, bits = workload("6x6_d32")
    idx = g["indices"]
    assert [int(bits[i]) for i in idx] == g["bitstrings"]
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])
    sim = sim_factory(circ)
    kw = dict(prefix_cols=3, prefix_group=64, max_lanes=16, hold_ties=True)
    for scheme in ("quadrants", "columns"):
        out = sim.amplitudes(bits, precision="fp16x3", scheme=scheme, **kw)
        err = relerr(out[idx], ref)
        print(f"6x6 d32 fp16x3 {scheme}, held bits: normwise rel.err {err:.3e}")
        assert err < TOL, scheme
    # the FP32 comparator as the bench times it: group 0 by the square partition
    out = sim.amplitudes(bits[:64], precision="fp32", scheme="quadrants", **kw)
    pos = [k for k, i in enumerate(idx) if i < 64]
    err = relerr(out[[idx[k] for k in pos]], ref[pos])
    print(f"6x6 d32 fp32 square partition, held bits, group 0: normwise rel.err {err:.3e}")
    assert err < TOL
