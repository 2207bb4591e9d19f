"""Marginal probabilities P(x_S) = <psi|Pi_S|psi> on the GPU (the double-layer
network through the same contraction kernels), against the CPU oracles: the
state vector's sums where it fits, the oracle's double-layer contraction
beyond.  Metric: normwise relative error over the checked set, 1e-5 for FP32
and FP16X3."""
import numpy as np
import pytest

from oracle import peps as op
from oracle import statevector as sv
from rqc_inputs import make_circuit, uniform_bitstrings

pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("scheme", ["columns", "quadrants"])
@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_4x4_against_the_state_vector(sim_factory, scheme, prec):
    circ = make_circuit(4, 4, 16, 21)
    x = uniform_bitstrings(16, 32, 21)
    sim = sim_factory(circ)
    for mask in (0x0001, 0x00FF, 0x5A5A, 0xFFFF):
        ref = sv.marginals(16, circ.gates, x, mask)
        got = sim.amplitudes(x, precision=prec, scheme=scheme, measured_mask=mask)
        assert relerr(got.real, ref) < TOL, mask
        assert np.abs(got.imag).max() < 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("scheme", ["columns", "quadrants"])
def test_5x5_against_the_state_vector(sim_factory, scheme):
    # quadrants: the odd-side square partition (Fig. S2(c)) on the double layer
    circ = make_circuit(5, 5, 16, 22)
    x = uniform_bitstrings(25, 8, 22)
    sim = sim_factory(circ)
    mask = (1 << 12) - 1
    ref = sv.marginals(25, circ.gates, x, mask)
    for prec in ("fp32", "fp16x3"):
        got = sim.amplitudes(x, precision=prec, scheme=scheme, measured_mask=mask)
        assert relerr(got.real, ref) < TOL, prec


def test_3x3_odd_partition_every_mask(sim_factory):
    circ = make_circuit(3, 3, 16, 23)
    x = uniform_bitstrings(9, 16, 23)
    sim = sim_factory(circ)
    for mask in (0x001, 0x010, 0x0F0, 0x1FF):
        ref = sv.marginals(9, circ.gates, x, mask)
        got = sim.amplitudes(x, precision="fp16x3", scheme="quadrants", measured_mask=mask)
        assert relerr(got.real, ref) < TOL, mask


def test_special_cases(sim_factory):
    circ = make_circuit(4, 4, 16, 23)
    x = uniform_bitstrings(16, 16, 23)
    sim = sim_factory(circ)
    # nothing measured: the norm; everything measured: |amplitude|^2
    one = sim.amplitudes(x, precision="fp16x3", measured_mask=0)
    assert np.abs(one.real - 1).max() < TOL
    amp = sim.amplitudes(x, precision="fp32")
    full = sim.amplitudes(x, precision="fp32", measured_mask=0xFFFF)
    assert relerr(full.real, np.abs(amp) ** 2) < TOL
    # the 2^k marginals of the first k qubits sum to 1
    k = 6
    xs = np.arange(1 << k, dtype=np.uint64)
    tot = sim.amplitudes(xs, precision="fp16x3", measured_mask=(1 << k) - 1).real.sum()
    assert abs(tot - 1) < TOL


@pytest.mark.parametrize("scheme", ["columns", "quadrants"])
def test_6x6_against_the_double_layer_oracle(sim_factory, scheme):
    # 6x6 (1+16+1): the double layer has bond dimension 16, the size of the
    # 6x6 (1+32+1) amplitude; the oracle contracts it by the square partition
    circ = make_circuit(6, 6, 16, 24)
    x = uniform_bitstrings(36, 2, 24)
    mask = (1 << 18) - 1
    p = op.build(6, 6, circ.gates)
    ref = np.array([op.marginal_quadrant(p, int(b), mask) for b in x])
    sim = sim_factory(circ)
    got = sim.amplitudes(x, precision="fp16x3", scheme=scheme, measured_mask=mask)
    assert relerr(got.real, ref) < TOL
