"""General two-qubit gates (main-text "factorize": operator-Schmidt split,
rank 1..4) through the C ABI on the GPU, against the state vector and the
FP64 PEPS oracle.  Bond dimensions become products of ranks (3 included), so
some steps run on the CUDA-core kernel.  Tolerance 1e-5 normwise for FP32
and FP16X3."""
import numpy as np
import pytest

from oracle import peps as op
from oracle import statevector as sv
from rqc_inputs import make_circuit_general, uniform_bitstrings

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


@pytest.mark.parametrize("R,C,layers,seed", [(2, 2, 2, 1), (3, 3, 3, 2), (4, 4, 3, 3)])
@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_against_the_state_vector(sim_factory, R, C, layers, seed, prec):
    circ = make_circuit_general(R, C, layers, seed)
    n = R * C
    x = np.arange(1 << n, dtype=np.uint64) if n <= 9 else uniform_bitstrings(n, 256, seed)
    ref = sv.amplitudes(n, circ.gates, x)
    sim = sim_factory(circ)
    assert relerr(sim.amplitudes(x, precision=prec), ref) < TOL


def test_5x5_and_both_schemes(sim_factory):
    circ = make_circuit_general(4, 6, 4, 4)
    x = uniform_bitstrings(24, 16, 4)
    ref = op.amplitudes(op.build(4, 6, circ.gates), x)
    sim = sim_factory(circ)
    for scheme in ("columns", "quadrants"):
        assert relerr(sim.amplitudes(x, precision="fp16x3", scheme=scheme), ref) < TOL, scheme
    circ5 = make_circuit_general(5, 5, 3, 5)
    x5 = uniform_bitstrings(25, 16, 5)
    ref5 = sv.amplitudes(25, circ5.gates, x5)
    sim5 = sim_factory(circ5)
    assert relerr(sim5.amplitudes(x5, precision="fp16x3"), ref5) < TOL


def test_marginals_with_general_gates(sim_factory):
    circ = make_circuit_general(3, 4, 3, 6)
    x = uniform_bitstrings(12, 16, 6)
    ref = sv.marginals(12, circ.gates, x, 0b111100001111)
    sim = sim_factory(circ)
    got = sim.amplitudes(x, precision="fp32", measured_mask=0b111100001111)
    assert relerr(got.real, ref) < TOL
