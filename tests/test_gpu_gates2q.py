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


def test_orientation_closed_forms(sim_factory):
    """G[(t0 t1), (s0 s1)] with the first-named qubit first, through the C ABI:
    CNOT (control first), a cyclic permutation (not symmetric, so a transposed
    G fails) given in both qubit orders, and a random U whose action on |00>
    is its first column.  Expected amplitudes written out, every other one 0."""
    from types import SimpleNamespace

    from rqc_inputs import Gate

    X = np.array([[0, 1], [1, 0]], dtype=complex)
    CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    CYC = np.zeros((4, 4), dtype=complex)
    for s, t in ((0, 1), (1, 3), (3, 2), (2, 0)):
        CYC[t, s] = 1.0
    z = np.random.default_rng(5).normal(size=(4, 4, 2)) @ np.array([1, 1j])
    U, _ = np.linalg.qr(z)
    q0, q1 = 1, 3
    bit = lambda t0, t1: (t0 << q0) | (t1 << q1)
    g1 = lambda q, M: Gate("1q", (q,), "U", M)
    g2 = lambda a, b, M: Gate("2q", (a, b), "G", M)
    cases = [([g1(q0, X), g2(q0, q1, CNOT)], {bit(1, 1): 1.0}),
             ([g1(q0, X), g2(q1, q0, CNOT)], {bit(1, 0): 1.0}),
             ([g2(q0, q1, CYC)], {bit(0, 1): 1.0}),
             ([g2(q1, q0, CYC)], {bit(1, 0): 1.0}),
             ([g2(q0, q1, U)], {bit(a, b): U[2 * a + b, 0] for a in (0, 1) for b in (0, 1)})]
    allx = np.arange(16, dtype=np.uint64)
    for k, (gates, amps) in enumerate(cases):
        ref = np.zeros(16, dtype=complex)
        for x, a in amps.items():
            ref[x] = a
        sim = sim_factory(SimpleNamespace(R=2, C=2, gates=gates))
        for prec in ("fp32", "fp16x3"):
            got = sim.amplitudes(allx, precision=prec)
            assert np.abs(got - ref).max() < 1e-6, (k, prec)
