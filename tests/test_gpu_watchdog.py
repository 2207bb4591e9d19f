"""Failure detection on the GPU without a fault: every wait of the tensor-core
contraction kernel is bounded by the call's watchdog budget.  With a budget of
1 ns the waits run out, the kernel raises the device timeout word, drains its
copies and MMAs, frees its tensor memory and returns; the call reports
PEPS_ETIMEOUT, the context refuses further calls with PEPS_ESTATE, it can
still be destroyed, and a fresh context on the same device computes correct
amplitudes (the CUDA context survived)."""
import numpy as np
import pytest

from oracle import peps as op
from paper_1905_08394_gb300 import binding as B
from rqc_inputs import make_circuit, uniform_bitstrings

pytestmark = pytest.mark.gpu


def test_watchdog_expiry_is_reported_and_the_device_stays_usable(cuda_device):
    from paper_1905_08394_gb300 import Simulator

    circ = make_circuit(6, 6, 24, 3)
    bits = uniform_bitstrings(36, 8, 3)
    ref = op.amplitudes(op.build(6, 6, circ.gates), bits)

    sim = Simulator(6, 6)
    sim.apply_circuit(circ)
    assert sim.plan_info(len(bits), precision="fp16x3")["n_tc_launches"] > 0
    with pytest.raises(B.PepsError) as e:
        sim.amplitudes(bits, precision="fp16x3", watchdog_ns=1)
    assert e.value.code == B.PEPS_ETIMEOUT, str(e.value)
    with pytest.raises(B.PepsError) as e:
        sim.amplitudes(bits, precision="fp16x3")
    assert e.value.code == B.PEPS_ESTATE
    sim.close()          # peps_destroy succeeds on a broken context

    fresh = Simulator(6, 6)
    fresh.apply_circuit(circ)
    out = fresh.amplitudes(bits, precision="fp16x3")
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-5
    assert fresh.stats()["launches_contract_tc"] > 0
    fresh.close()
