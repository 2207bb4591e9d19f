"""The allocation-free entry point, for callers that cannot call cudaMalloc
(code inside another framework's memory pool, plug-ins whose host owns every
device allocation).  It must give the same amplitudes as the ordinary device
entry point, call after call, although every call reuses one static device
array inside the library.  Collected last on purpose (file name), so that a
run stopping at the first failure has run every other test already."""
import numpy as np
import pytest

from paper_1905_08394_gb300 import binding as B
from rqc_inputs import make_circuit, uniform_bitstrings, workload

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the tolerance the FP32 parity tests use


def _ctx(circ):
    h = B.peps_create(circ.R, circ.C)
    C = circ.C
    for g in circ.gates:
        if g.kind == "1q":
            q = g.qubits[0]
            B.peps_apply_1q(h, q // C, q % C, g.U)
        else:
            a, b = g.qubits
            B.peps_apply_cz(h, a // C, a % C, b // C, b % C)
    return h


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_device_entry_point_twice(cuda_device):
    import torch

    circ = make_circuit(4, 5, 16, 21)
    bits = uniform_bitstrings(20, 96, 21)
    h = _ctx(circ)
    stream = torch.cuda.current_stream().cuda_stream
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()

    # ordinary entry point, caller-owned workspace
    opts, keep = B.make_opts(precision="fp32")
    need = B.peps_workspace_bytes(h, len(bits), opts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    ref = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
    B.peps_amplitudes_device(h, d_bits.data_ptr(), len(bits), ref.data_ptr(), opts,
                             ws.data_ptr(), need, stream)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()

    # a second context in between, so the shared scratch holds other contents
    other = _ctx(make_circuit(3, 3, 8, 5))
    other_bits = torch.from_numpy(uniform_bitstrings(9, 8, 5).view(np.int64)).cuda()
    other_out = torch.empty(8, dtype=torch.complex128, device="cuda")

    for call in range(2):
        out = torch.full((len(bits),), complex(np.nan, np.nan), dtype=torch.complex128,
                         device="cuda")
        B.peps_amplitudes_noalloc(h, d_bits.data_ptr(), len(bits), out.data_ptr(), opts, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert _relerr(got, ref) < TOL, f"call {call}"
        B.peps_amplitudes_noalloc(other, other_bits.data_ptr(), 8, other_out.data_ptr(), opts,
                                  stream)
        torch.cuda.synchronize()
    B.peps_destroy(other)
    B.peps_destroy(h)


def test_noalloc_rejects_workloads_beyond_its_scratch(cuda_device):
    import torch

    circ, bits = workload("6x6_d32")
    h = _ctx(circ)
    opts, keep = B.make_opts(precision="fp16x3")
    d_bits = torch.from_numpy(bits[:4].view(np.int64)).cuda()
    out = torch.empty(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.PepsError) as e:
        B.peps_amplitudes_noalloc(h, d_bits.data_ptr(), 4, out.data_ptr(), opts,
                                  torch.cuda.current_stream().cuda_stream)
    assert e.value.code == B.PEPS_ENOMEM
    assert "static scratch" in str(e.value)
    B.peps_destroy(h)
