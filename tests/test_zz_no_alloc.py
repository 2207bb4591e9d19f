"""The allocation-free entry point, for callers that cannot call cudaMalloc
(code inside another framework's memory pool, plug-ins whose host owns every
device allocation).  It must give the same amplitudes as the ordinary device
entry point, call after call, although every call reuses one static device
array inside the library.  Both entry points run the same deterministic
kernels, so the outputs must be bit-identical: stale scratch contents leaking
into a result at any magnitude would show.  Collected last on purpose (file
name), so that a run stopping at the first failure has run every other test
already."""
import numpy as np
import pytest

from paper_1905_08394_gb300 import binding as B
from rqc_inputs import make_circuit, uniform_bitstrings, workload

pytestmark = pytest.mark.gpu


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


def _device_call(h, bits, opts, stream):
    """The ordinary entry point with a caller-owned workspace."""
    import torch

    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    need = B.peps_workspace_bytes(h, len(bits), opts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
    B.peps_amplitudes_device(h, d_bits.data_ptr(), len(bits), out.data_ptr(), opts,
                             ws.data_ptr(), need, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_device_entry_point_twice(cuda_device):
    import torch

    circ = make_circuit(4, 5, 16, 21)
    bits = uniform_bitstrings(20, 96, 21)
    h = _ctx(circ)
    stream = torch.cuda.current_stream().cuda_stream
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    opts, keep = B.make_opts(precision="fp32")
    ref = _device_call(h, bits, opts, stream)

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
        assert np.array_equal(got, ref), f"call {call}"
        B.peps_amplitudes_noalloc(other, other_bits.data_ptr(), 8, other_out.data_ptr(), opts,
                                  stream)
        torch.cuda.synchronize()
    B.peps_destroy(other)
    B.peps_destroy(h)


def test_noalloc_back_to_back_on_one_stream(cuda_device):
    """Two contexts called one after the other on a non-blocking stream with no
    synchronisation in between: the second call's table upload must wait for
    the first call's kernels, which still read the same scratch."""
    import torch

    circ_a, bits_a = workload("5x5_d16")
    circ_b = make_circuit(4, 5, 16, 21)
    bits_b = uniform_bitstrings(20, 96, 21)
    ha, hb = _ctx(circ_a), _ctx(circ_b)
    opts, keep = B.make_opts(precision="fp32", max_lanes=64)
    s = torch.cuda.Stream()
    ref_a = _device_call(ha, bits_a, opts, s.cuda_stream)
    ref_b = _device_call(hb, bits_b, opts, s.cuda_stream)

    da = torch.from_numpy(bits_a.view(np.int64)).cuda()
    db = torch.from_numpy(bits_b.view(np.int64)).cuda()
    torch.cuda.synchronize()
    outs = []
    for _ in range(2):
        oa = torch.empty(len(bits_a), dtype=torch.complex128, device="cuda")
        ob = torch.empty(len(bits_b), dtype=torch.complex128, device="cuda")
        outs.append((oa, ob))
    with torch.cuda.stream(s):
        for oa, ob in outs:
            B.peps_amplitudes_noalloc(ha, da.data_ptr(), len(bits_a), oa.data_ptr(), opts,
                                      s.cuda_stream)
            B.peps_amplitudes_noalloc(hb, db.data_ptr(), len(bits_b), ob.data_ptr(), opts,
                                      s.cuda_stream)
    s.synchronize()
    for i, (oa, ob) in enumerate(outs):
        assert np.array_equal(oa.cpu().numpy(), ref_a), f"round {i}: context A"
        assert np.array_equal(ob.cpu().numpy(), ref_b), f"round {i}: context B"
    B.peps_destroy(ha)
    B.peps_destroy(hb)


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
    for flag in (B.PEPS_FLAG_TIMING, B.PEPS_FLAG_GRAPH):
        small, keep2 = B.make_opts(precision="fp32", flags=flag)
        with pytest.raises(B.PepsError) as e:
            B.peps_amplitudes_noalloc(h, d_bits.data_ptr(), 4, out.data_ptr(), small,
                                      torch.cuda.current_stream().cuda_stream)
        assert e.value.code == B.PEPS_EINVAL
    B.peps_destroy(h)
