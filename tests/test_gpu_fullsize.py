"""Full-size parity: the 6x6 (1+32+1) batch in the launch configuration that
bench.py times (512 bitstrings, 8 groups x 64 sharing columns 0-2, prefix
reuse, 16 lanes), against FP64 oracle amplitudes of 8 of the bitstrings
(tests/golden/oracle_6x6_d32.json, written by tests/golden/make_oracle_values.py
from oracle/ only), and the Porter-Thomas statistics of all 512."""
import json
import math
import os

import numpy as np
import pytest

from rqc_inputs import workload

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-5


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "oracle_6x6_d32.json")) as f:
        g = json.load(f)
    circ, bits = workload("6x6_d32")
    assert [int(bits[i]) for i in g["indices"]] == g["bitstrings"]
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])
    return circ, bits, g["indices"], ref


@pytest.fixture(scope="module")
def sim(golden, cuda_device):
    from paper_1905_08394_gb300 import Simulator

    circ = golden[0]
    s = Simulator(6, 6)
    s.apply_circuit(circ)
    yield s
    s.close()


def test_bench_configuration_fp16x3(golden, sim):
    circ, bits, idx, ref = golden
    out = sim.amplitudes(bits, precision="fp16x3", prefix_cols=3, prefix_group=64,
                         max_lanes=16)
    err = float(np.linalg.norm(out[idx] - ref) / np.linalg.norm(ref))
    print(f"6x6 d32 fp16x3 batched: normwise rel.err {err:.3e} on 8 oracle bitstrings")
    assert err < TOL
    # Porter-Thomas: N |a|^2 ~ Exp(1) for a deep random circuit
    pt = np.sort((2.0 ** 36) * np.abs(out) ** 2)
    assert abs(pt.mean() - 1) < 3 / math.sqrt(len(pt))
    assert abs(np.mean(pt ** 2) - 2) < 0.5
    # Kolmogorov-Smirnov distance to Exp(1): p > 0.01 needs D < 1.63 / sqrt(n)
    cdf = 1 - np.exp(-pt)
    ecdf_hi = np.arange(1, len(pt) + 1) / len(pt)
    ecdf_lo = np.arange(0, len(pt)) / len(pt)
    D = max(np.max(ecdf_hi - cdf), np.max(cdf - ecdf_lo))
    assert D < 1.63 / math.sqrt(len(pt))


def test_bench_configuration_square_partition(golden, sim):
    # the same 512 bitstrings by the square partition (quarters of 3 x 3, left
    # half shared by each group of 64); the amplitude does not depend on the order
    circ, bits, idx, ref = golden
    out = sim.amplitudes(bits, precision="fp16x3", prefix_cols=3, prefix_group=64,
                         max_lanes=16, scheme="quadrants")
    err = float(np.linalg.norm(out[idx] - ref) / np.linalg.norm(ref))
    print(f"6x6 d32 fp16x3 square partition: normwise rel.err {err:.3e} on 8 oracle bitstrings")
    assert err < TOL
    pt = (2.0 ** 36) * np.abs(out) ** 2
    assert abs(pt.mean() - 1) < 3 / math.sqrt(len(pt))


def test_fp32_path_on_the_oracle_groups(golden, sim):
    circ, bits, idx, ref = golden
    sel = np.concatenate([bits[0:64], bits[320:384]])
    out = sim.amplitudes(sel, precision="fp32", prefix_cols=3, prefix_group=64, max_lanes=16)
    pos = [0, 21, 42, 63, 64, 85, 106, 127]
    err = float(np.linalg.norm(out[pos] - ref) / np.linalg.norm(ref))
    print(f"6x6 d32 fp32 batched: normwise rel.err {err:.3e} on 8 oracle bitstrings")
    assert err < TOL


def test_fp32_path_in_the_bench_configuration(golden, sim):
    # the comparator form exactly as bench.py times it: group 0 (64 bitstrings)
    # by the square partition, prefix reuse, 16 lanes; it holds golden indices
    # 0, 21, 42 and 63
    circ, bits, idx, ref = golden
    out = sim.amplitudes(bits[:64], precision="fp32", prefix_cols=3, prefix_group=64,
                         max_lanes=16, scheme="quadrants")
    pos = [k for k, i in enumerate(idx) if i < 64]
    assert [idx[k] for k in pos] == [0, 21, 42, 63]
    err = float(np.linalg.norm(out[[idx[k] for k in pos]] - ref[pos]) / np.linalg.norm(ref[pos]))
    print(f"6x6 d32 fp32 square partition, group 0: normwise rel.err {err:.3e}")
    assert err < TOL


# ---------------------------------------------------------------------------
# 7x7 lattice
# ---------------------------------------------------------------------------

def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def sim7_d24(cuda_device):
    from paper_1905_08394_gb300 import Simulator
    from rqc_inputs import make_circuit

    s = Simulator(7, 7)
    s.apply_circuit(make_circuit(7, 7, 24, 5))
    yield s
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_7x7_d24_amplitudes(sim7_d24, prec):
    g = _golden("oracle_7x7_d24.json")
    bits = np.array(g["bitstrings"], dtype=np.uint64)
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])
    out = sim7_d24.amplitudes(bits, precision=prec)
    err = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    print(f"7x7 d24 {prec}: normwise rel.err {err:.3e}")
    assert err < TOL


def test_7x7_d24_slices_sum_to_the_amplitude(sim7_d24):
    from paper_1905_08394_gb300 import slicing
    from rqc_inputs import make_circuit

    g = _golden("oracle_7x7_d24.json")
    bits = np.array(g["bitstrings"], dtype=np.uint64)
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])
    ss = slicing.choose(make_circuit(7, 7, 24, 5), 2 ** 23, seed=5)
    assert 2 <= len(ss.sliced_cz) <= 10
    tot = sim7_d24.amplitudes(bits, precision="fp16x3", sliced_cz=ss.sliced_cz)
    err = float(np.linalg.norm(tot - ref) / np.linalg.norm(ref))
    print(f"7x7 d24 sum of {ss.n_slices} slices: normwise rel.err {err:.3e}")
    assert err < TOL


def test_7x7_d40_subslices(cuda_device):
    """The 7x7 (1+40+1) circuit with 84 CZ bits held (sub-slices; every
    running tensor of the column sweep at most 2^26 entries), at values that
    do not vanish (see the generating script): four sub-slices of magnitude
    ~1e-20 against the oracle, normwise.  Column sweep only: these held bits
    lie on horizontal edges, which leave the square partition's quarters
    near full size (836 GiB)."""
    from paper_1905_08394_gb300 import Simulator

    g = _golden("oracle_7x7_d40.json")
    circ, bits = workload("7x7_d40")
    assert int(bits[0]) == g["bitstring"]
    ref = np.array([complex(*sub["amplitude"]) for sub in g["subslices"]])
    assert len(ref) == 4 and np.abs(ref).min() > 1e-22
    s = Simulator(7, 7)
    s.apply_circuit(circ)
    for scheme in ("columns",):
        for prec in ("fp32", "fp16x3"):
            out = np.array([s.amplitudes(bits[:1], precision=prec, scheme=scheme,
                                         fixed_cz=g["fixed_cz"], fixed_s=sub["fixed_s"])[0]
                            for sub in g["subslices"]])
            err = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
            print(f"7x7 d40 sub-slices {scheme} {prec}: normwise rel.err {err:.3e}")
            assert err < TOL, (scheme, prec)
    s.close()


def test_8x8_d25_square_partition(cuda_device):
    """The paper's workstation experiment: 8x8 (1+25+1).  Amplitudes of 8
    bitstrings against the oracle's square partition (FP64), and the
    Porter-Thomas statistics of 2048 amplitudes."""
    from paper_1905_08394_gb300 import Simulator

    with open(os.path.join(HERE, "golden", "oracle_8x8_d25.json")) as f:
        g = json.load(f)
    circ, bits = workload("8x8_d25")
    assert [int(b) for b in bits[:8]] == g["bitstrings"]
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])
    sim = Simulator(8, 8)
    sim.apply_circuit(circ)
    for prec in ("fp16x3", "fp32"):
        out = sim.amplitudes(bits[:8], precision=prec, scheme="quadrants")
        err = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
        print(f"8x8 d25 {prec}: normwise rel.err {err:.3e} on 8 oracle bitstrings")
        assert err < TOL
    out = sim.amplitudes(bits[:2048], precision="fp16x3", scheme="quadrants")
    pt = np.sort((2.0 ** 64) * np.abs(out) ** 2)
    assert abs(pt.mean() - 1) < 3 / math.sqrt(len(pt))
    assert abs(np.mean(pt ** 2) - 2) < 0.5
    cdf = 1 - np.exp(-pt)
    D = max(np.max(np.arange(1, len(pt) + 1) / len(pt) - cdf), np.max(cdf - np.arange(len(pt)) / len(pt)))
    assert D < 1.63 / math.sqrt(len(pt))
    sim.close()
