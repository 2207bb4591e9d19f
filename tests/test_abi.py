"""The C-ABI library: it loads, exports every function include/peps_gb300.h
declares, and its host-side logic (argument checks, bond dimensions, plan
sizes) is right.  No GPU needed: nothing here launches a kernel."""
import re
from pathlib import Path

import numpy as np
import pytest

from paper_1905_08394_gb300 import binding as B
from paper_1905_08394_gb300 import complexity as cx
from rqc_inputs import make_circuit, workload

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    txt = (ROOT / "include" / "peps_gb300.h").read_text()
    return sorted(set(re.findall(r"PEPS_API\s+[\w\s\*]*?\b(peps_\w+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    lib = B.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.EXPORTED)
    assert "sm_103a" in B.peps_version()


def test_peak_microbenchmark_library_loads():
    # measurement only (bench.py --case peaks); kept out of the amplitude library
    import ctypes

    lib = ctypes.CDLL(str(ROOT / "paper_1905_08394_gb300" / "libpeps_peaks.so"))
    assert hasattr(lib, "peaks_fma_tflops") and hasattr(lib, "peaks_mma_tflops")
    assert not hasattr(B.load(), "peaks_fma_tflops")


def make(R, C, d, seed):
    c = make_circuit(R, C, d, seed)
    h = B.peps_create(R, C)
    for g in c.gates:
        if g.kind == "1q":
            q = g.qubits[0]
            B.peps_apply_1q(h, q // C, q % C, g.U)
        else:
            a, b = g.qubits
            B.peps_apply_cz(h, a // C, a % C, b // C, b % C)
    return c, h


def test_argument_checks():
    with pytest.raises(B.PepsError) as e:
        B.peps_create(0, 3)
    assert e.value.code == B.PEPS_EINVAL
    with pytest.raises(B.PepsError):
        B.peps_create(9, 8)  # 72 qubits > 64
    h = B.peps_create(3, 3)
    with pytest.raises(B.PepsError) as e:
        B.peps_apply_cz(h, 0, 0, 1, 1)
    assert e.value.code == B.PEPS_ENOTADJ
    with pytest.raises(B.PepsError) as e:
        B.peps_apply_1q(h, 3, 0, np.eye(2))
    assert e.value.code == B.PEPS_EINVAL
    with pytest.raises(B.PepsError):
        B.peps_apply_1q(h, 0, 0, np.array([[np.nan, 0], [0, 1]]))
    o, k = B.make_opts(prefix_cols=3)
    with pytest.raises(B.PepsError):
        B.peps_workspace_bytes(h, 8, o)   # prefix_cols must be < C
    o, k = B.make_opts(prefix_cols=1, prefix_group=3)
    with pytest.raises(B.PepsError):
        B.peps_workspace_bytes(h, 8, o)   # n not a multiple of the group
    o, k = B.make_opts(sliced_cz=[0])
    with pytest.raises(B.PepsError):
        B.peps_workspace_bytes(h, 8, o)   # no CZ yet
    B.peps_destroy(h)


@pytest.mark.parametrize("R,C,d", [(4, 4, 8), (5, 5, 16), (6, 6, 32), (7, 7, 40), (3, 5, 13),
                                   (6, 1, 10), (1, 6, 10)])
def test_bond_dims_follow_cz_counts(R, C, d):
    c, h = make(R, C, d, 1)
    for r in range(R):
        for col in range(C):
            q = r * C + col
            if col + 1 < C:
                assert B.peps_bond_dim(h, r, col, r, col + 1) == 2 ** c.cz_count(q, q + 1)
                assert B.peps_bond_dim(h, r, col + 1, r, col) == 2 ** c.cz_count(q, q + 1)
            if r + 1 < R:
                assert B.peps_bond_dim(h, r, col, r + 1, col) == 2 ** c.cz_count(q, q + C)
    assert B.peps_cz_count(h) == sum(1 for g in c.gates if g.kind == "cz")
    B.peps_destroy(h)


def test_plan_counts_match_cost_model():
    c, h = make(6, 6, 32, 4)
    o, k = B.make_opts(precision="fp32", fuse_rows=1)
    info = B.peps_plan_info_get(h, 1, o)
    assert info["n_steps"] == 36
    assert info["max_entries"] == 16 ** 7
    assert info["flops_per_chain"] == 8 * cx.column_sweep_cmacs(6, 6, 16)
    # prefix reuse: 8 groups x 64, first 3 columns shared
    o, k = B.make_opts(precision="fp32", prefix_cols=3, prefix_group=64, fuse_rows=1)
    info = B.peps_plan_info_get(h, 512, o)
    steps = cx.column_sweep_step_cmacs(6, 6, 16)
    # the first 3 columns are contracted once per group, the rest per bitstring
    assert info["flops_call"] == 8 * (8 * sum(steps[:18]) + 512 * sum(steps[18:]))
    assert info["n_launches"] == 8 * 18 + 8 * 4 * 18   # 16 lanes per launch
    B.peps_destroy(h)


def test_fused_boundary_rows_plan():
    # the two top and the two bottom rows of each column in one step each
    c, h = make(6, 6, 32, 4)
    o1, k1 = B.make_opts(precision="fp16x3", fuse_rows=1)
    o0, k0 = B.make_opts(precision="fp16x3")
    single = B.peps_plan_info_get(h, 1, o1)
    fused = B.peps_plan_info_get(h, 1, o0)
    blocks = cx.column_sweep_block_cmacs(6, 6, 16)
    # the last column's bottom pair would be one long dot product: kept single
    assert [k for _, k, _ in blocks] == [2, 1, 1, 2] * 5 + [2, 1, 1, 1, 1]
    assert single["n_steps"] == 36 and fused["n_steps"] == len(blocks) == 25
    assert fused["max_entries"] == single["max_entries"]
    assert fused["flops_per_chain"] == 8 * sum(m for _, _, m in blocks)
    assert fused["flops_per_chain"] < single["flops_per_chain"]
    # the running tensor between the two rows of a pair is never written
    assert fused["bytes_per_chain"] < 0.65 * single["bytes_per_chain"]
    B.peps_destroy(h)


def test_fusion_needs_four_rows():
    for R, C in ((2, 5), (3, 4)):
        c, h = make(R, C, 10, 3)
        o, k = B.make_opts(precision="fp32")
        info = B.peps_plan_info_get(h, 1, o)
        assert info["n_steps"] == R * C
        B.peps_destroy(h)


def _bond_dims(h, R, C):
    dims = {}
    for r in range(R):
        for c in range(C):
            q = r * C + c
            if c + 1 < C:
                dims[(q, q + 1)] = B.peps_bond_dim(h, r, c, r, c + 1)
            if r + 1 < R:
                dims[(q, q + C)] = B.peps_bond_dim(h, r, c, r + 1, c)
    return dims


@pytest.mark.parametrize("R,C,d,seed", [(6, 6, 32, 4), (4, 4, 8, 1), (6, 6, 16, 3)])
def test_quadrant_plan_matches_the_oracle_count(R, C, d, seed):
    # square partition: 4 quarter sweeps + 2 merges; on a square lattice with one
    # bond dimension the multiply-adds equal the oracle's direct count (quarters
    # + merges) less the last contraction, which the GPU does as a dot product.
    # (The GPU merges F_ul with F_bl first and the oracle F_ul with F_ur, which
    # cost the same only when the quarters are square.)
    from oracle import peps as op
    c, h = make(R, C, d, seed)
    o, k = B.make_opts(precision="fp16x3", scheme="quadrants", fuse_rows=1)
    info = B.peps_plan_info_get(h, 1, o)
    assert info["n_steps"] == 4 * (R // 2) * (C // 2) + 2
    cost = op.quadrant_contraction_cmacs(R, C, _bond_dims(h, R, C))
    last = 1
    for (a, b), v in _bond_dims(h, R, C).items():
        ra, ca = divmod(a, C)
        rb, cb = divmod(b, C)
        if (ra < R // 2) != (rb < R // 2):
            last *= v            # the edges cut by the middle row boundary
    assert info["flops_per_chain"] == 8 * (cost["quarters"] + cost["merges"] - last)
    assert info["max_entries"] == cost["largest"]
    B.peps_destroy(h)


@pytest.mark.parametrize("L,d,seed", [(3, 8, 1), (5, 16, 2), (5, 12, 7), (7, 24, 5)])
def test_odd_quadrant_plan_matches_the_oracle_count(L, d, seed):
    # odd side (Fig. S2(c)): the planner merges in the paper's order (ul with
    # ur, bl with br), so with single-site steps its multiply-adds equal the
    # oracle's direct count less the last contraction (the dot over the
    # horizontal cut), and the largest tensors agree
    from oracle import peps as op
    c, h = make(L, L, d, seed)
    o, k = B.make_opts(precision="fp16x3", scheme="quadrants", fuse_rows=1)
    info = B.peps_plan_info_get(h, 1, o)
    dims = _bond_dims(h, L, L)
    cost = op.quadrant_contraction_cmacs(L, L, dims)
    m = L // 2
    cut = 1
    for (a, b), v in dims.items():
        if (a // L <= m) != (b // L <= m):
            cut *= v
    assert info["flops_per_chain"] == 8 * (cost["quarters"] + cost["merges"] - cut)
    assert info["max_entries"] == cost["largest"]
    B.peps_destroy(h)


def test_quadrant_sweeps_fuse_their_top_row_pairs():
    # in each sweep column of a 3 x 3 quarter the top two rows go in one step
    # (no incoming vertical leg): 6 steps per quarter instead of 9, the same
    # largest tensor, fewer multiply-adds and about 40 % fewer bytes
    c, h = make(6, 6, 32, 4)
    single = B.peps_plan_info_get(h, 1, B.make_opts(precision="fp16x3", scheme="quadrants",
                                                   fuse_rows=1)[0])
    fused = B.peps_plan_info_get(h, 1, B.make_opts(precision="fp16x3", scheme="quadrants")[0])
    assert single["n_steps"] == 38 and fused["n_steps"] == 26
    assert fused["max_entries"] == single["max_entries"] == 2 ** 24
    assert fused["flops_per_chain"] <= single["flops_per_chain"]
    assert fused["bytes_per_chain"] < 0.75 * single["bytes_per_chain"]
    B.peps_destroy(h)


def test_quadrant_plan_6x6_d32_sizes_and_prefix_reuse():
    c, h = make(6, 6, 32, 4)
    o, k = B.make_opts(precision="fp16x3", scheme="quadrants", prefix_cols=3, prefix_group=64,
                       max_lanes=16)
    q = B.peps_plan_info_get(h, 512, o)
    o2, k2 = B.make_opts(precision="fp16x3", prefix_cols=3, prefix_group=64, max_lanes=16)
    col = B.peps_plan_info_get(h, 512, o2)
    assert q["max_entries"] == 2 ** 24 and col["max_entries"] == 2 ** 28
    # per group: ul, bl, F_l; per bitstring: ur, br, Y = 2^36 multiply-adds
    assert q["flops_call"] < col["flops_call"] / 6
    assert q["flops_call"] > 512 * 8 * 2 ** 36
    B.peps_destroy(h)


def test_quadrant_plan_rejects_bad_requests():
    c, h = make(5, 6, 16, 2)
    o, k = B.make_opts(precision="fp32", scheme="quadrants")
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 1, o)          # odd side
    B.peps_destroy(h)
    c, h = make(4, 6, 16, 2)                   # even rectangles are fine
    o1, k1 = B.make_opts(precision="fp32", scheme="quadrants", fuse_rows=1)
    info = B.peps_plan_info_get(h, 1, o1)
    assert info["n_steps"] == 4 * 2 * 3 + 2
    B.peps_destroy(h)
    c, h = make(6, 6, 16, 2)
    o, k = B.make_opts(precision="fp32", scheme="quadrants", prefix_cols=2, prefix_group=4)
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 8, o)          # prefix must be the left half
    o, k = B.make_opts(precision="fp32", scheme=7)
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 1, o)
    B.peps_destroy(h)


def test_general_two_qubit_gates_grow_the_bond_by_their_rank():
    from rqc_inputs import two_qubit_test_gates
    iswap, cnot, rank3, rnd = two_qubit_test_gates(1)
    h = B.peps_create(2, 3)
    B.peps_apply_2q(h, 0, 0, 0, 1, iswap)
    assert B.peps_bond_dim(h, 0, 0, 0, 1) == 4
    B.peps_apply_2q(h, 0, 1, 0, 0, cnot)          # either qubit order
    assert B.peps_bond_dim(h, 0, 0, 0, 1) == 8
    B.peps_apply_2q(h, 0, 1, 1, 1, rank3)
    assert B.peps_bond_dim(h, 0, 1, 1, 1) == 3
    B.peps_apply_cz(h, 0, 1, 1, 1)
    assert B.peps_bond_dim(h, 0, 1, 1, 1) == 6
    B.peps_apply_2q(h, 1, 1, 1, 2, np.diag([1, 1, 1, -1.0]))   # CZ as a general gate
    assert B.peps_bond_dim(h, 1, 1, 1, 2) == 2
    with pytest.raises(B.PepsError):
        B.peps_apply_2q(h, 0, 0, 1, 1, rnd)       # not neighbours
    with pytest.raises(B.PepsError):
        B.peps_apply_2q(h, 0, 0, 0, 1, np.zeros((4, 4)))
    # a CZ on an edge with a general gate cannot be sliced
    o, k = B.make_opts(precision="fp32", sliced_cz=[0])
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 1, o)
    B.peps_destroy(h)


def test_slicing_plan():
    c, h = make(5, 5, 16, 2)
    ncz = B.peps_cz_count(h)
    o, k = B.make_opts(precision="fp32", sliced_cz=[0, 1, 2])
    info = B.peps_plan_info_get(h, 4, o)
    assert info["n_slices"] == 8
    o2, k2 = B.make_opts(precision="fp32")
    full = B.peps_plan_info_get(h, 4, o2)
    assert info["max_entries"] <= full["max_entries"]
    o, k = B.make_opts(precision="fp32", sliced_cz=[0, 0])
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 4, o)
    o, k = B.make_opts(precision="fp32", sliced_cz=[ncz])
    with pytest.raises(B.PepsError):
        B.peps_plan_info_get(h, 4, o)
    B.peps_destroy(h)


def test_seven_by_seven_needs_slicing():
    c, h = make(7, 7, 40, 5)
    o, k = B.make_opts(precision="fp32")
    with pytest.raises(B.PepsError) as e:
        B.peps_workspace_bytes(h, 1, o)
    assert e.value.code == B.PEPS_EUNSUPPORTED
    B.peps_destroy(h)


def test_small_lattices_plan_one_contraction_launch():
    # every running tensor and operand of a 5x5 (1+16+1) sweep fits one
    # block's shared memory: one contraction launch for all bitstrings (FP32
    # and the split forms), and a smaller workspace (no running-tensor
    # buffers); STEPWISE, a single-pass form or a larger lattice plan one
    # launch per step and lane chunk
    c, h = make(5, 5, 16, 2)
    o, k = B.make_opts(precision="fp32")
    small = B.peps_plan_info_get(h, 1024, o)
    assert small["n_launches"] == 1 and small["n_tc_launches"] == 0
    ws_small = B.peps_workspace_bytes(h, 1024, o)
    o, k = B.make_opts(precision="fp32", flags=B.PEPS_FLAG_STEPWISE)
    step = B.peps_plan_info_get(h, 1024, o)
    assert step["n_launches"] == step["n_steps"] * (1024 // 16)
    assert step["flops_call"] == small["flops_call"]
    assert B.peps_workspace_bytes(h, 1024, o) > ws_small
    o, k = B.make_opts(precision="fp16x3")
    assert B.peps_plan_info_get(h, 1024, o)["n_launches"] == 1
    o, k = B.make_opts(precision="bf16")
    assert B.peps_plan_info_get(h, 1024, o)["n_launches"] > 1
    B.peps_destroy(h)
    c, h = make(6, 6, 24, 3)
    o, k = B.make_opts(precision="fp32")
    assert B.peps_plan_info_get(h, 64, o)["n_launches"] > 1
    B.peps_destroy(h)


def test_plan_steps_report_a_consistent_output_layout():
    # every step's stored output: N = dh dv, M = batch x Mr, Mr = P x (rows
    # kept in place); the 6x6 (1+32+1) square partition with held and linked
    # bits, both contraction orders
    c, h = make(6, 6, 32, 4)
    for scheme in ("quadrants", "columns"):
        o, k = B.make_opts(precision="fp16x3", scheme=scheme, prefix_cols=3, prefix_group=64,
                           max_lanes=64, hold_ties=True)
        steps = B.peps_plan_steps(h, 512, o)
        assert steps
        for s in steps:
            assert s["dh"] * s["dv"] == s["N"], s
            assert s["M"] % s["Mr"] == 0 and s["Mr"] % s["P"] == 0, s
            assert s["open_leg"] in (0, 1) and s["fused_dot"] in (0, 1)
        # on the tensor cores the last merge forms the dot product in its epilogue
        assert [s["fused_dot"] for s in steps] == [0] * (len(steps) - 1) + [int(scheme == "quadrants")]
    B.peps_destroy(h)


def test_tensor_core_tuning_knobs_are_validated():
    # K bytes per stage 0/64/128, CTA pairing 0/1/2, epilogue warps 0/4/8;
    # anything else is refused before any device work
    c, h = make(4, 4, 8, 1)
    for kw in ({"tc_kchunk": 64}, {"tc_cluster": 1}, {"tc_epi": 4}, {"tc_epi": 8}, {"tc_epi": 0}):
        o, k = B.make_opts(precision="fp16x3", **kw)
        B.peps_plan_info_get(h, 16, o)
    for kw in ({"tc_kchunk": 32}, {"tc_cluster": 3}, {"tc_epi": 6}, {"tc_epi": -1}):
        o, k = B.make_opts(precision="fp16x3", **kw)
        with pytest.raises(B.PepsError) as e:
            B.peps_plan_info_get(h, 16, o)
        assert "tc_epi" in str(e.value)
    B.peps_destroy(h)


def test_square_partition_merges_share_launches():
    # 6x6 (1+32+1), 8 groups of 64: the groups' left halves (and their merge
    # F_l) in one launch per step, and one launch of the last merge per chunk
    # of member lanes, whatever groups the chunk spans
    c, h = make(6, 6, 32, 4)
    for lanes, chunks in ((512, 1), (64, 8), (16, 32)):
        o, k = B.make_opts(precision="fp16x3", scheme="quadrants", prefix_cols=3,
                           prefix_group=64, max_lanes=lanes, hold_ties=True)
        steps = B.peps_plan_steps(h, 512, o)
        merges = [s for s in steps if s["part"] == 4]
        assert len(merges) == 2
        assert merges[0]["launches"] == 1            # F_l of all 8 groups
        assert merges[1]["launches"] == chunks       # Y = F_br F_l^T and the dot
        left = [s for s in steps if s["part"] in (0, 1) and s["sites"] > 0]
        assert all(s["launches"] == 1 for s in left)
    B.peps_destroy(h)
