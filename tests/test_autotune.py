"""Host-side logic of the autotuner: the candidate grid and the workload
signature that keys its cache (no GPU needed)."""
import json

from paper_1905_08394_gb300 import autotune


class FakeSim:
    R, C = 2, 2

    def bond_dim(self, *a):
        return 4


def test_candidates_span_the_grid():
    c = list(autotune.candidates(lanes=(8, 16), kchunk=(128,), cluster=(1, 2),
                                 schemes=("columns", "quadrants")))
    assert len(c) == 2 * 2 * 1 * 2
    assert {x["scheme"] for x in c} == {"columns", "quadrants"}
    assert all(set(x) == {"scheme", "max_lanes", "tc_kchunk", "tc_cluster", "tc_epi"} for x in c)
    assert {x["tc_epi"] for x in c} == {0}
    e = list(autotune.candidates(lanes=(8,), kchunk=(128,), cluster=(2,), epi=(0, 4, 8)))
    assert [x["tc_epi"] for x in e] == [0, 4, 8]


def test_signature_depends_on_the_workload_and_order():
    s = FakeSim()
    a = autotune.signature(s, 64, {"precision": "fp16x3", "scheme": "columns"})
    b = autotune.signature(s, 64, {"precision": "fp16x3", "scheme": "quadrants"})
    c = autotune.signature(s, 128, {"precision": "fp16x3", "scheme": "columns"})
    assert len({a, b, c}) == 3
    assert json.loads(a)["dims"] == [4, 4, 4, 4]
