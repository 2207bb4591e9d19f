"""Cost model of the contraction against the numbers the paper prints (P7)
and against the oracle's direct count of the column sweep."""
from oracle import peps as op
from paper_1905_08394_gb300 import complexity as cx

TiB = 2 ** 40
PiB = 2 ** 50


def test_paper_memory_figures():
    # main text: 8x8 at (1+40+1) needs 32 TB (even-square partition)
    assert cx.bytes_c128(cx.space_square_even(8, 40)) == 32 * TiB
    # 10x10 at (1+32+1) has the same space complexity as 8x8 at (1+40+1)
    assert cx.space_square_even(10, 32) == cx.space_square_even(8, 40)
    # 8 x l (l > 8) at (1+40+1): about 0.5 PB (generic scheme, L = 8)
    assert cx.bytes_c128(cx.space_generic(20, 8, 40)) == PiB // 2
    # 9x9 at (1+40+1): 16 PB (odd-square partition; 2^50 + 2^45 entries)
    b = cx.bytes_c128(cx.space_square_odd(9, 40))
    assert b == 16 * (2 ** 50 + 2 ** 45) and 16 * PiB <= b < 17 * PiB
    # 12x12 at (1+32+1): 8 PB
    assert cx.bytes_c128(cx.space_square_even(12, 32)) == 8 * PiB
    # Bristlecone-72 at (1+32+1): 2^45 entries, "less than 0.6 PB"
    assert cx.space_bristlecone(32) == 2 ** 45
    assert cx.bytes_c128(cx.space_bristlecone(32)) < 0.6 * 1e15 * 1.13  # 0.5 PiB
    # 7x7 at (1+40+1): theoretical 16 TB
    assert cx.bytes_c128(cx.space_generic(7, 7, 40)) == 16 * TiB


def test_chi_bound():
    assert [cx.chi_exp(d) for d in (8, 16, 24, 32, 40, 25, 39)] == [1, 2, 3, 4, 5, 4, 5]


def test_time_equations():
    assert cx.time_generic(6, 6, 32) == 16 * 2 ** 36
    assert cx.time_square_even(6, 32) == 2 ** 37
    assert cx.time_square_odd(7, 40) == 33 * 2 ** 50


def test_column_sweep_count_matches_oracle_and_time_equation():
    for (R, C, chi) in [(4, 4, 2), (5, 5, 4), (6, 6, 8), (6, 6, 16), (7, 7, 32), (3, 5, 4)]:
        dims = {}
        for r in range(R):
            for col in range(C):
                q = r * C + col
                if col + 1 < C:
                    dims[(q, q + 1)] = chi
                if r + 1 < R:
                    dims[(q, q + C)] = chi
        assert op.column_contraction_cmacs(R, C, dims) == cx.column_sweep_cmacs(R, C, chi)
    full = cx.column_sweep_cmacs(6, 6, 16)
    assert full == 1134980891136
    assert 1.03 < full / cx.time_generic(6, 6, 32) < 1.035
