"""Cost model of the exact contraction: the paper's space/time formulas and a
direct count of the column sweep.  Host-side planning logic.

Units (the paper states none): "space" counts tensor entries and "time"
counts complex multiply-adds of the dominant steps; a byte figure is entries
x 16 (complex128, the paper runs in double precision).
"""
from __future__ import annotations

import math


def chi_exp(d: int) -> int:
    """ceil(d/8): log2 of the bond-dimension bound (main-text "chi" equation)."""
    return -(-d // 8)


def space_generic(Lv: int, Lh: int, d: int) -> int:
    """Largest tensor of the generic row/column scheme: 2^(ceil(d/8)(L+1)),
    L = min(Lh, Lv) (main-text "space" equation and its supplementary
    restatement)."""
    return 2 ** (chi_exp(d) * (min(Lh, Lv) + 1))


def time_generic(Lv: int, Lh: int, d: int) -> int:
    """(Lh-2)(Lv-2) 2^(ceil(d/8)(L+3)) (main-text "time" equation)."""
    L = min(Lh, Lv)
    return (Lh - 2) * (Lv - 2) * 2 ** (chi_exp(d) * (L + 3))


def space_square_even(L: int, d: int) -> int:
    """2^(ceil(d/8) sqrt(N) + 1), sqrt(N) = L even (supplementary
    "spacesquareeven")."""
    return 2 ** (chi_exp(d) * L + 1)


def time_square_even(L: int, d: int) -> int:
    """2^(3 ceil(d/8) sqrt(N)/2 + 1) (supplementary "timesquareeven")."""
    return 2 ** (3 * chi_exp(d) * L // 2 + 1)


def space_square_odd(L: int, d: int) -> int:
    """2^(ceil(d/8)(sqrt(N)+1)) + 2^(ceil(d/8) sqrt(N)) (supplementary
    "spacesquareodd")."""
    k = chi_exp(d)
    return 2 ** (k * (L + 1)) + 2 ** (k * L)


def time_square_odd(L: int, d: int) -> int:
    """(2^ceil(d/8) + 1) 2^(ceil(d/8)(3 sqrt(N) - 1)/2) (supplementary
    "timesquareodd")."""
    k = chi_exp(d)
    return (2 ** k + 1) * 2 ** (k * (3 * L - 1) // 2)


def space_bristlecone(d: int, max_legs: int = 11) -> int:
    """Bristlecone-72 partition: tensors of at most 11 legs, two of them kept:
    2^(ceil(d/8) * 11 + 1) (supplementary Bristlecone section)."""
    return 2 ** (chi_exp(d) * max_legs + 1)


def bytes_c128(entries: int) -> int:
    return 16 * entries


def column_sweep_step_cmacs(R: int, C: int, chi: int) -> list:
    """Complex multiply-adds of every site absorption of the column sweep
    (in sweep order) with every bond of dimension chi: step (r, c) costs
    M*K*N with M the product of the untouched horizontal legs,
    K = dim(h_r) dim(v), N = dim(h'_r) dim(v')."""
    out = []
    for c in range(C):
        left = 1 if c == 0 else chi
        right = 1 if c == C - 1 else chi
        for r in range(R):
            up = 1 if r == 0 else chi
            down = 1 if r == R - 1 else chi
            # untouched legs: rows < r already carry h' (right dims), rows > r carry h (left)
            M = right ** r * left ** (R - 1 - r)
            out.append(M * (left * up) * (right * down))
    return out


def column_sweep_block_cmacs(R: int, C: int, chi: int, fuse: bool = True) -> list:
    """Like column_sweep_step_cmacs, but with the two top rows and the two
    bottom rows of a column absorbed in one step each (when R >= 4, the
    pair costs no more than its two single steps, and it has at least 152
    output tiles of 128 x 64 or a K no longer than the two singles' K).  A block of rows
    r0 .. r0+k-1 costs M*K*N with M the product of the untouched horizontal
    legs (rows above the block carry h', rows below carry h), K the product of
    the block's incoming horizontal legs times the vertical leg above it, N the
    product of its outgoing horizontal legs times the vertical leg below it.
    Returns [(r0, k, cmacs)] in sweep order."""
    out = []
    for c in range(C):
        left = 1 if c == 0 else chi
        right = 1 if c == C - 1 else chi
        vdim = lambda r: chi if 0 <= r < R - 1 else 1   # leg between rows r, r+1
        def mkn(r0, k):
            M = right ** r0 * left ** (R - r0 - k)
            return M, left ** k * vdim(r0 - 1), right ** k * vdim(r0 + k - 1)

        def cost(r0, k):
            M, K, N = mkn(r0, k)
            return M * K * N

        def parallel_enough(r0):
            # enough 128 x 64 output tiles, or a K no longer than the singles'
            M, K, N = mkn(r0, 2)
            tiles = -(-M // 128) * -(-N // 64)
            return tiles >= 152 or K <= mkn(r0, 1)[1] + mkn(r0 + 1, 1)[1]

        r = 0
        while r < R:
            k = 1
            if (fuse and R >= 4 and (r == 0 or r == R - 2)
                    and cost(r, 2) <= cost(r, 1) + cost(r + 1, 1) and parallel_enough(r)):
                k = 2
            out.append((r, k, cost(r, k)))
            r += k
    return out


def column_sweep_cmacs(R: int, C: int, chi: int) -> int:
    """Sum of column_sweep_step_cmacs (boundary steps included)."""
    return sum(column_sweep_step_cmacs(R, C, chi))


def fmt_bytes(b: float) -> str:
    for unit, s in (("PiB", 2 ** 50), ("TiB", 2 ** 40), ("GiB", 2 ** 30)):
        if b >= s:
            return f"{b / s:.3g} {unit}"
    return f"{b:.3g} B"


def log2(x: float) -> float:
    return math.log2(x)
