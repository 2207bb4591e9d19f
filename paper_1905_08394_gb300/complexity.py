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
