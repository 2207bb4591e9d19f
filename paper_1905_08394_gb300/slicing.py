"""Choice of the sliced CZ set (the "cut" technique the paper names as future
work: one large contraction becomes a sum of smaller ones over fixed indices).

Fixing the Schmidt bit s of a CZ fixes one bit of its edge's bond index on
both sites, halving that bond for the whole sweep.  For the left-to-right
column sweep the running tensor before/after site (r, c) holds one horizontal
bond per row (the boundary between columns c-1|c for rows below r, c|c+1 for
rows up to r) plus one vertical bond, so a memory budget is met by cutting
horizontal bonds.  The chooser below is greedy: while some step's running
tensor exceeds the budget, it cuts one more bit of the widest horizontal bond
of the largest running tensor (ties broken by a seeded draw), choosing which
CZ of that edge to slice by a seeded draw as well.  Host-side planning only.
"""
from __future__ import annotations

from dataclasses import dataclass

from rqc_inputs import SplitMix64


@dataclass
class SliceSet:
    sliced_cz: list        # CZ ordinals (order of application)
    max_entries: int       # largest running tensor with these cuts
    n_slices: int          # 2 ** len(sliced_cz)
    step_cmacs: list       # complex multiply-adds per step of one slice


def cz_edges(circ):
    """For every CZ ordinal: ('h'|'v', r, c) of its edge, and per edge the
    ordinals applied to it (in order)."""
    C = circ.C
    edges, per_edge = [], {}
    for g in circ.gates:
        if g.kind != "cz":
            continue
        a, b = g.qubits
        r, c = divmod(a, C)
        key = ("h", r, c) if b == a + 1 and (b // C) == r else ("v", r, c)
        per_edge.setdefault(key, []).append(len(edges))
        edges.append(key)
    return edges, per_edge


def sweep_sizes(R: int, C: int, hdim, vdim):
    """Running-tensor entries after each absorption and the complex
    multiply-adds of each absorption of the column sweep, for bond dims
    hdim[(r, c)] (edge (r,c)-(r,c+1)) and vdim[(r, c)] (edge (r,c)-(r+1,c))."""
    h = lambda r, c: hdim.get((r, c), 1) if 0 <= c < C - 1 else 1
    v = lambda r, c: vdim.get((r, c), 1) if 0 <= r < R - 1 else 1
    sizes, cmacs = [], []
    for c in range(C):
        for r in range(R):
            M = 1
            for rr in range(R):
                if rr < r:
                    M *= h(rr, c)
                elif rr > r:
                    M *= h(rr, c - 1)
            K = h(r, c - 1) * v(r - 1, c)
            N = h(r, c) * v(r, c)
            cmacs.append(M * K * N)
            sizes.append((M * max(K, N), c, r))
    return sizes, cmacs


def choose(circ, max_entries: int, seed: int = 0, base=None) -> SliceSet:
    """Greedy cut set with every running tensor <= max_entries.  `base`
    (optional) lists CZ ordinals already sliced (they stay sliced)."""
    R, C = circ.R, circ.C
    edges, per_edge = cz_edges(circ)
    rng = SplitMix64(seed ^ 0x511CE)
    sliced = list(base or [])
    taken = set(sliced)

    def dims():
        hd, vd = {}, {}
        for key, ords in per_edge.items():
            free = sum(1 for o in ords if o not in taken)
            (hd if key[0] == "h" else vd)[key[1:]] = 2 ** free
        return hd, vd

    while True:
        hd, vd = dims()
        sizes, cmacs = sweep_sizes(R, C, hd, vd)
        worst = max(s[0] for s in sizes)
        if worst <= max_entries:
            return SliceSet(sorted(sliced), worst, 2 ** len(sliced), cmacs)
        # the largest running tensor (first in sweep order on ties)
        _, c, r = max(sizes, key=lambda s: s[0])
        # its horizontal legs: rows <= r on boundary c|c+1, rows > r on c-1|c
        cand = []
        for rr in range(R):
            cc = c if rr <= r else c - 1
            if 0 <= cc < C - 1 and hd.get((rr, cc), 1) > 1:
                cand.append((hd[(rr, cc)], rr, cc))
        if not cand:
            raise ValueError("budget cannot be met by cutting horizontal bonds")
        widest = max(w for w, _, _ in cand)
        ties = [(rr, cc) for w, rr, cc in cand if w == widest]
        rr, cc = ties[rng.next() % len(ties)]
        free = [o for o in per_edge[("h", rr, cc)] if o not in taken]
        o = free[rng.next() % len(free)]
        sliced.append(o)
        taken.add(o)


def seeded_slice_ids(n_sliced: int, count: int, seed: int):
    """`count` distinct slice ids drawn uniformly from [0, 2^n_sliced)."""
    rng = SplitMix64(seed ^ 0x1D5)
    mask = (1 << n_sliced) - 1
    out = []
    while len(out) < count:
        x = rng.next() & mask
        if x not in out:
            out.append(x)
    return out
