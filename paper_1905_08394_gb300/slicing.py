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

For the square partition (Fig. S2(b, c)) the cost of a slice set is not a
property of one running tensor: a bit cut on a quarter's open leg shrinks its
sweep from the column where that leg appears, and a quarter is recomputed for
every bit it does not touch.  `choose_quadrants` therefore searches on the C
planner's own figures (multiply-adds per slice and workspace bytes): a beam
search that adds one cut bit at a time and keeps the cheapest total
(per-slice flops x 2^|S|) among the sets whose workspace fits the budget.
"""
from __future__ import annotations

from dataclasses import dataclass

from rqc_inputs import SplitMix64


@dataclass
class SliceSet:
    sliced_cz: list        # CZ ordinals (order of application)
    max_entries: int       # largest running tensor with these cuts
    n_slices: int          # 2 ** len(sliced_cz)
    step_cmacs: list       # complex multiply-adds per step of one slice (column sweep)
    flops_per_slice: float = 0.0   # the planner's figure (square partition)
    workspace_bytes: int = 0       # the planner's figure (square partition)


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


def choose_quadrants(h, circ, ws_budget: int, precision: str = "fp16x3", seed: int = 0,
                     beam: int = 16, max_bits: int = 24) -> SliceSet:
    """Slice set for the square partition on the planner of handle `h` (the
    circuit `circ` applied to it): the cheapest total flops found whose
    workspace is at most `ws_budget` bytes.  Each beam level adds one cut bit
    on one edge (which CZ of the edge by a seeded draw); candidates are ranked
    by log2(total flops) + 2 log2(workspace / budget) above the budget."""
    import math

    from . import binding as B

    _, per_edge = cz_edges(circ)
    keys = sorted(per_edge)
    rng = SplitMix64(seed ^ 0x9A4D)
    pick = {k: [per_edge[k][i] for i in _seeded_perm(len(per_edge[k]), rng)] for k in keys}

    def evaluate(counts):
        sl = sorted(o for k, c in counts.items() for o in pick[k][:c])
        kw = dict(precision=precision, scheme="quadrants", sliced_cz=sl, slice_ids=[0] if sl else None,
                  flags=B.PEPS_FLAG_ESTIMATE)
        o, keep = B.make_opts(**kw)
        try:
            info = B.peps_plan_info_get(h, 1, o)
            ws = B.peps_workspace_bytes(h, 1, o)
        except B.PepsError:
            return None
        del keep
        return sl, info, ws

    best = None
    frontier = [{}]
    seen = set()
    for _ in range(max_bits + 1):
        scored = []
        for counts in frontier:
            for k in keys:
                c = counts.get(k, 0)
                if c >= len(per_edge[k]):
                    continue
                nc = dict(counts)
                nc[k] = c + 1
                tag = tuple(sorted(nc.items()))
                if tag in seen:
                    continue
                seen.add(tag)
                r = evaluate(nc)
                if r is None:
                    continue
                sl, info, ws = r
                total = info["flops_per_chain"] * 2.0 ** len(sl)
                if ws <= ws_budget and (best is None or total < best[0]):
                    best = (total, sl, info, ws)
                over = max(0.0, math.log2(ws / ws_budget))
                scored.append((math.log2(total) + 2.0 * over, tag, nc))
        if not scored:
            break
        scored.sort(key=lambda t: (t[0], t[1]))
        frontier = [nc for _, _, nc in scored[:beam]]
    if best is None:
        raise ValueError("no slice set within the budget was found")
    total, sl, info, ws = best
    return SliceSet(sl, int(info["max_entries"]), 2 ** len(sl), [], float(info["flops_per_chain"]),
                    int(ws))


def _seeded_perm(n: int, rng):
    """A seeded permutation of range(n) (Fisher-Yates on SplitMix64 draws)."""
    p = list(range(n))
    for i in range(n - 1, 0, -1):
        j = rng.next() % (i + 1)
        p[i], p[j] = p[j], p[i]
    return p
