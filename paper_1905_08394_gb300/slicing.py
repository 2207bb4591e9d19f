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
search that adds one cut bit at a time and keeps the cheapest total among the
sets whose workspace fits the budget.  The total counts the odd side's lower
half once per value of its own bits (one bitstring: consecutive slices that
share them keep F_b) and, for a given output bitstring, only the slices that
can be nonzero: ties between slice bits (`slice_constraints`, below) make the
others vanish exactly.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from rqc_inputs import SplitMix64


@dataclass
class SliceSet:
    sliced_cz: list        # CZ ordinals (order of application)
    max_entries: int       # largest running tensor with these cuts
    n_slices: int          # 2 ** len(sliced_cz)
    step_cmacs: list       # complex multiply-adds per step of one slice (column sweep)
    flops_per_slice: float = 0.0   # the planner's figure (square partition)
    workspace_bytes: int = 0       # the planner's figure (square partition)
    flops_total: float = 0.0       # every slice, the odd side's lower-half reuse counted
    n_lower_bits: int = 0          # sliced bits the odd side's lower half depends on


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
                     beam: int = 16, max_bits: int = 24, x=None, keep: int = 1):
    """Slice set for the square partition on the planner of handle `h` (the
    circuit `circ` applied to it): the cheapest total flops found whose
    workspace is at most `ws_budget` bytes.  Each beam level adds one cut bit
    on one edge; candidates are ranked by log2(total flops) + 2 log2(workspace
    / budget) above the budget.  Which CZ of an edge is cut next: a seeded
    order, or, for one output bitstring `x`, first the CZs whose bit `x`
    fixes (slice_constraints), so that the cut costs no extra slices; the
    total then counts only the slices that can be nonzero.  With keep > 1 the
    `keep` cheapest sets found are returned (a list, cheapest first), for a
    choice by measured time."""
    import math

    from . import binding as B

    _, per_edge = cz_edges(circ)
    keys = sorted(per_edge)
    rng = SplitMix64(seed ^ 0x9A4D)
    pick = {}
    for k in keys:
        order = [per_edge[k][i] for i in _seeded_perm(len(per_edge[k]), rng)]
        if x is not None:
            fixed = [o for o in order if slice_constraints(circ, [o], x)]
            order = fixed + [o for o in order if o not in fixed]
        pick[k] = order

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
    found = {}
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
                total = call_flops(info, len(sl), circ, sl, x)
                if ws <= ws_budget and (best is None or total < best[0]):
                    best = (total, sl, info, ws)
                if ws <= ws_budget:
                    found[tuple(sl)] = (total, sl, info, ws)
                over = max(0.0, math.log2(ws / ws_budget))
                scored.append((math.log2(total) + 2.0 * over, tag, nc))
        if not scored:
            break
        scored.sort(key=lambda t: (t[0], t[1]))
        frontier = [nc for _, _, nc in scored[:beam]]
    if best is None:
        raise ValueError("no slice set within the budget was found")

    def as_set(entry):
        total, sl, info, ws = entry
        return SliceSet(sl, int(info["max_entries"]), 2 ** len(sl), [],
                        float(info["flops_per_chain"]), int(ws), float(total),
                        int(info["n_lower_bits"]))

    if keep > 1:
        ranked = sorted(found.values(), key=lambda e: (e[0], e[1]))[:keep]
        return [as_set(e) for e in ranked]
    return as_set(best)


def call_flops(info: dict, n_sliced: int, circ=None, sliced_cz=None, x=None) -> float:
    """Flops of the call over all 2^n_sliced slices from a one-slice plan's
    figures: the odd-side lower half runs once per value of its own bits.
    With the circuit, the slice set and a bitstring, only the slices that can
    be nonzero (slice_counts) are counted."""
    fl = float(info.get("flops_lower", 0.0))
    upper = float(info["flops_per_chain"]) - fl
    if circ is not None and x is not None:
        lm = lower_half_mask(circ, sliced_cz) if fl > 0 else (1 << n_sliced) - 1
        n_cons, n_low = slice_counts(circ, sliced_cz, x, lm)
        return upper * n_cons + fl * n_low
    return upper * 2.0 ** n_sliced + fl * 2.0 ** int(info.get("n_lower_bits", n_sliced))


def lower_half_mask(circ, sliced_cz) -> int:
    """Bits of a slice id (bit j = sliced_cz[j]) whose CZ touches the lower
    half of the odd-side square partition (rows R//2+1 ..)."""
    edges, _ = cz_edges(circ)
    m = circ.R // 2
    mask = 0
    for j, o in enumerate(sliced_cz):
        kind, r, _ = edges[o]
        if r > m or (kind == "v" and r + 1 > m):
            mask |= 1 << j
    return mask


def slice_group(n_sliced: int, lower_mask: int, seed: int):
    """All slice ids that share one seeded value of the lower-half bits (the
    run of slices between two lower-half contractions)."""
    rng = SplitMix64(seed ^ 0x6A0)
    base = rng.next() & lower_mask & ((1 << n_sliced) - 1)
    free = [j for j in range(n_sliced) if not (lower_mask >> j) & 1]
    out = []
    for t in range(1 << len(free)):
        x = base
        for i, j in enumerate(free):
            if (t >> i) & 1:
                x |= 1 << j
        out.append(x)
    return out


def _seeded_perm(n: int, rng):
    """A seeded permutation of range(n) (Fisher-Yates on SplitMix64 draws)."""
    p = list(range(n))
    for i in range(n - 1, 0, -1):
        j = rng.next() % (i + 1)
        p[i], p[j] = p[j], p[i]
    return p


# ---------------------------------------------------------------------------
# Slices that vanish exactly.  A sliced CZ (Schmidt bit s) puts the projector
# P_s = |s><s| on its lower-index qubit and Z^s on the other.  Between two
# events on one qubit, every CZ factor acting on it is diagonal in its basis;
# if each run of single-qubit gates between such factors is a monomial matrix
# (diagonal or anti-diagonal), the basis state |s> is carried to a basis
# state, so the next projector's bit (or, after the last one, the measured
# bit x_q) is fixed: equal to s, or flipped.  Slices that break such a tie
# contribute exactly zero (e.g. sqrt(Y) followed by the final Hadamard is
# diagonal up to a phase, which ties a late projector to the output bit).
# ---------------------------------------------------------------------------

def _monomial(U, tol=1e-12):
    """0 for a diagonal 2x2 matrix, 1 for an anti-diagonal one, None else."""
    U = np.asarray(U, dtype=np.complex128).reshape(2, 2)
    s = float(np.abs(U).max())
    if abs(U[0, 1]) <= tol * s and abs(U[1, 0]) <= tol * s:
        return 0
    if abs(U[0, 0]) <= tol * s and abs(U[1, 1]) <= tol * s:
        return 1
    return None


class _Runs:
    """Per qubit: the CZs acting on it in order, and the runs of single-qubit
    gates around them (run i precedes the qubit's i-th CZ; the last run ends
    at the measurement), each monomial with a parity or not; prefix sums give
    the status of any span of runs in O(1)."""

    def __init__(self, circ):
        n = circ.R * circ.C
        self.n = n
        runs = [[] for _ in range(n)]          # (monomial-or-None) per closed run
        cur = [np.eye(2, dtype=np.complex128) for _ in range(n)]
        self.proj_at = {}                      # CZ ordinal -> (projector qubit, its event index)
        k = 0

        def close(q, force_bad=False):
            m = None if force_bad else _monomial(cur[q])
            runs[q].append(m)
            cur[q] = np.eye(2, dtype=np.complex128)

        for g in circ.gates:
            if g.kind == "1q":
                q = g.qubits[0]
                cur[q] = np.asarray(g.U, dtype=np.complex128).reshape(2, 2) @ cur[q]
            elif g.kind == "cz":
                a, b = sorted(g.qubits)
                self.proj_at[k] = (a, len(runs[a]))
                close(a)
                close(b)
                k += 1
            else:
                for q in g.qubits:   # a general two-qubit gate: no tie across it
                    close(q, force_bad=True)
        for q in range(n):
            close(q)                  # the last run, up to the measurement
        self.bad = []
        self.par = []
        for q in range(n):
            b, p = [0], [0]
            for m in runs[q]:
                b.append(b[-1] + (m is None))
                p.append(p[-1] ^ (m or 0))
            self.bad.append(b)
            self.par.append(p)

    def span(self, q, lo, hi):
        """Runs lo .. hi-1 of qubit q: their parity, or None if one is not monomial."""
        if self.bad[q][hi] - self.bad[q][lo]:
            return None
        return self.par[q][hi] ^ self.par[q][lo]

    def constraints(self, sliced_cz, x=None):
        per_q = {}
        for j, o in enumerate(sliced_cz):
            q, ev = self.proj_at[int(o)]
            per_q.setdefault(q, []).append((ev, j))
        out = []
        for q, lst in per_q.items():
            lst.sort()
            prev_ev, prev_j = -1, -1          # the initial |0>: before run 0
            for ev, j in lst:
                # runs prev_ev+1 .. ev lie between the two events
                f = self.span(q, prev_ev + 1, ev + 1)
                if f is not None:
                    out.append((j, prev_j, f))
                prev_ev, prev_j = ev, j
            if x is not None:
                f = self.span(q, prev_ev + 1, len(self.bad[q]) - 1)
                if f is not None:
                    out.append((prev_j, -1, ((int(x) >> q) & 1) ^ f))
        return out


_RUNS_CACHE = {}


def _runs_of(circ):
    key = id(circ)
    hit = _RUNS_CACHE.get(key)
    if hit is None or hit[0] is not circ:
        hit = (circ, _Runs(circ))
        _RUNS_CACHE.clear()
        _RUNS_CACHE[key] = hit
    return hit[1]


def slice_constraints(circ, sliced_cz, x=None):
    """Ties between slice bits (bit j = sliced_cz[j]): a list of (j, i, c)
    meaning bit_j = bit_i xor c, with i = -1 for a constant (bit_j = c; the
    initial |0> or, when x is given, the measured output bit)."""
    return _runs_of(circ).constraints(sliced_cz, x)


def _tie_components(circ, sliced_cz, x):
    """Union-find with parities over the slice bits and a constant node (S);
    None when the ties contradict one another."""
    S = len(sliced_cz)
    parent = list(range(S + 1))
    par = [0] * (S + 1)

    def find(u):
        p = 0
        while parent[u] != u:
            p ^= par[u]
            u = parent[u]
        return u, p

    for j, i, c in slice_constraints(circ, sliced_cz, x):
        a, b = (j, S if i < 0 else i)
        ra, pa = find(a)
        rb, pb = find(b)
        if ra == rb:
            if pa ^ pb != c:
                return None
            continue
        parent[ra] = rb
        par[ra] = pa ^ pb ^ c
    return find


def slice_counts(circ, sliced_cz, x=None, lower_mask: int = 0):
    """(slices that can be nonzero, distinct values of the lower-half bits
    among them): 2^(free tie classes) and 2^(free classes holding a lower bit)."""
    S = len(sliced_cz)
    find = _tie_components(circ, sliced_cz, x)
    if find is None:
        return 0, 0
    const = find(S)[0]
    free = {}
    for u in range(S):
        r = find(u)[0]
        if r != const:
            free[r] = free.get(r, False) or bool((lower_mask >> u) & 1)
    return 2 ** len(free), 2 ** sum(1 for v in free.values() if v)


def consistent_slice_ids(circ, sliced_cz, x=None):
    """The slice ids that satisfy every tie of slice_constraints (the others
    are exactly zero), ascending; [] when the ties contradict one another."""
    S = len(sliced_cz)
    find = _tie_components(circ, sliced_cz, x)
    if find is None:
        return []
    const = find(S)[0]
    roots = sorted({find(u)[0] for u in range(S)} - {const})
    out = []
    for t in range(1 << len(roots)):
        val = {r: (t >> i) & 1 for i, r in enumerate(roots)}
        val[const] = 0
        sid = 0
        for u in range(S):
            r, p = find(u)
            if val[r] ^ p:
                sid |= 1 << u
        out.append(sid)
    return sorted(out)
