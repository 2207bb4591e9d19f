"""Autotuner for the contraction: times candidate configurations on the
caller's own workload and keeps the fastest.  The candidates vary the
contraction order (the column sweep, or the square partition of the
supplementary Fig. S2(b) on even lattices) and the tile configuration (K bytes
per pipeline stage, CTA pairs, lanes per launch).  Results are cached in a
JSON file keyed by the workload signature.  Every candidate computes the same
amplitudes (to rounding), so the choice is purely about speed.
"""
from __future__ import annotations

import itertools
import json
import os
import time

DEFAULT_CACHE = os.environ.get("PEPS_TUNE_CACHE", "")


def signature(sim, n: int, kw: dict) -> str:
    dims = []
    for r in range(sim.R):
        for c in range(sim.C):
            if c + 1 < sim.C:
                dims.append(sim.bond_dim(r, c, r, c + 1))
            if r + 1 < sim.R:
                dims.append(sim.bond_dim(r, c, r + 1, c))
    keys = ("precision", "prefix_cols", "prefix_group", "sliced_cz", "scheme", "hold_ties")
    rest = {k: (list(kw[k]) if k == "sliced_cz" else kw[k]) for k in keys if k in kw and kw[k] is not None}
    return json.dumps({"R": sim.R, "C": sim.C, "dims": dims, "n": n, **rest}, sort_keys=True)


def candidates(lanes=(8, 16, 32), kchunk=(128, 64), cluster=(1, 2), schemes=("columns",),
               epi=(0,)):
    """The product of the given choices; pass schemes=("columns", "quadrants")
    on an even lattice to let the contraction order be tuned as well."""
    for sc, l, k, c, e in itertools.product(schemes, lanes, kchunk, cluster, epi):
        yield {"scheme": sc, "max_lanes": l, "tc_kchunk": k, "tc_cluster": c, "tc_epi": e}


def tune(sim, d_bits, d_out, kw: dict, cands=None, repeats: int = 2, cache: str = DEFAULT_CACHE,
         stream=None, log=None) -> dict:
    """Return the fastest candidate (a dict of amplitude-call keywords) for
    this workload; `kw` holds the call's other keywords."""
    import torch

    n = d_bits.numel()
    sig = signature(sim, n, kw)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if sig in table:
            return table[sig]["best"]
    cands = list(cands if cands is not None else candidates())
    timings = []
    for cand in cands:
        if cand.get("max_lanes", 1) > max(1, n):
            continue
        args = dict(kw)
        args.update(cand)
        sim.amplitudes_device(d_bits, d_out, stream=stream, **args)  # plan + warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(repeats):
            sim.amplitudes_device(d_bits, d_out, stream=stream, **args)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / repeats
        timings.append((dt, cand))
        if log:
            log(f"autotune {cand}: {dt * 1e3:.1f} ms")
    timings.sort(key=lambda x: x[0])
    best = timings[0][1]
    if cache:
        table = {}
        if os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        table[sig] = {"best": best, "ms": [[t * 1e3, c] for t, c in timings]}
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return best
