#!/usr/bin/env python3
"""Benchmark of the PEPS amplitude path on GB300.

Workload: the 6x6 lattice at depth (1+32+1) (bond dimension 16 on every
edge), 512 seeded bitstrings in 8 groups of 64 that share the bits of columns
0-2, whose running tensor after column 2 is computed once per group.  One
step = the whole path over the batch: circuit evolution (PEPS init, gate
absorption), projection / operand build, the 25 absorption steps of every
chain (36 sites; the two top and two bottom rows of a column are absorbed
together where that pays), FP64 reduction.

value   amplitudes/s of the mixed-precision path (FP16 hi/lo split, three
        tensor-core products, FP32 accumulate), bitstrings resident in HBM,
        CUDA events around the timed steps on the launch stream.
e2e     the same through the host C-ABI call (pinned host bitstrings copied
        in, amplitudes copied out, inside the timed region).
fp32_path  the plain FP32 CUDA-core form on the same GPU (timed on one group
        of 64 bitstrings; the work per amplitude is identical across groups).
square_partition  the same batch contracted by the square partition of the
        lattice (supplementary Fig. S2(b)): the same amplitudes (to 1e-5) at a
        fraction of the work.
roofline  the tensor-core contraction kernel: algorithmic flops per launch
        (8 real flops per complex multiply-add) / mean launch time from CUDA
        events recorded by the library around each launch.  `traffic` is the
        mean DRAM bytes (read + write) per launch of this kernel in a
        single-pass ncu capture of this bench command; it is reported only
        while the kernel's sources hash to the captured version.
cpu_baseline  the CPU FP64 oracle on a bounded sample (see "sample").

--impl reference times the CPU FP64 oracle on the same workload (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitudes/s at 6x6 (1+32+1), mixed vs FP32 path, rel.err <= 1e-5"
UNIT = "amplitudes/s"
WORKLOAD = "6x6_d32"
FLOPS_PER_CMAC = 8
REL_ERR_GATE = 1e-5
# the workload, identical in both arms' lines
CONFIG = {"workload": "6x6 (1+32+1), 512 bitstrings = 8 groups x 64 sharing columns 0-2",
          "seed": 4, "bitstrings": 512,
          "l2": "inputs larger than L2: with held and linked bits the square partition's "
                "running tensors have up to 2^22 entries (32 MiB) per lane, 4 buffers per lane "
                "x 512 lanes, 70 GB of workspace; the column sweep's up to 2^25 (256 MiB) "
                "per lane"}
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_6x6_d32.json")


def golden_check(out, bits, first=0):
    """Normwise relative error of `out` (amplitudes of bits[first:first+len(out)])
    against the FP64 oracle values of this batch stored in tests/golden (written
    by the oracle alone).  Returns None when the batch holds none of them."""
    import numpy as np

    with open(GOLDEN) as f:
        g = json.load(f)
    idx, ref, got = [], [], []
    for i, b, a in zip(g["indices"], g["bitstrings"], g["amplitudes"]):
        j = i - first
        if 0 <= j < len(out) and int(bits[i]) == int(b):
            idx.append(i)
            ref.append(complex(a[0], a[1]))
            got.append(complex(out[j]))
    if not idx:
        return None
    ref, got = np.array(ref), np.array(got)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"rel_err": err, "rel_err_ok": bool(err <= REL_ERR_GATE), "gate": REL_ERR_GATE,
            "checked": len(idx), "indices": idx,
            "against": "FP64 oracle values of these bitstrings (tests/golden/oracle_6x6_d32.json)"}

# DRAM bytes (read + write) of the tensor-core kernel per algorithmic byte,
# from one ncu capture (gpu__time_duration.sum, dram__bytes_read.sum,
# dram__bytes_write.sum) of the small case `bench.py --case group --lanes 16`
# (one prefix group of the batch, 16 lanes per launch, a few GB on the device):
# the sum over its tensor-core launches of the measured bytes over the sum of
# their algorithmic bytes (which the case prints).  The bench line's traffic
# per launch is this ratio times its own algorithmic bytes per launch: the
# same steps, with more lanes per launch, and traffic in proportion to the
# lanes.  Valid while the kernel's sources hash to the captured version.
TRAFFIC = {"sources_sha256_16": "99a6e6e12e7c04e0", "dram_per_algorithmic_byte": 0.836}
TRAFFIC_SOURCES = ("contract_tc.cu", "common.h", "format.cuh")


def measured_traffic(scheme, algorithmic_bytes_per_launch):
    """DRAM bytes per launch of the tensor-core kernel on this line, or None
    (no capture for this scheme, or the kernel changed since)."""
    import hashlib

    if scheme != "quadrants" or TRAFFIC["dram_per_algorithmic_byte"] is None:
        return None
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1905_08394_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != TRAFFIC["sources_sha256_16"]:
        return None
    return TRAFFIC["dram_per_algorithmic_byte"] * algorithmic_bytes_per_launch


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--precision", default="fp16x3")
    ap.add_argument("--lanes", type=int, default=16)
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--scheme", default="auto", choices=["auto", "columns", "quadrants"],
                    help="contraction scheme of the timed steps; auto = the faster of the "
                         "two on this workload, chosen by the autotuner")
    ap.add_argument("--other-steps", type=int, default=2,
                    help="timed calls of the scheme not chosen (reported under 'schemes'; "
                         "0 = skip)")
    ap.add_argument("--hold-ties", dest="hold_ties", action="store_true", default=True,
                    help="hold the CZ bits that each output bitstring fixes (default)")
    ap.add_argument("--no-hold-ties", dest="hold_ties", action="store_false")
    ap.add_argument("--tune-tiles", dest="tune_tiles", action="store_true", default=True,
                    help="after the contraction order, autotune lanes, K bytes per stage "
                         "and CTA pairing on this batch (default)")
    ap.add_argument("--no-tune-tiles", dest="tune_tiles", action="store_false")
    ap.add_argument("--slices7", dest="slices7", action="store_true", default=True,
                    help="also time the 7x7 (1+40+1) whole amplitude (180 GB slice set) and "
                         "add it to the line as slices_7x7 (default; about 75 s)")
    ap.add_argument("--no-slices7", dest="slices7", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--case", default="bench",
                    choices=["bench", "profile", "slices", "precision", "small", "peaks",
                             "quadrants", "pt8x8", "marginals", "evolution", "group"],
                    help="profile: one amplitude of the workload on one lane, no timing "
                         "(the small case for ncu captures, about 4 GiB on the device); "
                         "slices: 7x7 (1+40+1), the whole amplitude of one bitstring on "
                         "the sliced square partition, timed, with a second decomposition "
                         "as its check; precision: "
                         "6x6 (1+24+1), every form's amplitudes/s on 4096 bitstrings and its "
                         "error against the oracle on 64; small: 4x4 (1+8+1) and 5x5 (1+16+1), "
                         "eager launches vs CUDA-graph replay; peaks: this GPU's FP32 FMA "
                         "and tcgen05 kind::f16 / kind::tf32 rates from the microbenchmarks "
                         "in libpeps_peaks.so; quadrants: the bench workload by the square "
                         "partition of the lattice (supplementary Fig. S2(b)); pt8x8: the "
                         "paper's workstation experiment, 10000 amplitudes of an 8x8 (1+25+1) "
                         "circuit and their Porter-Thomas statistics; marginals: marginal "
                         "probabilities of the top half's 18 qubits of a 6x6 (1+16+1) "
                         "circuit (the double-layer network), 512 bitstrings; evolution: the "
                         "7x7 (1+40+1) circuit's evolution and operand build at full size (the "
                         "bandwidth kernels' case for ncu), one small slice contracted; group: "
                         "one prefix group of the bench batch with --lanes lanes (the tensor-"
                         "core kernel's case for ncu)")
    ap.add_argument("--check-full", action="store_true",
                    help="--case slices: also the amplitude from the slice set chosen without x")
    ap.add_argument("--group-only", action="store_true",
                    help="--case slices: only one run of slices that share the lower half "
                         "(the profiling case), timed in one call")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample
# ---------------------------------------------------------------------------

def oracle_sample(seconds: float, scheme: str = "quadrants", start: int = 0):
    """Time the FP64 oracle, as it stands, on this workload for about `seconds`.
      quadrants  the oracle's square partition (four quarters, the two pair
                 merges, the last contraction) of whole amplitudes of the
                 batch's bitstrings start, start+1, ... until the time is up
                 (at least one): measured amplitudes/s, nothing projected;
      columns    the oracle's column sweep of the batch's first bitstring,
                 cut off after `seconds` (one amplitude takes far longer) and
                 scaled by flops to the batched job's flops per amplitude
                 (prefix reuse over each group of 64): a projection.
    Returns (amplitudes/s, description, cores, projected, seconds spent,
    amplitudes done)."""
    import numpy as np

    from oracle import peps as op
    from paper_1905_08394_gb300 import complexity as cx
    from rqc_inputs import workload

    circ, bits = workload(WORKLOAD)
    p = op.build(circ.R, circ.C, circ.gates)
    R, C = circ.R, circ.C
    if scheme == "quadrants":
        t0 = time.perf_counter()
        done = 0
        while True:
            op.amplitude_quadrant(p, int(bits[(start + done) % len(bits)]))
            done += 1
            if time.perf_counter() - t0 > seconds:
                break
        dt = time.perf_counter() - t0
        rate = done / dt
        desc = (f"oracle O3 (numpy complex128 tensordot), square partition, {done} whole "
                f"amplitude(s) of the batch's bitstrings {start}..{start + done - 1} in {dt:.1f} s "
                f"(measured, not projected)")
        return rate, desc, os.cpu_count(), False, dt, done
    E = p.project(int(bits[0]))
    steps = cx.column_sweep_step_cmacs(R, C, 16)
    order = op.sweep_order(R, C, "column")
    G, labels = np.ones((), dtype=np.complex128), []
    t0 = time.perf_counter()
    done = 0
    cmacs = 0
    for i, q in enumerate(order):
        G, labels = op.absorb(G, labels, E[q], q, R, C)
        cmacs += steps[i]
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    per_amp = (8 * sum(steps[:18]) + 512 * sum(steps[18:])) / 512  # prefix reuse, as the GPU job
    rate = (cmacs / dt) / per_amp
    desc = (f"oracle O3 (numpy complex128 tensordot) column sweep of bitstring 0, first {done} "
            f"of 36 site absorptions ({cmacs * FLOPS_PER_CMAC:.3e} flops in {dt:.1f} s), scaled "
            f"by {per_amp * FLOPS_PER_CMAC:.3e} flops per amplitude of the batched job "
            f"(projected)")
    return rate, desc, os.cpu_count(), True, dt, 0


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"peps_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1].split()[0]))
                    smax.append(float(parts[2].split()[0]))
                    power.append(float(parts[3].split()[0]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# Arms
# ---------------------------------------------------------------------------


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world:
        raise SystemExit(f"bench.py --gpus {args.gpus} needs one process per GPU: launch it with "
                         f"torchrun --nproc-per-node {args.gpus} (WORLD_SIZE is {world})")
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "mine" else "gloo")
        pg = dist
    return world, rank, local, pg


def run_reference(args):
    """The reference arm: the CPU FP64 oracle as it stands, on this machine's host
    cores, on the workload of the GPU arm.  Each step is a bounded sample
    (whole amplitudes of the batch's bitstrings by the square partition),
    sized so that warm-up plus timed steps take about two and a half minutes;
    `value` is the amplitudes per second measured over the timed steps."""
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        if pg:
            pg.barrier()
        return
    scheme = args.scheme if args.scheme != "auto" else "quadrants"
    per_step = min(args.cpu_seconds, max(1.0, 150.0 / max(1, args.steps + args.warmup)))
    nxt = 0
    for _ in range(args.warmup):
        _, _, _, _, _, k = oracle_sample(0.0 if scheme == "quadrants" else 1.0, scheme, nxt)
        nxt += k
    spent, amps, rates = 0.0, 0, []
    desc = cores = None
    projected = False
    for _ in range(args.steps):
        v, desc, cores, projected, dt, k = oracle_sample(per_step, scheme, nxt)
        nxt += k
        spent += dt
        amps += k
        rates.append(v)
    value = amps / spent if not projected else sum(rates) / len(rates)
    sample = (f"{args.steps} step(s) of about {per_step:.1f} s each; last step: {desc}"
              if not projected else desc)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": spent / args.steps * 1000, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": dict(CONFIG),
            "scheme": scheme, "projected": projected,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "projected": projected},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()


def run_mine(args):
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator, autotune
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    from paper_1905_08394_gb300 import distributed as D

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    circ, _ = workload(WORKLOAD)
    # weak scaling: every rank contracts its own 8 prefix groups of 64 (rank 0
    # of a one-rank job gets exactly the single-GPU batch); no data exchange
    bits = D.rank_prefix_batch(6, 6, 3, 8, 64, 4, world, rank)
    n = len(bits)
    sim = Simulator(circ.R, circ.C, device=local)
    sim.apply_circuit(circ)
    stream = torch.cuda.Stream(device=dev)
    base_kw = dict(precision=args.precision, prefix_cols=3, prefix_group=64, max_lanes=args.lanes,
                   hold_ties=args.hold_ties)
    d_bits = torch.from_numpy(bits.view(np.int64)).to(dev)
    d_out = torch.empty(n, dtype=torch.complex128, device=dev)
    peaks, src = load_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    split = args.precision in ("fp16x3", "bf16x3")

    # contraction order: the autotuner times both schemes on this batch
    tuned = None
    if args.scheme == "auto":
        log = []
        best = autotune.tune(sim, d_bits, d_out, base_kw,
                             cands=[{"scheme": "columns"}, {"scheme": "quadrants"}], repeats=1,
                             stream=stream, log=log.append)
        scheme = best["scheme"]
        if pg:   # every rank runs the same order (rank 0's choice)
            t = torch.tensor([0 if scheme == "columns" else 1], device=dev)
            torch.distributed.broadcast(t, 0, group=pg)
            scheme = "columns" if int(t.item()) == 0 else "quadrants"
        tuned = {"chosen": scheme, "trials": log}
    else:
        scheme = args.scheme
    kw = dict(base_kw, scheme=scheme)
    # tile configuration for that order: lanes per launch, K bytes per stage,
    # CTA pairs (2-SM MMA) or single CTAs
    if args.tune_tiles:
        log = []
        lanes_c = (64, 128, 256, 512) if scheme == "quadrants" else (16, 32, 64)
        cands = [c for c in autotune.candidates(lanes=lanes_c, kchunk=(128, 64),
                                                cluster=(2, 1), schemes=(scheme,))]
        best = autotune.tune(sim, d_bits, d_out, kw, cands=cands, repeats=1, stream=stream,
                             log=log.append)
        if pg:   # rank 0's choice everywhere
            t = torch.tensor([best["max_lanes"], best["tc_kchunk"], best["tc_cluster"],
                              best.get("tc_epi", 0)], device=dev)
            torch.distributed.broadcast(t, 0, group=pg)
            best = {"scheme": scheme, "max_lanes": int(t[0]), "tc_kchunk": int(t[1]),
                    "tc_cluster": int(t[2]), "tc_epi": int(t[3])}
        kw.update(best)
        tuned = dict(tuned or {}, tile=best, tile_trials=log)
    # every step replays the call's CUDA graph (circuit evolution included);
    # the first and the last timed steps also record events around each
    # contraction launch (the graph with its 2 x 21 event nodes; reading them
    # back synchronises), which give the per-launch times of the roofline
    flags = B.PEPS_FLAG_GRAPH
    timed_event_steps = {0, args.steps - 1}

    def step(s, events=True):
        f = flags | (B.PEPS_FLAG_TIMING if events else 0)
        sim.amplitudes_device(d_bits, d_out, stream=s, flags=f, **kw)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):   # both graphs (with and without events) captured here
            step(stream, events=i == 0)
    stream.synchronize()
    if pg:
        pg.barrier()
    clocks = Clocks(local)
    clocks.start()
    tc_ms = tc_launches = 0.0
    tc_flops = tc_bytes = 0.0
    launches = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    tc_log = []   # (flops, bytes, ms) of every tensor-core contraction launch
    for i in range(args.steps):
        ev = i in timed_event_steps
        step(stream, events=ev)
        st = sim.stats()
        launches += st["launches_total"]
        if ev:
            tc_ms += st["contract_tc_ms"]
            tc_launches += st["launches_contract_tc"]
            tc_flops += st["contract_tc_flops"]
            tc_bytes += st["contract_tc_bytes"]
            tc_log += [(r["flops"], r["bytes"], r["ms"]) for r in B.peps_launch_log(sim.h)
                       if r["tensor_cores"]]
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if pg:
        ms = D.max_over_ranks(ms, pg, device=dev)
    ms_per_step = ms / args.steps
    value = world * n * args.steps / (ms / 1e3)

    # the timed output against the oracle's values of this batch (outside the
    # timed region)
    out = d_out.cpu().numpy()
    finite = bool(np.isfinite(out).all())
    check = golden_check(out, bits)

    # e2e through the host C-ABI call with pinned buffers
    pin_bits = torch.from_numpy(bits.view(np.int64)).pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    opts, keep = B.make_opts(flags=B.PEPS_FLAG_GRAPH, **kw)
    ws, nbytes = sim.workspace(n, opts)
    out_host = torch.empty(n, dtype=torch.complex128).pin_memory()
    lib = B.load()
    sptr = stream.cuda_stream

    def e2e_step():
        rc = lib.peps_amplitudes(sim.h, pin_bits.data_ptr(), n, out_host.data_ptr(),
                                 B.ct.byref(opts), ws, nbytes, sptr)
        if rc != 0:
            raise B.PepsError(rc, B.peps_last_error())

    e2e_step()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * n * e2e_steps / e2e_s

    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    def roofline_of(flops, ms_tc, nl, nbytes_alg, which, log=None):
        """The tensor-core kernel against its two ceilings.  Per launch the
        roofline time is max(issued flops / tensor peak, algorithmic bytes /
        HBM peak) (issued = 3x useful for the split forms); `bound` is the
        ceiling that accounts for more of that time over the launches, and
        achieved / peak / frac are given for it; both views are reported, as
        is the fraction of the summed roofline time the launches reached."""
        if not nl:
            return None
        avg = ms_tc / nl
        ach_t = (flops / nl) / (avg / 1e3) / 1e12
        ach_b = (nbytes_alg / nl) / (avg / 1e3) / 1e9
        mult = 3.0 if split else 1.0
        t_tensor = t_hbm = t_roof = 0.0
        if log:
            for f, b, ms in log:
                tt = mult * f / (peak * 1e12) * 1e3   # ms
                tb = b / (hbm_peak * 1e9) * 1e3
                t_roof += max(tt, tb)
                if tt >= tb:
                    t_tensor += tt
                else:
                    t_hbm += tb
        bound = "tensor" if t_tensor >= t_hbm else "hbm"
        tensor_view = {"achieved": ach_t, "peak": peak, "unit": "TFLOP/s", "frac": ach_t / peak,
                       "issued_frac": mult * ach_t / peak}
        hbm_view = {"achieved": ach_b, "peak": hbm_peak, "unit": "GB/s", "frac": ach_b / hbm_peak}
        main = tensor_view if bound == "tensor" else hbm_view
        return {"bound": bound, "achieved": main["achieved"], "peak": main["peak"],
                "unit": main["unit"], "frac": main["frac"],
                "traffic": measured_traffic(which, nbytes_alg / nl),
                "algorithmic_bytes": nbytes_alg / nl,
                "kernel": "k_contract_tc (tcgen05, fp16 hi/lo, 3 MMAs per k-step)",
                "peak_source": f"{src}: bf16 dense sustained (fp16 dense rate = bf16 rate), "
                               f"HBM copy",
                "tensor_view": tensor_view, "hbm_view": hbm_view,
                "roofline_time_frac": (t_roof / ms_tc) if log and ms_tc else None,
                "launches_tensor_bound_ms": t_tensor, "launches_hbm_bound_ms": t_hbm,
                "mean_launch_ms": avg, "launches": int(nl)}

    roof = roofline_of(tc_flops, tc_ms, tc_launches, tc_bytes, scheme, tc_log)
    schemes = {scheme: {"value": value, "ms_per_step": ms_per_step,
                        "flops_per_step": sim.plan_info(n, **kw)["flops_call"]}}

    # the other contraction order on the same batch, for comparison
    other = "quadrants" if scheme == "columns" else "columns"
    if args.other_steps > 0:
        kwo = dict(base_kw, scheme=other)   # untuned tiles
        sim.amplitudes_device(d_bits, d_out, stream=stream, flags=B.PEPS_FLAG_REBUILD, **kwo)
        stream.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(args.other_steps):
            sim.amplitudes_device(d_bits, d_out, stream=stream, flags=B.PEPS_FLAG_REBUILD, **kwo)
        q1.record(stream)
        stream.synchronize()
        mso = q0.elapsed_time(q1) / args.other_steps
        check_o = golden_check(d_out.cpu().numpy(), bits)
        sim.amplitudes_device(d_bits, d_out, stream=stream, flags=B.PEPS_FLAG_TIMING, **kwo)
        stream.synchronize()
        sto = sim.stats()
        schemes[other] = {"value": world * n / (mso / 1e3), "ms_per_step": mso,
                          "steps": args.other_steps, "check": check_o,
                          "flops_per_step": sim.plan_info(n, **kwo)["flops_call"],
                          "roofline": roofline_of(sto["contract_tc_flops"], sto["contract_tc_ms"],
                                                  sto["launches_contract_tc"],
                                                  sto["contract_tc_bytes"], other)}

    # FP32 CUDA-core form on one group of 64, same contraction order
    f32 = None
    if args.fp32_steps > 0:
        kw32 = dict(precision="fp32", prefix_cols=3, prefix_group=64,
                    max_lanes=kw.get("max_lanes", args.lanes), scheme=scheme,
                    hold_ties=args.hold_ties)
        d_b64 = d_bits[:64].contiguous()
        d_o64 = torch.empty(64, dtype=torch.complex128, device=dev)
        sim.amplitudes_device(d_b64, d_o64, stream=stream, flags=B.PEPS_FLAG_REBUILD, **kw32)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp32_steps):
            sim.amplitudes_device(d_b64, d_o64, stream=stream, flags=B.PEPS_FLAG_REBUILD, **kw32)
        e1.record(stream)
        stream.synchronize()
        ms32 = e0.elapsed_time(e1) / args.fp32_steps
        check32 = golden_check(d_o64.cpu().numpy(), bits)
        fl32 = sim.plan_info(64, **kw32)["flops_call"]
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = sms * 128 * 2 * 2070e6 / 1e12   # FP32 lanes x 2 flops x max SM clock
        f32 = {"value": 64 / (ms32 / 1e3), "unit": UNIT, "bitstrings": 64,
               "ms_per_step": ms32, "scheme": scheme,
               "note": "plain FP32 CUDA-core form, one group of 64", "check": check32,
               "roofline": {"bound": "alu", "achieved": fl32 / (ms32 / 1e3) / 1e12,
                            "peak": alu_peak, "unit": "TFLOP/s",
                            "frac": fl32 / (ms32 / 1e3) / 1e12 / alu_peak,
                            "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x 2070 MHz"}}

    # the paper's large run, after this workload's memory is released
    s7 = None
    if args.slices7 and rank == 0:
        sim.close()
        del d_bits, d_out
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        s7 = slices_7x7(args, check=False, warm=False)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, desc, cores, projected, _, _ = oracle_sample(args.cpu_seconds, scheme)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "projected": projected}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "fp16x3" if args.precision == "fp16x3" else args.precision,
                "data": "synthetic", "config": dict(CONFIG),
                "tuning": {"precision": args.precision, "lanes": kw.get("max_lanes", args.lanes),
                           "scheme": scheme, "hold_ties": args.hold_ties,
                           "tc_kchunk": kw.get("tc_kchunk", 0), "tc_cluster": kw.get("tc_cluster", 0),
                           "tc_epi": kw.get("tc_epi", 0),
                           "prefix_reuse": "columns 0-2 per group of 64", "autotune": tuned},
                "rel_err": check["rel_err"] if check else None,
                "rel_err_ok": check["rel_err_ok"] if check else None, "check": check,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                        "d2h_bytes_per_step": 16 * n},
                "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu,
                "fp32_path": f32, "schemes": schemes, "clocks": clk, "finite": finite,
                "slices_7x7": s7}
        print(json.dumps(line), flush=True)
    sim.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_profile_case(args):
    """One amplitude (bitstring 0) of the workload through one lane, by the
    given contraction scheme (auto = the square partition, which the
    autotuner picks on this workload), with the tied bits held as in the
    bench (--no-hold-ties: without)."""
    import numpy as np

    from paper_1905_08394_gb300 import Simulator
    from rqc_inputs import workload

    circ, bits = workload(WORKLOAD)
    sim = Simulator(circ.R, circ.C)
    sim.apply_circuit(circ)
    scheme = "quadrants" if args.scheme == "auto" else args.scheme
    out = sim.amplitudes(bits[:1], precision=args.precision, max_lanes=1, scheme=scheme,
                         hold_ties=args.hold_ties)
    st = sim.stats()
    print(json.dumps({"case": "profile", "scheme": scheme, "hold_ties": args.hold_ties,
                      "amplitude": [out[0].real, out[0].imag],
                      "launches": st["launches_total"], "tc_launches": st["launches_contract_tc"],
                      "finite": bool(np.isfinite(out).all())}))
    sim.close()


def slices_7x7(args, check: bool = True, check_full: bool = False, warm: bool = True):
    """7x7 (1+40+1), one bitstring x, on the odd-side square partition (Fig.
    S2(c)): the whole amplitude.  The slice set is the square-partition
    chooser's under a 180 GB workspace, given x: the CZs whose bit x fixes
    are cut first (they add no slices), and only the slices that can be
    nonzero run (slicing.consistent_slice_ids), lower-half reuse included.
    Timed in one call, the evolution included, with clocks sampled meanwhile.
    With `check`, the same amplitude from a second slice set (another budget
    and seed) is the cross-check; with `check_full` also from the slice set
    chosen without x (every slice of it that can be nonzero, ~10 min).
    Returns the record (a dict)."""
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator, slicing
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    circ, bits = workload("7x7_d40")
    x = int(bits[0])
    sim = Simulator(circ.R, circ.C)
    sim.apply_circuit(circ)
    t0 = time.time()
    ss = slicing.choose_quadrants(sim.h, circ, 180 * 10 ** 9, precision=args.precision, seed=5, x=x)
    choose_s = time.time() - t0
    ids = slicing.consistent_slice_ids(circ, ss.sliced_cz, x)
    lmask = slicing.lower_half_mask(circ, ss.sliced_cz)
    stream = torch.cuda.current_stream()
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    base = dict(precision=args.precision, scheme="quadrants")
    kw = dict(base, sliced_cz=ss.sliced_cz, slice_ids=ids)
    ws_opts, ws_keep = B.make_opts(**kw)
    ws_bytes = B.peps_workspace_bytes(sim.h, 1, ws_opts)
    # warm-up: one run of slices that share the lower half (evolution, kernels)
    group = [i for i in ids if (i & lmask) == (ids[0] & lmask)]
    t0 = time.time()
    if warm:
        sim.amplitudes_device(d_bits, flags=B.PEPS_FLAG_TIMING, **dict(kw, slice_ids=group))
        torch.cuda.synchronize()
    if args.group_only:
        st = sim.stats()
        rec = {"case": "slices", "workload": "7x7 (1+40+1), one run of slices that share the "
               "lower half", "slices": len(group), "wall_seconds": time.time() - t0,
               "contract_seconds": st["contract_ms"] / 1e3, "flops": st["contract_flops"],
               "launches": st["launches_total"]}
        sim.close()
        return rec
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = sim.amplitudes_device(d_bits, flags=B.PEPS_FLAG_TIMING | B.PEPS_FLAG_REBUILD, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_call = e0.elapsed_time(e1) / 1e3
    st = sim.stats()
    amp = complex(out.cpu().numpy()[0])
    n = circ.R * circ.C
    rec = {"workload": "7x7 (1+40+1), 1 bitstring, the whole amplitude (the paper's Table I run)",
           "scheme": "quadrants (odd side)", "precision": args.precision,
           "sliced_cz": len(ss.sliced_cz), "slices_run": len(ids),
           "lower_groups": len({i & lmask for i in ids}),
           "max_entries": ss.max_entries, "workspace_bytes": ws_bytes,
           "workspace_within_180GB": bool(ws_bytes <= 180 * 10 ** 9),
           "flops_total": ss.flops_total, "planned_flops_call": st["contract_flops"],
           "chooser_seconds": choose_s, "seconds": t_call,
           "seconds_per_slice": t_call / max(1, len(ids)),
           "contract_seconds": st["contract_ms"] / 1e3, "launches": st["launches_total"],
           "useful_tflops": st["contract_flops"] / t_call / 1e12,
           "amplitude": [amp.real, amp.imag], "n_abs2": (2 ** n) * abs(amp) ** 2,
           "clocks": clk,
           "paper": "Tianhe-2, 4096 fat nodes, FP64: 31 min for one amplitude "
                    "(odd-square partition, 92.51 TB)"}
    if check:
        # a second decomposition of the same amplitude
        s2 = slicing.choose_quadrants(sim.h, circ, 120 * 2 ** 30, precision=args.precision, seed=7,
                                      x=x)
        ids2 = slicing.consistent_slice_ids(circ, s2.sliced_cz, x)
        t1 = time.time()
        amp2 = complex(sim.amplitudes(bits, sliced_cz=s2.sliced_cz, slice_ids=ids2, **base)[0])
        rec["check"] = {"sliced_cz": len(s2.sliced_cz), "slices": len(ids2),
                        "flops": s2.flops_total, "amplitude": [amp2.real, amp2.imag],
                        "wall_seconds": time.time() - t1,
                        "rel_diff": abs(amp2 - amp) / abs(amp) if amp != 0 else None}
    if check_full:
        s3 = slicing.choose_quadrants(sim.h, circ, 180 * 10 ** 9, precision=args.precision, seed=5)
        ids3 = slicing.consistent_slice_ids(circ, s3.sliced_cz, x)
        t1 = time.time()
        amp3 = complex(sim.amplitudes(bits, sliced_cz=s3.sliced_cz, slice_ids=ids3, **base)[0])
        rec.setdefault("check", {})["without_x"] = {
            "sliced_cz": len(s3.sliced_cz), "slices": len(ids3),
            "amplitude": [amp3.real, amp3.imag], "wall_seconds": time.time() - t1,
            "rel_diff": abs(amp3 - amp) / abs(amp) if amp != 0 else None}
    # the column sweep's slice set, for comparison (planner figures only)
    cs = slicing.choose(circ, 2 ** 33, seed=5)
    rec["columns"] = {"sliced_cz": len(cs.sliced_cz), "max_entries": cs.max_entries,
                      "flops_per_slice": 8 * sum(cs.step_cmacs),
                      "flops_total": 8 * sum(cs.step_cmacs) * 2.0 ** len(cs.sliced_cz)}
    sim.close()
    return rec


def run_group_case(args):
    """One prefix group of the bench batch (its first 64 bitstrings, sharing
    columns 0-2) in the bench's configuration (square partition, tied bits
    held, --lanes lanes per launch): the small case whose kernel launches
    have the bench's shapes per lane, for ncu counter captures."""
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    circ, bits = workload(WORKLOAD)
    sim = Simulator(circ.R, circ.C)
    sim.apply_circuit(circ)
    kw = dict(precision=args.precision, prefix_cols=3, prefix_group=64, max_lanes=args.lanes,
              scheme="quadrants", hold_ties=args.hold_ties)
    out = sim.amplitudes(bits[:64], flags=B.PEPS_FLAG_TIMING, **kw)
    check = golden_check(out, bits)
    st = sim.stats()
    o, keep = B.make_opts(**kw)
    log = B.peps_launch_log(sim.h)
    print(json.dumps({"case": "group", "lanes": args.lanes, "hold_ties": args.hold_ties,
                      "launches": st["launches_total"], "tc_launches": st["launches_contract_tc"],
                      "workspace_bytes": B.peps_workspace_bytes(sim.h, 64, o),
                      "tc_launch_bytes": [r["bytes"] for r in log if r["tensor_cores"]],
                      "tc_launch_steps": [r["step"] for r in log if r["tensor_cores"]],
                      "check": check, "finite": bool(np.isfinite(out).all())}), flush=True)
    sim.close()


def run_slices_case(args):
    rec = slices_7x7(args, check=True, check_full=args.check_full)
    print(json.dumps(dict({"case": "slices"}, **rec)), flush=True)


def _time_calls(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def run_precision_case(args):
    """6x6 (1+24+1), 4096 seeded bitstrings: throughput of every form and its
    normwise error against the FP64 oracle on the first 64."""
    import numpy as np
    import torch

    from oracle import peps as op
    from paper_1905_08394_gb300 import Simulator
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    circ, bits = workload("6x6_d24")
    ref = op.amplitudes(op.build(6, 6, circ.gates), bits[:64])
    sim = Simulator(6, 6)
    sim.apply_circuit(circ)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    d_out = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
    peaks, src = load_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    bf16_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rows = []
    for prec in ("fp32", "tf32", "bf16", "bf16x3", "fp16", "fp16x3"):
        kw = dict(precision=prec, max_lanes=args.lanes, flags=B.PEPS_FLAG_REBUILD)
        sec = _time_calls(lambda: sim.amplitudes_device(d_bits, d_out, **kw), max(1, args.steps))
        out = d_out.cpu().numpy()
        err = float(np.linalg.norm(out[:64] - ref) / np.linalg.norm(ref))
        pt = float(np.mean((2.0 ** 36) * np.abs(out) ** 2))
        info = sim.plan_info(len(bits), precision=prec, max_lanes=args.lanes)
        tf = info["flops_call"] / sec / 1e12
        gbs = info["bytes_call"] / sec / 1e9
        # the form's own ceilings: its tensor rate (issued = 3x useful for the split
        # forms), or the FP32 lanes for the CUDA-core form; and HBM for the bytes
        if prec == "fp32":
            peak_t = sms * 128 * 2 * 2070e6 / 1e12
        elif prec == "tf32":
            peak_t = bf16_peak * 1100.0 / 2250.0
        else:
            peak_t = bf16_peak
        issued = 3 if prec in ("bf16x3", "fp16x3") else 1
        rows.append({"precision": prec, "amplitudes_per_s": len(bits) / sec, "rel_err": err,
                     "mean_N_abs2": pt, "useful_tflops": tf, "algorithmic_gbs": gbs,
                     "compute_frac": issued * tf / peak_t, "hbm_frac": gbs / hbm_peak})
    print(json.dumps({"case": "precision", "workload": "6x6 (1+24+1), 4096 bitstrings",
                      "oracle_bitstrings": 64, "forms": rows,
                      "peaks": {"hbm_gbs": hbm_peak, "bf16_tflops_sustained": bf16_peak,
                                "tf32": "bf16 x 1100/2250 (nominal ratio)",
                                "fp32": "SMs x 128 lanes x 2 flops x 2070 MHz",
                                "source": src}}), flush=True)
    sim.close()


def run_small_case(args):
    """4x4 (1+8+1) with 64 bitstrings and 5x5 (1+16+1) with 1024: launch-latency
    bound.  The whole-sweep path (the evolution as one launch with a block per
    site, every bitstring's column sweep in one persistent launch with the
    running tensor in shared memory) against the step-by-step launches
    (STEPWISE), each eager and replayed as a CUDA graph."""
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    out = []
    for name, prec in (("4x4_d8", "fp32"), ("5x5_d16", "fp32"), ("5x5_d16", "fp16x3")):
        circ, bits = workload(name)
        sim = Simulator(circ.R, circ.C)
        sim.apply_circuit(circ)
        d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
        d_out = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
        res = {"workload": name, "precision": prec, "bitstrings": len(bits)}
        ref = None
        for mode, flags in (("eager", B.PEPS_FLAG_REBUILD), ("graph", B.PEPS_FLAG_GRAPH),
                            ("stepwise_eager", B.PEPS_FLAG_REBUILD | B.PEPS_FLAG_STEPWISE),
                            ("stepwise_graph", B.PEPS_FLAG_GRAPH | B.PEPS_FLAG_STEPWISE)):
            kw = dict(precision=prec, max_lanes=64, flags=flags)
            sec = _time_calls(lambda: sim.amplitudes_device(d_bits, d_out, **kw), 50)
            amps = d_out.cpu().numpy()
            if ref is None:
                ref = amps
            res[mode] = {"amplitudes_per_s": len(bits) / sec, "us_per_call": sec * 1e6,
                         "launches_per_call": sim.stats()["launches_total"],
                         "rel_diff_vs_eager": float(np.linalg.norm(amps - ref) /
                                                    np.linalg.norm(ref))}
        out.append(res)
        sim.close()
    print(json.dumps({"case": "small", "results": out}), flush=True)


def run_quadrants_case(args):
    """The bench workload (6x6 (1+32+1), 512 bitstrings in 8 groups of 64
    sharing columns 0-2) contracted by the square partition: per group the
    two left quarters and F_l = F_ul F_bl^T, per bitstring the two right
    quarters, Y = F_br F_l^T and the dot product with F_ur.  Amplitudes/s of
    the FP16X3 and FP32 forms, and the tensor-core roofline of the merges."""
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    circ, bits = workload(WORKLOAD)
    sim = Simulator(circ.R, circ.C)
    sim.apply_circuit(circ)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    d_out = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
    peaks, src = load_peaks()
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    clocks = Clocks(0)
    clocks.start()
    res = {}
    for prec, reps in ((args.precision, max(1, args.steps)), ("fp32", 1)):
        kw = dict(precision=prec, prefix_cols=3, prefix_group=64, max_lanes=args.lanes,
                  scheme="quadrants")
        sec = _time_calls(lambda: sim.amplitudes_device(d_bits, d_out, flags=B.PEPS_FLAG_REBUILD,
                                                        **kw), reps)
        sim.amplitudes_device(d_bits, d_out, flags=B.PEPS_FLAG_TIMING, **kw)
        torch.cuda.synchronize()
        st = sim.stats()
        info = sim.plan_info(len(bits), **kw)
        r = {"amplitudes_per_s": len(bits) / sec, "ms_per_call": sec * 1e3,
             "useful_tflops": info["flops_call"] / sec / 1e12,
             "launches": st["launches_total"]}
        if st["launches_contract_tc"]:
            ach = st["contract_tc_flops"] / (st["contract_tc_ms"] / 1e3) / 1e12
            r["tc_roofline"] = {"achieved": ach, "peak": bf16, "frac": ach / bf16,
                                "issued_frac": 3 * ach / bf16 if prec in ("fp16x3", "bf16x3") else None}
        res[prec] = r
    clk = clocks.stop()
    print(json.dumps({"case": "quadrants", "workload": "6x6 (1+32+1), 512 bitstrings = 8 groups "
                      "x 64 sharing columns 0-2", "results": res, "clocks": clk,
                      "peak_source": src}), flush=True)
    sim.close()


def run_pt8x8_case(args):
    """The paper's workstation experiment: 10000 amplitudes of an 8x8
    (1+25+1) circuit (uniform seeded bitstrings) by the square partition, and
    the Porter-Thomas statistics of N |a|^2 (mean 1, second moment 2, and the
    Kolmogorov-Smirnov distance to Exp(1)).  The paper took under an hour per
    amplitude on a 2-core PC."""
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    circ, bits = workload("8x8_d25")
    sim = Simulator(8, 8)
    sim.apply_circuit(circ)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    d_out = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
    kw = dict(precision=args.precision, scheme="quadrants", max_lanes=32)
    sim.amplitudes_device(d_bits[:64], d_out[:64], flags=B.PEPS_FLAG_REBUILD, **kw)  # warm-up
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sim.amplitudes_device(d_bits, d_out, flags=B.PEPS_FLAG_REBUILD, **kw)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = e0.elapsed_time(e1) / 1e3
    out = d_out.cpu().numpy()
    pt = np.sort((2.0 ** 64) * np.abs(out) ** 2)
    cdf = 1 - np.exp(-pt)
    n = len(pt)
    D = float(max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(n) / n)))
    info = sim.plan_info(len(bits), **kw)
    print(json.dumps({"case": "pt8x8", "workload": "8x8 (1+25+1), seed 6, 10000 uniform bitstrings",
                      "precision": args.precision, "scheme": "quadrants",
                      "seconds": sec, "amplitudes_per_s": n / sec,
                      "useful_tflops": info["flops_call"] / sec / 1e12,
                      "flops_per_amplitude": info["flops_call"] / n,
                      "max_entries": info["max_entries"],
                      "porter_thomas": {"mean_N_abs2": float(pt.mean()),
                                        "second_moment": float(np.mean(pt ** 2)),
                                        "ks_distance": D, "ks_p01_threshold": 1.63 / n ** 0.5},
                      "paper": "under 1 h per amplitude on a PC (2 cores, 2.8 GHz, 16 GB), "
                               "10000 amplitudes",
                      "clocks": clk}), flush=True)
    sim.close()


def run_marginals_case(args):
    """Marginal probabilities P(x_S) of the 18 qubits in rows 0-2 of a 6x6
    (1+16+1) circuit (seed 24), for 512 seeded bitstrings: the double-layer
    network (bond dimension 16, the size of the 6x6 (1+32+1) amplitude)
    through the same kernels, by both contraction schemes."""
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import make_circuit, uniform_bitstrings

    circ = make_circuit(6, 6, 16, 24)
    bits = uniform_bitstrings(36, 512, 24)
    mask = (1 << 18) - 1
    sim = Simulator(6, 6)
    sim.apply_circuit(circ)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    d_out = torch.empty(len(bits), dtype=torch.complex128, device="cuda")
    res = {}
    for scheme in ("quadrants", "columns"):
        kw = dict(precision=args.precision, scheme=scheme, max_lanes=args.lanes, measured_mask=mask)
        reps = 2 if scheme == "quadrants" else 1
        sec = _time_calls(lambda: sim.amplitudes_device(d_bits, d_out, flags=B.PEPS_FLAG_REBUILD, **kw), reps)
        out = d_out.cpu().numpy()
        info = sim.plan_info(len(bits), **kw)
        res[scheme] = {"marginals_per_s": len(bits) / sec, "ms_per_call": sec * 1e3,
                       "useful_tflops": info["flops_call"] / sec / 1e12,
                       "mean_2^18_P": float(np.mean(out.real) * 2 ** 18),
                       "max_abs_imag_over_real": float(np.max(np.abs(out.imag)) / np.max(np.abs(out.real)))}
    print(json.dumps({"case": "marginals", "workload": "6x6 (1+16+1) seed 24, qubits 0-17 measured, "
                      "512 bitstrings", "precision": args.precision, "results": res}), flush=True)
    sim.close()


def run_evolution_case(args):
    """The bandwidth kernels at the paper's size: the circuit evolution (PEPS
    init, single-qubit gate absorption, CZ absorption with bond doubling) and
    the projection / operand build of the 7x7 (1+40+1) circuit, whose site
    tensors reach 2 x 32^4 complex entries (32 MiB each as float-float).  The
    contraction is kept small by holding the 80 CZ bits of the column sweep's
    cut set under 2^24 entries (one sub-slice).  One timed call; the
    evolution's share is reported from its launch count and the
    contraction's event time."""
    import numpy as np
    import torch

    from paper_1905_08394_gb300 import Simulator, slicing
    from paper_1905_08394_gb300 import binding as B
    from rqc_inputs import workload

    circ, bits = workload("7x7_d40")
    sim = Simulator(circ.R, circ.C)
    sim.apply_circuit(circ)
    cs = slicing.choose(circ, 2 ** 24, seed=5)
    kw = dict(precision=args.precision, fixed_cz=cs.sliced_cz, fixed_s=[0] * len(cs.sliced_cz),
              fuse_rows=1)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    sim.amplitudes_device(d_bits, flags=B.PEPS_FLAG_REBUILD, **kw)   # plan + warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sim.amplitudes_device(d_bits, flags=B.PEPS_FLAG_REBUILD | B.PEPS_FLAG_TIMING, **kw)
    e1.record()
    torch.cuda.synchronize()
    st = sim.stats()
    o, keep = B.make_opts(**kw)
    print(json.dumps({"case": "evolution", "workload": "7x7 (1+40+1): evolution and operand "
                      "build at full size, one sub-slice of an 80-bit cut set",
                      "call_ms": e0.elapsed_time(e1), "contract_ms": st["contract_ms"],
                      "launches_evolve": st["launches_evolve"],
                      "launches_operand": st["launches_operand"],
                      "workspace_bytes": B.peps_workspace_bytes(sim.h, 1, o)}), flush=True)
    sim.close()


def run_peaks_case(args):
    """Peak rates measured by this repository's own microbenchmarks: the FP32
    FMA rate of the CUDA cores and the dense tcgen05 rate for kind::f16 and
    kind::tf32 (operands in shared memory, no DRAM traffic), with the clocks
    seen meanwhile and the nominal figures they compare to."""
    import ctypes as ct

    import torch

    lib = ct.CDLL(os.path.join(ROOT, "paper_1905_08394_gb300", "libpeps_peaks.so"))
    for f in (lib.peaks_fma_tflops, lib.peaks_mma_tflops):
        f.restype = ct.c_int
    torch.cuda.init()
    props = torch.cuda.get_device_properties(0)
    clocks = Clocks(0)
    clocks.start()
    res = {}
    for name, call in (("fp32_fma", lambda t, m: lib.peaks_fma_tflops(1000000, t, m)),
                       ("tcgen05_f16", lambda t, m: lib.peaks_mma_tflops(0, 200000, t, m)),
                       ("tcgen05_tf32", lambda t, m: lib.peaks_mma_tflops(1, 100000, t, m))):
        best = 0.0
        for _ in range(3):
            t, ms = ct.c_double(0), ct.c_double(0)
            rc = call(ct.byref(t), ct.byref(ms))
            if rc != 0:
                raise RuntimeError(f"{name}: microbenchmark failed ({rc})")
            best = max(best, t.value)
        res[name] = best
    clk = clocks.stop()
    sms = props.multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    peaks, src = load_peaks()
    print(json.dumps({
        "case": "peaks", "sms": sms, "tflops": res, "clocks": clk,
        "nominal_tflops": {"fp32_fma": sms * 128 * 2 * mhz * 1e6 / 1e12,
                           "f16_dense": 2250.0, "tf32_dense": 1100.0},
        "cublas_bf16_tflops": {"burst": peaks.get("bf16_tflops"),
                               "sustained": peaks.get("bf16_tflops_sustained"), "source": src},
    }), flush=True)


def main():
    args = parse()
    if args.case == "profile":
        run_profile_case(args)
    elif args.case == "slices":
        run_slices_case(args)
    elif args.case == "precision":
        run_precision_case(args)
    elif args.case == "peaks":
        run_peaks_case(args)
    elif args.case == "quadrants":
        run_quadrants_case(args)
    elif args.case == "pt8x8":
        run_pt8x8_case(args)
    elif args.case == "marginals":
        run_marginals_case(args)
    elif args.case == "small":
        run_small_case(args)
    elif args.case == "evolution":
        run_evolution_case(args)
    elif args.case == "group":
        run_group_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
