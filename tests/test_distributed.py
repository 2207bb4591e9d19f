"""Multi-rank host logic on CPU with the gloo backend (world size 2): shards
of independent units are disjoint and cover the batch, the timing reduction
takes the max, and sliced partial amplitudes sum in FP64."""
import os
import socket

import numpy as np
import pytest

from paper_1905_08394_gb300 import distributed as D
from rqc_inputs import workload


def test_shard_covers_and_is_balanced():
    for n in (0, 1, 7, 8, 512, 513):
        for world in (1, 2, 3, 8):
            spans = [D.shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_rank_batches_weak_scaling():
    circ, bits = workload("6x6_d32")
    one = D.rank_prefix_batch(6, 6, 3, 8, 64, 4, 1, 0)
    assert np.array_equal(one, bits)           # one rank = the single-GPU batch
    b0 = D.rank_prefix_batch(6, 6, 3, 8, 64, 4, 2, 0)
    b1 = D.rank_prefix_batch(6, 6, 3, 8, 64, 4, 2, 1)
    assert len(b0) == len(b1) == 512
    assert np.array_equal(b0, bits)
    assert not set(b0.tolist()) & set(b1.tolist())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bits = D.rank_prefix_batch(4, 4, 2, 3, 5, 9, world, rank)
        t = D.max_over_ranks(1.5 + rank, dist)
        part = np.array([complex(rank + 1, -rank), complex(0.25, 0.5 * rank)])
        tot = D.allreduce_sum_c128(part, dist)
        q.put((rank, bits.tolist(), t, tot.tolist()))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, t0, s0), (r1, b1, t1, s1) = res
    assert t0 == t1 == 2.5
    assert s0 == s1 == [complex(3, -1), complex(0.5, 0.5)]
    assert not set(b0) & set(b1) and len(b0) == len(b1) == 15


def test_rank_slices_keep_lower_runs_whole():
    ids = [0, 1, 4, 5, 8, 9, 12, 13, 2, 6]
    mask = 0b1100
    shares = [D.rank_slice_ids(ids, mask, 3, r) for r in range(3)]
    assert sorted(i for s in shares for i in s) == sorted(ids)
    for s in shares:
        for t in shares:
            if s is not t:
                assert not {i & mask for i in s} & {i & mask for i in t}


def _slice_worker(rank, world, port, q):
    # each rank sums its share of a sliced amplitude (the CPU oracle stands in
    # for the GPU contraction here); the FP64 allreduce gives the amplitude
    import torch.distributed as dist

    from oracle import peps as op
    from paper_1905_08394_gb300 import slicing
    from rqc_inputs import make_circuit, uniform_bitstrings

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        circ = make_circuit(3, 3, 16, 5)
        x = int(uniform_bitstrings(9, 1, 5)[0])
        ncz = sum(1 for g in circ.gates if g.kind == "cz")
        sl = [1, 4, 9, ncz - 3, ncz - 2, ncz - 1]
        ids = slicing.consistent_slice_ids(circ, sl, x)
        mine = D.rank_slice_ids(ids, slicing.lower_half_mask(circ, sl), world, rank)
        part = sum((op.amplitudes(op.build(3, 3, circ.gates, sliced=sl, slice_id=i), [x])
                    for i in mine), np.zeros(1, dtype=np.complex128))
        tot = D.allreduce_sum_c128(part, dist)
        full = op.amplitudes(op.build(3, 3, circ.gates), [x])
        q.put((rank, len(mine), tot.tolist(), full.tolist()))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_share_the_slices_of_an_amplitude():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slice_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, t0, f0), (r1, n1, t1, f1) = res
    assert n0 > 0 and n1 > 0 and t0 == t1
    assert abs(t0[0] - f0[0]) <= 1e-12 * abs(f0[0])
