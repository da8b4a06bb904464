"""Replica path on several ranks, on CPU with the gloo backend: frames are
sharded round-robin, each rank detects its own with the oracle, and the merged
volume histogram equals the histogram of all frames detected in one process.
Also the max / sum reductions used for whole-job throughput."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as torchdist
import torch.multiprocessing as mp

import oracle
from paper_2010_08486_gb300 import dist, synth

P = oracle.OracleParams(min_sigma=1.0, max_sigma=10.0, ratio=1.6, threshold=0.1)
SEEDS = [31, 32, 33, 34, 35]


def _frame(seed):
    return synth.small_blob_frame(seed, 96, 80, n_blobs=6).astype(np.float64)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    torchdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = dist.shard(SEEDS, rank, world)
        h = torch.zeros(P.nbins, dtype=torch.int32)
        n_blobs = 0
        for s in mine:
            d = oracle.detect(_frame(s), P)
            h += torch.from_numpy(d.counts.astype(np.int32))
            n_blobs += len(d.blobs)
        merged = dist.merge_hists(h)
        total = dist.sum_over_ranks(n_blobs)
        slowest = dist.max_over_ranks(10.0 + rank)
        dist.barrier()
        out.put((rank, mine, merged.tolist(), total, slowest))
    finally:
        torchdist.destroy_process_group()


def test_shard_round_robin():
    items = list(range(11))
    parts = [dist.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        dist.shard(items, 3, 3)


def test_merge_single_process_is_identity():
    h = torch.tensor([1, 2, 3], dtype=torch.int32)
    assert dist.merge_hists(h).tolist() == [1, 2, 3]
    assert dist.max_over_ranks(2.5) == 2.5


def test_two_gloo_ranks_merge_equals_single_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # every frame went to exactly one rank
    assert sorted(sum((r[1] for r in res), [])) == SEEDS
    want = np.zeros(P.nbins, np.int64)
    n_all = 0
    for s in SEEDS:
        d = oracle.detect(_frame(s), P)
        want += d.counts.astype(np.int64)
        n_all += len(d.blobs)
    assert want.sum() > 0
    for r in res:
        assert r[2] == want.tolist()        # every rank holds the merged histogram
        assert r[3] == n_all
        assert r[4] == 10.0 + world - 1
