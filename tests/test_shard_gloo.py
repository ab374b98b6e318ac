"""Multi-rank path on CPU: world_size-2 gloo process groups.

The batch shards with no data-path collective; these tests check on the
host that the shards cover every transform exactly once and balance the
work, that the timing reduction takes the max over ranks, and (with the
FP64 oracle standing in for each rank's kernels) that transforming the
shards independently and reassembling them equals transforming the whole
batch."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2603_27569_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rows of a fixed-length batch
        batch, N = 37, 64
        x = synth.gaussian((batch, N), seed=0)
        s, c = shard.shard_rows(batch, rank, world)
        mine = oracle.fft(x[s:s + c])
        # a ragged list
        d = synth.ragged_draw(50, seed=1, log2_lo=4, log2_hi=9)
        owner = shard.shard_ragged(d["N"], world)
        xr = synth.gaussian(d["total"], seed=2)
        rag = {int(i): oracle.fft(xr[d["offset"][i]:d["offset"][i] + d["N"][i]],
                                  inverse=d["direction"][i] > 0)
               for i in np.nonzero(owner == rank)[0]}
        t_max = shard.max_over_ranks(1.5 + rank)
        out = [None] * world
        dist.all_gather_object(out, (rank, s, c, mine, rag, owner.tolist(), t_max))
        if rank == 0:
            q.put(out)
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding_matches_whole_batch():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle

    # rows: shards tile [0, batch) and reassemble to the whole transform
    batch, N = 37, 64
    x = synth.gaussian((batch, N), seed=0)
    whole = oracle.fft(x)
    got = np.empty_like(whole)
    covered = np.zeros(batch, int)
    for rank, s, c, mine, rag, owner, t_max in out:
        got[s:s + c] = mine
        covered[s:s + c] += 1
        assert t_max == 2.5                       # max over ranks of 1.5 + rank
    assert (covered == 1).all()
    assert np.array_equal(got, whole)
    # ragged: every transform computed once, by its owner, equal to the oracle
    d = synth.ragged_draw(50, seed=1, log2_lo=4, log2_hi=9)
    xr = synth.gaussian(d["total"], seed=2)
    seen = {}
    for rank, s, c, mine, rag, owner, t_max in out:
        assert owner == out[0][5]                 # every rank derived the same map
        for i, y in rag.items():
            assert i not in seen and owner[i] == rank
            seen[i] = y
    assert sorted(seen) == list(range(50))
    for i, y in seen.items():
        o, n = d["offset"][i], d["N"][i]
        assert np.array_equal(y, oracle.fft(xr[o:o + n], inverse=d["direction"][i] > 0))


@pytest.mark.parametrize("batch,world", [(0, 1), (7, 3), (2048, 8), (5, 8)])
def test_shard_rows_partition(batch, world):
    spans = [shard.shard_rows(batch, r, world) for r in range(world)]
    pos = 0
    for s, c in spans:
        assert s == pos
        pos += c
    assert pos == batch
    assert max(c for _, c in spans) - min(c for _, c in spans) <= 1


def test_shard_ragged_balances_work():
    d = synth.ragged_draw(20000, seed=0)
    for world in (2, 4, 8):
        owner = shard.shard_ragged(d["N"], world)
        cost = shard.transform_cost(d["N"])
        loads = np.array([cost[owner == r].sum() for r in range(world)])
        # LPT bound: imbalance below the largest single transform
        assert loads.max() - loads.min() <= cost.max()
        assert np.array_equal(owner, shard.shard_ragged(d["N"], world))  # deterministic
