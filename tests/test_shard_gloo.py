"""Multi-process sharding on CPU: two gloo ranks split the chunk space and
gather their 256-bit partials exactly (the GPU part of each rank is tor_chunks,
covered by the GPU tests)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2009_01177_gb300 import shard


def test_chunk_ranges_partition_the_space():
    for nchunks in (1, 7, 64, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            ranges = [shard.chunk_range(r, world, nchunks) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == nchunks
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [h - l for l, h in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_exact_sum_of_partials_wraps_like_256_bit_integers():
    rng = np.random.default_rng(0)
    vals = [int(rng.integers(-2**62, 2**62)) << 100 for _ in range(5)]
    absv = [abs(v) for v in vals]
    rows = np.stack([shard.ints_to_limbs(v, a) for v, a in zip(vals, absv)])
    lo, hi = shard.limbs_to_ints(shard.sum_partials(rows))
    assert lo == sum(vals) % (1 << 256) and hi == sum(absv)


def _rank_main(rank, world, port, partials, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.chunk_range(rank, world, len(partials))
    local = shard.sum_partials(np.stack(partials[lo:hi])) if hi > lo else np.zeros(len(partials[0]), np.uint64)
    total = shard.gather_partials(local)
    out[rank] = [int(x) for x in total]
    dist.destroy_process_group()


@pytest.mark.parametrize("limbs", [8, 16])   # 256-bit pairs, and the 256-bit tier's 512-bit pairs
def test_two_gloo_ranks_gather_exactly(limbs):
    rng = np.random.default_rng(1)
    # per-chunk partials as the GPU writes them: signed sums and sums of |t|
    vals = [int(rng.integers(-2**60, 2**60)) * (1 << 90) + int(rng.integers(0, 2**40)) for _ in range(37)]
    partials = [shard.ints_to_limbs(v, abs(v), limbs=limbs) for v in vals]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29500 + os.getpid() % 1000
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, partials, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = [out[0], out[1]]
    assert res[0] == res[1]
    lo, hi = shard.limbs_to_ints(np.array(res[0], dtype=np.uint64))
    assert lo == sum(vals) % (1 << (32 * limbs))
    assert hi == sum(abs(v) for v in vals)
