"""Sharding one Torontonian across processes (one GPU each).

The 2^d prefix chunks are independent and equal in cost (the paper's
balanced partition, Algorithm 1), so rank r of R evaluates the contiguous
chunk range [r 2^d / R, (r+1) 2^d / R) with tor_chunks and the ranks exchange
one fixed-point pair each (256-bit, or 512-bit for the 256-bit fixed-point
tier).  Those partials add exactly (integer addition), so the gathered total
is bit-identical to a single-GPU run.  The exchange is the only collective; it
moves 64 (or 128) bytes per rank.
"""
from __future__ import annotations

import numpy as np



def chunk_range(rank: int, world: int, nchunks: int):
    """Contiguous, disjoint ranges covering [0, nchunks) with sizes differing by at most one."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    return rank * nchunks // world, (rank + 1) * nchunks // world


def limbs_to_ints(limbs):
    """(signed sum, sum_abs) as Python integers modulo 2^(64 L) from 2 L little-endian 64-bit
    limbs (L = 4, or 8 for the 256-bit fixed-point tier)."""
    a = [int(x) & 0xFFFFFFFFFFFFFFFF for x in np.asarray(limbs).ravel()]
    L = len(a) // 2
    lo = sum(a[i] << (64 * i) for i in range(L))
    hi = sum(a[L + i] << (64 * i) for i in range(L))
    return lo, hi


def ints_to_limbs(lo: int, hi: int, limbs: int = 8) -> np.ndarray:
    L = limbs // 2
    mask = (1 << (64 * L)) - 1
    out = np.zeros(limbs, dtype=np.uint64)
    lo &= mask
    hi &= mask
    for i in range(L):
        out[i] = (lo >> (64 * i)) & 0xFFFFFFFFFFFFFFFF
        out[L + i] = (hi >> (64 * i)) & 0xFFFFFFFFFFFFFFFF
    return out


def sum_partials(rows) -> np.ndarray:
    """Exact sum of several partials (rows of an (n, 8) or (n, 16) array) by the library's
    tor_sum_partials; 16 limbs are the 256-bit tier's pairs, 8 any other tier's."""
    rows = np.asarray(rows)
    limbs = rows.shape[-1] if rows.ndim > 1 else rows.size
    if limbs not in (8, 16):
        raise ValueError(f"partials have 8 or 16 limbs, got {limbs}")
    from . import tor
    return tor.sum_partials(rows.reshape(-1, limbs), "fx256" if limbs == 16 else "fp64")


def gather_partials(local, group=None) -> np.ndarray:
    """All-gather each rank's partial (8 limbs, or 16 for the 256-bit tier) and add them exactly
    (any backend)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.from_numpy(np.asarray(local, dtype=np.uint64).view(np.int64).copy()).to(dev)
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    return sum_partials(np.stack([b.cpu().numpy().view(np.uint64) for b in bufs]))


def tor_sharded(ctx, O, chunk_bits: int, prec: str, group=None):
    """This rank's chunk range on its GPU, gathered exactly; returns (TorResult, total limbs)."""
    import torch.distributed as dist
    from . import tor
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, hi = chunk_range(rank, world, 1 << chunk_bits)
    part = ctx.chunks(O, chunk_bits, lo, hi, prec=prec).cpu().numpy().view(np.uint64)
    local = sum_partials(part) if part.size else np.zeros(tor.partial_limbs(prec), dtype=np.uint64)
    total = gather_partials(local, group)
    k = O.shape[0] // 2
    return tor.fixed_to_result([int(x) for x in total], k, prec), total
