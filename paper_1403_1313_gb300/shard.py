"""Multi-worker search: the index-range split of Sec. IV.A across processes.

Static split (sharded_search): each rank searches one contiguous range of the candidate index
space (sizes in proportion to optional weights, e.g. measured throughput), holding its own copy
of the sequences — the paper's per-thread first/last l-mer assignment, one process per GPU.  The
only exchange is one variable-size gather of the accepted codes: counts first, then the codes
padded to the largest count.  Ranges are contiguous and each rank's codes ascend, so
concatenating in rank order gives the globally ascending result.

Dynamic split (dynamic_sharded_search): the skip makes the work of a range depend on the data,
so ranks instead claim fixed-size chunks of the index space one at a time from a shared counter
in the process group's key-value store (an atomic add) until none are left, then gather their
(chunk, codes) pairs; concatenating the chunks in index order gives the ascending result.

Both work over any torch.distributed backend: NCCL with CUDA tensors on GPUs, gloo with CPU
tensors elsewhere.
"""
from __future__ import annotations

import numpy as np


def _rank_search_gpu(seqs, l, d, lo, hi):
    import paper_1403_1313_gb300 as m
    rows = np.ascontiguousarray(seqs, dtype=np.uint8) if isinstance(seqs, np.ndarray) else seqs
    n = len(rows)
    t = rows.shape[1] if isinstance(rows, np.ndarray) else len(rows[0])
    o = m.motif_opts_default()
    o.range_lo, o.range_hi = lo, hi
    plan = m.motif_plan_create(n, t, l, d, o)
    try:
        m.motif_load_seqs(plan, rows)
        return m.motif_search(plan)
    finally:
        m.motif_plan_destroy(plan)


TILE = 1 << 16  # candidates of one tile of the prefix-tiled pass


def rank_range(total: int, rank: int, world: int, tile: int = TILE):
    """This rank's contiguous share [lo, hi) of [0, total): whole tiles where there are at least
    as many tiles as ranks (so that every rank's plan runs the tiled pass, whose tiles start on a
    tile boundary), else an even split of the candidates (motif_shard_range)."""
    import paper_1403_1313_gb300 as m
    tiles = total // tile
    if tile > 1 and tiles >= world and total % tile == 0:
        lo, hi = m.motif_shard_range(tiles, rank, world)
        return lo * tile, hi * tile
    return m.motif_shard_range(total, rank, world)


def gather_codes(codes: np.ndarray, group=None) -> np.ndarray:
    """All-gathers every rank's ascending codes; returns their rank-order concatenation."""
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    world = dist.get_world_size(group)
    cnt = torch.tensor([codes.size], dtype=torch.int64, device=dev)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    width = max(1, max(counts))
    mine = torch.zeros(width, dtype=torch.int64, device=dev)
    if codes.size:
        mine[:codes.size] = torch.from_numpy(codes.astype(np.int64)).to(dev)
    parts = [torch.zeros(width, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    return np.concatenate([p[:c].cpu().numpy().astype(np.uint64) for p, c in zip(parts, counts)])


def gather_codes_device(d_codes, d_count, group=None):
    """All-gathers every rank's ascending device codes (d_codes[0 .. d_count[0]), int64 CUDA
    tensors, d_count holding one count) and returns the rank-order concatenation as a CUDA
    tensor: counts first (read on the host to size the exchange), then the codes padded to the
    largest count.  NCCL backend; the codes stay on the device."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    counts = torch.zeros(world, dtype=torch.int64, device=d_count.device)
    dist.all_gather_into_tensor(counts, d_count.reshape(1), group=group)
    host_counts = counts.tolist()
    width = max(1, max(host_counts))
    mine = d_codes[:width]
    if mine.numel() < width:
        mine = torch.cat([mine, torch.zeros(width - mine.numel(), dtype=mine.dtype,
                                            device=mine.device)])
    parts = torch.empty(world * width, dtype=d_codes.dtype, device=d_codes.device)
    dist.all_gather_into_tensor(parts, mine.contiguous(), group=group)
    parts = parts.view(world, width)
    return torch.cat([parts[r, :c] for r, c in enumerate(host_counts)])


def sharded_search(seqs, l: int, d: int, rank: int, world: int, weights=None, search_fn=None,
                   group=None) -> np.ndarray:
    """Searches this rank's share of [0, 4^l) and gathers the global ascending result.

    search_fn(seqs, l, d, lo, hi) -> ascending codes in [lo, hi); default: the CUDA path."""
    import paper_1403_1313_gb300 as m
    lo, hi = m.motif_shard_range(4 ** l, rank, world, weights)
    fn = search_fn or _rank_search_gpu
    local = np.asarray(fn(seqs, l, d, lo, hi), dtype=np.uint64) if hi > lo else np.zeros(0, np.uint64)
    if world == 1:
        return local
    return gather_codes(local, group)


def dynamic_sharded_search(seqs, l: int, d: int, store, key: str, chunk: int = 1 << 24,
                           search_fn=None, group=None) -> np.ndarray:
    """Searches chunks of [0, 4^l) claimed from `store` (a torch.distributed Store shared by the
    ranks, e.g. dist.distributed_c10d._get_default_store()) under the counter `key` (unique per
    search), then all-gathers and returns the global ascending result on every rank.

    search_fn(seqs, l, d, lo, hi) -> ascending codes in [lo, hi); default: the CUDA path."""
    import torch.distributed as dist
    if chunk < 1:
        raise ValueError("chunk must be positive")
    fn = search_fn or _rank_search_gpu
    space = 4 ** l
    nchunks = (space + chunk - 1) // chunk
    mine = []  # (chunk index, codes)
    while True:
        i = int(store.add(key, 1)) - 1  # claim the next unclaimed chunk
        if i >= nchunks:
            break
        lo = i * chunk
        hi = min(space, lo + chunk)
        mine.append((i, np.asarray(fn(seqs, l, d, lo, hi), dtype=np.uint64)))
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        parts = mine
    else:
        everyone = [None] * dist.get_world_size(group)
        dist.all_gather_object(everyone, mine, group=group)
        parts = [p for r in everyone for p in r]
    parts.sort(key=lambda x: x[0])
    if len(parts) != nchunks or any(i != k for k, (i, _) in enumerate(parts)):
        raise RuntimeError("chunks were lost or claimed twice")
    return np.concatenate([c for _, c in parts]) if parts else np.zeros(0, np.uint64)
