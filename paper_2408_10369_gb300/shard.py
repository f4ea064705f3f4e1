"""Sharding independent units of the method across ranks (one GPU per rank).

The units of BMLP that need no exchange are the query rows of a selective
query batch (Eq. 5 / Algorithm 2: each row v_q R1+ depends only on R1 and its
own sources) and the problems of a grouped batch or corpus (each closure or
composition, Sec. 3.3-3.4, is its own program). They are split across ranks
by predicted cost with the longest-processing-time rule, every rank runs its
share on its own GPU through the library, and one final all-gather puts the
outputs back in their original order on every rank. There is no collective
inside the method's loops.

Every rank computes the same partition from the same costs, so the layout of
the gathered buffer is known everywhere without exchanging sizes. The
collectives are plain ``torch.distributed`` calls and work on NCCL (device
tensors) or gloo (host tensors).
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Sequence

import numpy as np


def lpt_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest processing time first: units in order of decreasing cost (ties
    by index), each to the rank with the least assigned cost so far (ties by
    rank). Returns per rank the unit indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def part_loads(costs: Sequence[float], parts: List[List[int]]) -> List[float]:
    return [float(sum(costs[i] for i in p)) for p in parts]


def _dist():
    import torch.distributed as dist
    return dist


def gather_rows(local, parts: List[List[int]], rank: int, total: int):
    """All-gather row blocks: ``local`` (torch tensor, len(parts[rank]) x w)
    holds this rank's rows, parts[r] the original row index of each row of
    rank r. Returns the total x w tensor in the original order (same device
    and dtype as ``local``). One all_gather of equal-sized padded blocks."""
    import torch
    dist = _dist()
    world = len(parts)
    w = local.shape[1] if local.dim() == 2 else 0
    cap = max(len(p) for p in parts)
    buf = torch.zeros((cap, w), dtype=local.dtype, device=local.device)
    if len(parts[rank]):
        buf[:len(parts[rank])] = local
    if world == 1:
        blocks = [buf]
    else:
        blocks = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(blocks, buf)
    out = torch.empty((total, w), dtype=local.dtype, device=local.device)
    for r, p in enumerate(parts):
        if p:
            out[torch.as_tensor(p, device=local.device, dtype=torch.long)] = blocks[r][:len(p)]
    return out


def gather_outputs(local: list, parts: List[List[int]], rank: int, numel: Sequence[int], device=None):
    """All-gather per-unit outputs of different sizes: ``local`` holds this
    rank's outputs (int64 torch tensors, e.g. packed bit rows, in the order of
    parts[rank]), numel[i] the number of 64-bit words of unit i's output.
    ``device`` is where the collective runs (a CUDA device for NCCL, the CPU
    for gloo; default: that of the first local output, else the CPU).
    Returns a list, indexed by unit, of 1-D int64 tensors of numel[i] words."""
    import torch
    dist = _dist()
    world = len(parts)
    dev = device if device is not None else (local[0].device if local else torch.device("cpu"))
    sizes = [int(sum(numel[i] for i in p)) for p in parts]
    cap = max(max(sizes), 1)
    buf = torch.zeros(cap, dtype=torch.int64, device=dev)
    off = 0
    for i, t in zip(parts[rank], local):
        if t.dtype != torch.int64:
            raise TypeError("outputs are gathered as 64-bit words (packed bit rows)")
        flat = t.reshape(-1)
        assert flat.numel() == numel[i], (i, flat.numel(), numel[i])
        buf[off:off + numel[i]] = flat
        off += numel[i]
    if world == 1:
        blocks = [buf]
    else:
        blocks = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(blocks, buf)
    out: list = [None] * len(numel)
    for r, p in enumerate(parts):
        o = 0
        for i in p:
            out[i] = blocks[r][o:o + numel[i]]
            o += numel[i]
    return out


def share_layout(parts: List[List[int]], rank: int, numel: Sequence[int]):
    """Word offsets of this rank's units inside one contiguous buffer (the
    order of parts[rank]) and the buffer size every rank pads to, so that the
    units' outputs can be written in place and gathered with no copy."""
    sizes = [int(sum(numel[i] for i in p)) for p in parts]
    offs, o = {}, 0
    for i in parts[rank]:
        offs[i] = o
        o += int(numel[i])
    return offs, max(max(sizes), 1)


def gather_flat(buf, parts: List[List[int]], numel: Sequence[int]):
    """All-gather of per-rank contiguous buffers laid out by ``share_layout``
    (``buf``: 1-D int64 tensor of the padded size, this rank's outputs at
    their offsets). Returns a list, indexed by unit, of 1-D views."""
    import torch
    dist = _dist()
    world = len(parts)
    if world == 1:
        blocks = [buf]
    else:
        blocks = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(blocks, buf)
    out: list = [None] * len(numel)
    for r, p in enumerate(parts):
        o = 0
        for i in p:
            out[i] = blocks[r][o:o + int(numel[i])]
            o += int(numel[i])
    return out


def query_costs(src_rows: np.ndarray) -> np.ndarray:
    """Predicted cost of each selective query row: its number of sources
    (each one starts a frontier of its own), at least 1."""
    bits = np.unpackbits(np.ascontiguousarray(src_rows).view(np.uint8), axis=1).sum(1)
    return np.maximum(bits, 1).astype(np.float64)


def problem_costs(ns: Sequence[int], kinds: Sequence[int] = None) -> np.ndarray:
    """Predicted cost of a closure or composition of n constants: n^3
    (squaring work per product on the tensor-core engine; the product count
    grows only as log n), plus a fixed launch cost; compositions count twice."""
    ns = np.asarray(ns, np.float64)
    c = ns ** 3 + 2.0e9
    if kinds is not None:
        c = c * np.where(np.asarray(kinds) == 1, 2.0, 1.0)
    return c


def run_sharded(units: int, costs: Sequence[float], world: int, rank: int,
                execute: Callable[[List[int]], list], numel: Sequence[int], device=None):
    """Partition ``units`` by LPT on ``costs``, run this rank's share with
    ``execute(indices) -> list of int64 output tensors`` and all-gather every
    unit's output (``numel`` 64-bit words each). Returns (outputs by unit,
    the partition)."""
    assert len(costs) == units == len(numel)
    parts = lpt_partition(costs, world)
    local = execute(parts[rank]) if parts[rank] else []
    return gather_outputs(local, parts, rank, numel, device), parts
