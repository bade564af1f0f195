"""Splitting the work over ranks (one process per GPU).

Two forms, both without a collective on the data path except where the method has a real
exchange step:
  * independent problems (the batched workloads): each rank solves a contiguous range of the
    problems (`shard_range`); only the timing is reduced (`max_over_ranks`);
  * one very long scan (a fine grid, a large array): the angle grid is cut into contiguous
    slices, B is replicated, each rank scans its slice plus one halo point on each side
    (`doa_scan_slice`), summarises its peaks (`doa_slice_peaks`), the summaries are all-gathered
    (a few hundred bytes per rank) and every rank merges them (`doa_merge_slices`, host) into the
    d peaks doa_peaks would return for the whole spectrum.
This module only partitions, marshals and exchanges; the arithmetic runs in libdoa.so.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import doa

SUMMARY_BYTES = ctypes.sizeof(doa.SliceSummary)


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous part [lo, hi) of n units for `rank` of `world` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def slice_bounds(L: int, rank: int, world: int) -> Tuple[int, int, int, int]:
    """(k0, k1, b0, b1): owned grid points [k0, k1) and the computed points [b0, b1) with halo."""
    k0, k1 = shard_range(L, rank, world)
    return k0, k1, max(k0 - 1, 0), min(k1 + 1, L)


def max_over_ranks(x: float, group=None, device=None) -> float:
    """The maximum of x over the ranks of the default (or given) process group."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_summaries(local: torch.Tensor, group=None) -> List[doa.SliceSummary]:
    """All-gathers one summary per rank (a uint8 tensor of SUMMARY_BYTES on the collective's
    device: CUDA for NCCL, CPU for gloo) and returns them in rank order, i.e. slice order."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [doa.slice_summary_from_bytes(local.cpu().numpy().tobytes())]
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(bufs, local, group=group)
    return [doa.slice_summary_from_bytes(b.cpu().numpy().tobytes()) for b in bufs]


def scan_slice_summary(B: torch.Tensor, M: int, K: int, grid: doa.Grid, d: int, rank: int, world: int,
                       stream=None) -> Tuple[torch.Tensor, torch.Tensor, Tuple[int, int, int, int]]:
    """This rank's part of a sliced scan: the spectrum on [b0, b1) and its peak summary (device)."""
    L = int(grid.L)
    k0, k1, b0, b1 = slice_bounds(L, rank, world)
    P = torch.empty(b1 - b0, dtype=torch.float32, device=B.device)
    doa.doa_scan_slice(B, M, K, grid, b0, b1 - b0, P, stream=stream)
    out = torch.zeros(SUMMARY_BYTES, dtype=torch.uint8, device=B.device)
    doa.doa_slice_peaks(P, b0, k0, k1, L, d, out, stream=stream)
    return P, out, (k0, k1, b0, b1)


def sliced_scan_peaks(B: torch.Tensor, M: int, K: int, grid: doa.Grid, d: int, group=None,
                      stream=None) -> Tuple[np.ndarray, np.ndarray, torch.Tensor, Tuple[int, int, int, int]]:
    """One spectrum scanned across the ranks of the group: returns the global peak indices and
    values (identical on every rank), this rank's slice of the spectrum and its bounds."""
    import torch.distributed as dist
    on = dist.is_available() and dist.is_initialized()
    rank = dist.get_rank(group) if on else 0
    world = dist.get_world_size(group) if on else 1
    P, out, bounds = scan_slice_summary(B, M, K, grid, d, rank, world, stream=stream)
    if on and dist.get_backend(group) != "nccl":
        out = out.cpu()
    sums = gather_summaries(out, group=group)
    idx, val = doa.doa_merge_slices(sums, d)
    return idx, val, P, bounds


def merge(summaries: Sequence[doa.SliceSummary], d: int) -> Tuple[np.ndarray, np.ndarray]:
    return doa.doa_merge_slices(summaries, d)
