"""Solving from host memory with the copies hidden behind the solves.

A batch of equally shaped problems (same M, N, d, algorithms and grid) held in pinned host memory
is processed in chunks through two sets of device buffers: while chunk c is solved on the compute
stream, chunk c+1's snapshots are copied in on an upload stream and chunk c-1's peaks and status
are copied out on a download stream. Events order the three streams (a buffer set is refilled only
after its previous solve has read it, and solved into only after its previous results were copied
out), so the host never waits inside `enqueue`. Spectra stay on the device (each set keeps the
last chunk it solved). Every solve is one doa_solve_batch call; this module only orchestrates.
"""
from __future__ import annotations

from typing import List, Optional

import torch

from . import doa


class StreamedBatch:
    def __init__(self, M: int, N: int, d: int, alg_mask: int, grid: doa.Grid, chunk: int, device: str = "cuda",
                 tuning_scan_pt=None, tuning_eig_mats=None, polish: bool = False):
        self.M, self.N, self.d, self.mask, self.grid, self.chunk = M, N, d, alg_mask, grid, chunk
        self.nalg = bin(alg_mask).count("1")
        self.dev = torch.device(device)
        L, D = int(grid.L), max(d, 1)
        self.sets = []
        for _ in range(2):
            s = {
                "X": torch.empty((chunk, M, N), dtype=torch.complex64, device=self.dev),
                "P": torch.empty((chunk, self.nalg, L), dtype=torch.float32, device=self.dev),
                "idx": torch.empty((chunk, self.nalg, D), dtype=torch.int32, device=self.dev),
                "val": torch.empty((chunk, self.nalg, D), dtype=torch.float32, device=self.dev),
                "cnt": torch.empty((chunk, self.nalg), dtype=torch.int32, device=self.dev),
                "status": torch.empty(chunk, dtype=torch.int32, device=self.dev),
            }
            s["probs"] = [doa.make_problem(s["X"][i], d, alg_mask, grid, s["P"][i], s["idx"][i], s["val"][i],
                                           s["cnt"][i], polish=polish) for i in range(chunk)]
            s["plan"] = doa.BatchPlan(s["probs"], device=str(self.dev), scan_pt=tuning_scan_pt,
                                      eig_mats=tuning_eig_mats)
            s["ws"] = doa.workspace(s["plan"], device=str(self.dev))
            self.sets.append(s)
        self.up = torch.cuda.Stream(self.dev)
        self.down = torch.cuda.Stream(self.dev)
        self.compute = torch.cuda.current_stream(self.dev)
        self.read_done = [None, None]     # solve of the set has consumed its snapshots
        self.out_done = [None, None]      # results of the set have been copied out

    def launches_per_chunk(self) -> int:
        return self.sets[0]["plan"].launches()

    def enqueue(self, X_host: torch.Tensor, idx_host: torch.Tensor, val_host: torch.Tensor, cnt_host: torch.Tensor,
                status_host: torch.Tensor) -> torch.cuda.Event:
        """Queues the whole batch (X_host: pinned (B, M, N) complex64, B a multiple of the chunk;
        the outputs: pinned (B, nalg, d), (B, nalg, d), (B, nalg), (B,)). Returns an event that
        completes when the last results have reached the host."""
        B = X_host.shape[0]
        assert B % self.chunk == 0 and X_host.is_pinned()
        last: Optional[torch.cuda.Event] = None
        for c in range(B // self.chunk):
            s = self.sets[c % 2]
            k = c % 2
            lo, hi = c * self.chunk, (c + 1) * self.chunk
            with torch.cuda.stream(self.up):
                if self.read_done[k] is not None:
                    self.up.wait_event(self.read_done[k])
                s["X"].copy_(X_host[lo:hi], non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(self.up)
            self.compute.wait_event(loaded)
            if self.out_done[k] is not None:
                self.compute.wait_event(self.out_done[k])
            doa.doa_solve_batch(s["plan"], s["ws"], s["status"], stream=self.compute)
            solved = torch.cuda.Event()
            solved.record(self.compute)
            self.read_done[k] = solved
            with torch.cuda.stream(self.down):
                self.down.wait_event(solved)
                idx_host[lo:hi].copy_(s["idx"], non_blocking=True)
                val_host[lo:hi].copy_(s["val"], non_blocking=True)
                cnt_host[lo:hi].copy_(s["cnt"], non_blocking=True)
                status_host[lo:hi].copy_(s["status"], non_blocking=True)
                done = torch.cuda.Event()
                done.record(self.down)
            self.out_done[k] = done
            last = done
        return last

    def spectra(self, c: int) -> torch.Tensor:
        """Device spectra of chunk c (valid until that buffer set is solved into again)."""
        return self.sets[c % 2]["P"]
