"""Scan tile autotuner for doa_solve_batch.

The batched scan evaluates tiles of 128 threads x PT consecutive grid points, with the PT x M
steering phasors of a thread held in registers. PT trades register pressure (occupancy)
against reuse of each B element loaded from shared memory, and the best value depends on the
M bucket (8, 16, 32, 64) and on how long the spectra are. The tuner times the scan stage of
the caller's own batch for every allowed PT of every occupied bucket (per-stage events of
doa_solve_batch), keeps the fastest, and persists the table as JSON keyed by GPU name, M bucket
and grid-size class (decade of the mean L), so later runs reuse it without timing.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Dict, List, Optional, Sequence

import torch

from . import doa

CANDIDATES = ((1, 2, 4), (1, 2, 4), (1, 2), (1,))
DEFAULT = (4, 2, 1, 1)


def cache_path() -> str:
    return os.environ.get("DOA_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2007_14135_gb300", "scan_tune.json"))


def _bucket(M: int) -> int:
    return 0 if M <= 8 else (1 if M <= 16 else (2 if M <= 32 else 3))


def _keys(problems: Sequence[doa.Problem], device) -> Dict[int, str]:
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    Ls: Dict[int, List[int]] = {}
    for p in problems:
        Ls.setdefault(_bucket(p.M), []).append(int(p.grid.L) * bin(int(p.alg_mask)).count("1"))
    return {b: f"{name}|M{b}|L1e{int(round(math.log10(max(1.0, sum(v) / len(v)))))}" for b, v in Ls.items()}


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _scan_ms(plan: doa.BatchPlan, ws: torch.Tensor, status: torch.Tensor, reps: int) -> float:
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(doa.BATCH_STAGES + 1)]
    doa.doa_solve_batch(plan, ws, status, stage_events=ev)      # warm-up
    times = []
    for _ in range(reps):
        doa.doa_solve_batch(plan, ws, status, stage_events=ev)
        torch.cuda.synchronize()
        times.append(ev[3].elapsed_time(ev[4]))
    return statistics.median(times)


def tune(problems: Sequence[doa.Problem], device: str = "cuda", reps: int = 3, use_cache: bool = True,
         persist: bool = True, path: Optional[str] = None, log: Optional[list] = None) -> List[int]:
    """Returns scan_pt (4 ints) for doa.BatchPlan. Buckets without problems keep the default."""
    path = path or cache_path()
    keys = _keys(problems, device)
    table = _load(path) if use_cache else {}
    choice = list(DEFAULT)
    todo = []
    for b, key in keys.items():
        if key in table:
            choice[b] = int(table[key]["pt"])
        else:
            todo.append(b)
    if todo:
        base = doa.BatchPlan(problems, device=device, scan_pt=choice)
        ws = doa.workspace(base, device=device)
        status = torch.empty(base.nprob, dtype=torch.int32, device=device)
        for b in todo:
            results = {}
            for pt in CANDIDATES[b]:
                trial = list(choice)
                trial[b] = pt
                plan = doa.BatchPlan(problems, device=device, scan_pt=trial)
                results[pt] = _scan_ms(plan, ws, status, reps)
            best = min(results, key=results.get)
            choice[b] = best
            table[keys[b]] = {"pt": best, "scan_ms": {str(k): round(v, 4) for k, v in results.items()}}
            if log is not None:
                log.append({"bucket": b, "key": keys[b], "ms": results, "best": best})
        if persist:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
    return choice
