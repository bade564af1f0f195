"""Launch-shape autotuner for doa_solve_batch.

Two knobs per M bucket (8, 16, 32, 64), neither of which changes a result bit:
  * scan_pt — the batched scan evaluates tiles of 128 threads x PT consecutive grid points, with
    the PT x M steering phasors of a thread held in registers; PT trades register pressure
    (occupancy) against reuse of each factor element loaded from shared memory;
  * eig_mats — matrices per Jacobi warp; packing several small matrices into one warp gives every
    lane a rotation pair, but leaves fewer warps to hide the FP64 latency of the rotations.
The best values depend on the bucket and on the batch (how many problems, how long the
spectra). The tuner times the scan and eig stages of the caller's own batch for every allowed
value of every occupied bucket (per-stage events of doa_solve_batch), keeps the fastest, and
persists the table as JSON keyed by GPU name, M bucket and size class (decade of the bucket's
problem count and of its mean points per problem), so later runs reuse it without timing.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import doa

CANDIDATES = ((1, 2, 4), (1, 2, 4), (1, 2), (1,))
EIG_CANDIDATES = ((1, 2, 4, 8), (1, 2, 4), (1, 2), (1,))
DEFAULT = (4, 4, 1, 1)


def cache_path() -> str:
    return os.environ.get("DOA_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_2007_14135_gb300", "scan_tune.json"))


def _bucket(M: int) -> int:
    return 0 if M <= 8 else (1 if M <= 16 else (2 if M <= 32 else 3))


def _keys(problems: Sequence[doa.Problem], device, gpu_name: Optional[str] = None) -> Dict[int, str]:
    """Cache key per occupied bucket: GPU, bucket, decades of the problem count and of the mean
    points x algorithms per problem, and the scan kind (ULA, 2-D geometry evaluating its own
    phasors, 2-D geometry reading a steering table shared with other problems, or a mix)."""
    name = (gpu_name or torch.cuda.get_device_name(device)).replace(" ", "_")
    Ls: Dict[int, List[int]] = {}
    kinds: Dict[int, set] = {}
    # the plan shares a steering table among problems with one positions pointer, grid and M
    def tab_key(p):
        return (int(p.geom.pos), p.grid.lo_deg, p.grid.step_deg, int(p.grid.L), p.geom.el_lo_deg,
                p.geom.el_step_deg, int(p.geom.Le), int(p.M))

    uses: Dict[tuple, int] = {}
    for p in problems:
        if p.geom.pos:
            uses[tab_key(p)] = uses.get(tab_key(p), 0) + 1
    for p in problems:
        b = _bucket(p.M)
        geo = bool(p.geom.pos)
        pts = int(p.grid.L) * (int(p.geom.Le) if geo else 1)
        Ls.setdefault(b, []).append(pts * bin(int(p.alg_mask)).count("1"))
        if geo:
            kinds.setdefault(b, set()).add("geotab" if uses[tab_key(p)] >= 2 else "geo")
        else:
            kinds.setdefault(b, set()).add("ula")
    return {b: f"{name}|M{b}|n1e{int(round(math.log10(len(v))))}|L1e{int(round(math.log10(max(1.0, sum(v) / len(v)))))}"
               f"|{'+'.join(sorted(kinds[b]))}"
            for b, v in Ls.items()}


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _stage_ms(plan: doa.BatchPlan, ws: torch.Tensor, status: torch.Tensor, reps: int, stage: int) -> float:
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(doa.BATCH_STAGES + 1)]
    doa.doa_solve_batch(plan, ws, status, stage_events=ev)      # warm-up
    times = []
    for _ in range(reps):
        doa.doa_solve_batch(plan, ws, status, stage_events=ev)
        torch.cuda.synchronize()
        times.append(ev[stage].elapsed_time(ev[stage + 1]))
    return statistics.median(times)


EIG_STAGE, SCAN_STAGE = 2, 3


def tune(problems: Sequence[doa.Problem], device: str = "cuda", reps: int = 3, use_cache: bool = True,
         persist: bool = True, path: Optional[str] = None, log: Optional[list] = None) -> Tuple[List[int], List[int]]:
    """Returns (scan_pt, eig_mats), 4 ints each, for doa.BatchPlan. Empty buckets keep 0 (default)."""
    path = path or cache_path()
    keys = _keys(problems, device)
    table = _load(path) if use_cache else {}
    pt, em = list(DEFAULT), [0, 0, 0, 0]
    todo = []
    for b, key in keys.items():
        if key in table and "eig_mats" in table[key]:
            pt[b] = int(table[key]["pt"])
            em[b] = int(table[key]["eig_mats"])
        else:
            todo.append(b)
    if todo:
        base = doa.BatchPlan(problems, device=device, scan_pt=pt, eig_mats=em)
        em = [v if v else d for v, d in zip(em, base.eig_mats)]
        ws = doa.workspace(base, device=device)
        status = torch.empty(base.nprob, dtype=torch.int32, device=device)
        for b in todo:
            res_pt, res_em = {}, {}
            for v in CANDIDATES[b]:
                trial = list(pt)
                trial[b] = v
                res_pt[v] = _stage_ms(doa.BatchPlan(problems, device=device, scan_pt=trial, eig_mats=em), ws, status,
                                      reps, SCAN_STAGE)
            pt[b] = min(res_pt, key=res_pt.get)
            for v in EIG_CANDIDATES[b]:
                trial = list(em)
                trial[b] = v
                res_em[v] = _stage_ms(doa.BatchPlan(problems, device=device, scan_pt=pt, eig_mats=trial), ws, status,
                                      reps, EIG_STAGE)
            em[b] = min(res_em, key=res_em.get)
            table[keys[b]] = {"pt": pt[b], "scan_ms": {str(k): round(v, 4) for k, v in res_pt.items()},
                              "eig_mats": em[b], "eig_ms": {str(k): round(v, 4) for k, v in res_em.items()}}
            if log is not None:
                log.append({"bucket": b, "key": keys[b], "scan_ms": res_pt, "pt": pt[b], "eig_ms": res_em,
                            "eig_mats": em[b]})
        if persist:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
    return pt, [em[b] if b in keys else 0 for b in range(4)]
