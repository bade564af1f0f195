#!/usr/bin/env python
"""Throughput of the noise-subspace DOA hot path (PHD, MUSIC, EV, MN) on GB300.

Workload (one step): a batch of independent ULA problems shaped like the paper-density
configuration -- M=16 elements, d=4 sources in U[-60,60] deg with 5 deg separation, SNR U[0,20]
dB, N=4096 complex64 snapshots, scan -90:0.01:90 deg (L=18001) -- each solved with all four
algorithms: covariance, FP64 Jacobi eig + noise subspace, fused FP32 scan, peak picking, all in
the library's CUDA kernels through one doa_solve_batch call. Inputs are seeded synthetic data
(Eq. 1) resident in HBM; per-GPU batch fixed (weak scaling), no collective on the data path.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on a bounded sample
of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scan points/s and DOA solves/s vs plain GPU form at equal peak-index accuracy"
M, D, N_SNAP, STEP, LO = 16, 4, 4096, 0.01, -90.0
ALGS = (0, 1, 2, 3)
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3   # derived FFMA peak, 80.5 TFLOP/s
FP64_PEAK_TFLOPS = 1.25                                          # nominal FP64 rate of the part


def grid_L():
    return int(round(180.0 / STEP)) + 1


def workload_name(batch):
    return (f"paper-density batch: {batch} ULA problems M={M}, d={D}, N={N_SNAP} complex64 snapshots, "
            f"grid -90:{STEP}:90 deg (L={grid_L()}), PHD+MUSIC+EV+MN on each")


# DRAM bytes (read + write) per launch of the dominant kernels, from ncu: the paper-density kernels
# captured at the bench's 4096 problems (one pass, profiles/paper_density_batch_launches.md), the
# circular array from a smaller case scaled to the bench's batch by the problem count (every problem
# is an independent, equal unit; profiles/paper_uca_geometry_scan_ncu.md). Reset an entry to None
# when its kernel changes.
TRAFFIC_BYTES = {
    "scan_shared_kernel<16,4>": 35197696 + 1122881024,        # read + written, 4096-problem launch
    "covariance_tc_batch_kernel<16>": 2148942336 + 15538176,
    "scan_geometry_batch_kernel<8,4>": 2 * (4493312 + 206536704),   # 2048-problem capture x 2
    "scan_geometry_batch_kernel<8,2>": None,
}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# --------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------- oracle leg
_SHM = {}


def _oracle_task(args):
    """One (problem, algorithm) oracle solve; the snapshots come from a shared-memory block."""
    from multiprocessing import shared_memory
    name, shape, i, alg, want_P = args
    if name not in _SHM:
        _SHM.clear()
        shm = shared_memory.SharedMemory(name=name)
        _SHM[name] = (shm, np.ndarray(shape, dtype=np.complex64, buffer=shm.buf))
    X = _SHM[name][1][i]
    import oracle
    r = oracle.solve(X, D, alg, LO, STEP, grid_L())
    return i, alg, r["idx"], (r["P"].astype(np.float32) if want_P else None), r["status"]


def oracle_sample(Xh, S, workers, full=0):
    """Times the FP64 oracle on problems 0..S-1 of Xh x all four algorithms in spawned workers
    (snapshots shared, not copied per task). The first `full` problems also return spectra."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import oracle
    oracle.build()
    X = np.ascontiguousarray(Xh[:S])
    shm = shared_memory.SharedMemory(create=True, size=X.nbytes)
    try:
        np.ndarray(X.shape, dtype=np.complex64, buffer=shm.buf)[:] = X
        tasks = [(shm.name, X.shape, i, a, i < full) for i in range(S) for a in ALGS]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_oracle_task, tasks[:workers], chunksize=1)     # imports + attach, untimed
            t0 = time.perf_counter()
            res = pool.map(_oracle_task, tasks, chunksize=4)
            dt = time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    return res, dt


def parity_summary(res, ig, cg, Pg, Xh, L):
    """Peak agreement of the GPU results (ig, cg: peak indices / counts of the sampled problems;
    Pg: spectra of the first problems) with the oracle's `res`, ties classified, dB and Eq. 4."""
    import oracle
    worst_db, agree, differ = 0.0, 0, []
    eq4 = {a: [] for a in ALGS}
    for i, a, io, Po, sto in res:
        same = list(ig[i, a, :cg[i, a]]) == list(io)
        agree += same
        if not same:
            differ.append((i, a, list(io)))
        if Po is not None and i < len(Pg):
            Pi = Pg[i, a].astype(np.float64)
            worst_db = max(worst_db, float(np.max(np.abs(10 * np.log10(Pi / Po.astype(np.float64))))))
            eq4[a].append(eq4_percent(Pi, Po))
    # a disagreement is a tie within tolerance when the oracle's values at the differing indices
    # are within 1e-4 relative (the FP32 path's error bound near a peak)
    ties = 0
    for i, a, io in differ[:64]:
        Po = oracle.solve(Xh[i], D, a, LO, STEP, L)["P"]
        gi = [int(k) for k in ig[i, a, :cg[i, a]]]
        ks = sorted(set(gi) ^ set(io))
        ties += all(abs(Po[k] - max(Po[k - 1], Po[k + 1])) / Po[k] < 1e-4 or
                    any(abs(Po[k] - Po[j]) / Po[k] < 1e-4 for j in ks if j != k) for k in ks)
    names = {0: "PHD", 1: "MUSIC", 2: "EV", 3: "MN"}
    return {"sampled_solves": len(res), "peak_index_agreement": agree,
            "disagreements_tie_within_1e-4": f"{ties}/{len(differ)}",
            "spectra_compared": sum(len(v) for v in eq4.values()), "max_db_err": worst_db,
            "eq4_percent_max": {names[a]: max(v) for a, v in eq4.items() if v},
            "eq4_percent_mean": {names[a]: statistics.fmean(v) for a, v in eq4.items() if v}}


def eq4_percent(P_meas, P_truth):
    """Eq. 4: 100/N sum |y_meas - y_truth| / |y_truth| over the N spectrum points."""
    P_meas, P_truth = np.asarray(P_meas, np.float64), np.asarray(P_truth, np.float64)
    return float(100.0 * np.mean(np.abs(P_meas - P_truth) / np.abs(P_truth)))


# --------------------------------------------------------------------------------- GPU leg
def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2007_14135_gb300 import synth
    # inputs first (spawned generator processes, before any CUDA call)
    Xh, meta = synth.paper_density_batch_parallel(args.batch, base_seed=20071414 + rank * args.batch)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2007_14135_gb300 import build
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2007_14135_gb300", "libdoa.so")):
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2007_14135_gb300 import doa, shard

    B, L = args.batch, grid_L()
    nalg = len(ALGS)
    dev = torch.device("cuda", local)
    X = torch.from_numpy(Xh).to(dev)
    P = torch.empty((B, nalg, L), dtype=torch.float32, device=dev)
    idx = torch.empty((B, nalg, D), dtype=torch.int32, device=dev)
    val = torch.empty((B, nalg, D), dtype=torch.float32, device=dev)
    cnt = torch.empty((B, nalg), dtype=torch.int32, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    g = doa.grid(LO, STEP, L)
    # peak polish on: the points around every picked peak are re-evaluated in FP64 and the peaks
    # picked again, so near ties between neighbouring grid points fall as in the FP64 spectrum
    probs = [doa.make_problem(X[i], D, 0xF, g, P[i], idx[i], val[i], cnt[i], polish=True) for i in range(B)]
    plan = doa.BatchPlan(probs, device=str(dev))
    ws = doa.workspace(plan, device=str(dev))
    stream = torch.cuda.current_stream(dev)

    launches_per_step = plan.launches()

    def step(events=None):
        doa.doa_solve_batch(plan, ws, status, stage_events=events, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    st = status.cpu().numpy()
    if np.any(st != 0):
        raise RuntimeError(f"device status errors: {np.unique(st, return_counts=True)}")

    nst = doa.BATCH_STAGES + 1
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst)] for _ in range(args.steps)]
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_begin.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = t_begin.elapsed_time(t_end) / args.steps
    stage_ms = [statistics.fmean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps))
                for i in range(doa.BATCH_STAGES)]
    if world > 1:
        ms = shard.max_over_ranks(ms, device=dev)

    # ---- end to end through the C ABI from pinned host buffers: H2D of X, solve, D2H of the peaks
    # Streamed through two buffer sets in chunks of `e2e_chunk` problems: the upload of chunk c+1
    # and the download of chunk c-1's peaks overlap the solve of chunk c (streamed.StreamedBatch).
    from paper_2007_14135_gb300 import streamed
    Xpin = torch.from_numpy(Xh).pin_memory()
    out_idx = torch.empty(idx.shape, dtype=idx.dtype).pin_memory()
    out_val = torch.empty(val.shape, dtype=val.dtype).pin_memory()
    out_cnt = torch.empty(cnt.shape, dtype=cnt.dtype).pin_memory()
    out_st = torch.empty(status.shape, dtype=status.dtype).pin_memory()
    h2d = Xpin.numel() * Xpin.element_size()
    d2h = sum(t.numel() * t.element_size() for t in (out_idx, out_val, out_cnt, out_st))
    chunk = args.e2e_chunk if B % args.e2e_chunk == 0 else B
    sb = streamed.StreamedBatch(M, N_SNAP, D, 0xF, g, chunk, device=str(dev), polish=True)

    for _ in range(max(1, args.warmup)):
        sb.enqueue(Xpin, out_idx, out_val, out_cnt, out_st)
    torch.cuda.synchronize(dev)
    if not np.array_equal(out_idx.numpy(), idx.cpu().numpy()):
        raise RuntimeError("streamed solve disagrees with the resident solve")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    e0.record(stream)
    sb.up.wait_event(e0)
    last = None
    for _ in range(args.steps):
        last = sb.enqueue(Xpin, out_idx, out_val, out_cnt, out_st)
    stream.wait_event(last)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        e2e_ms = shard.max_over_ranks(e2e_ms, device=dev)

    points = B * nalg * L * world
    solves = B * nalg * world
    value = points / (ms / 1e3)

    # ---- measured FMA issue rates (context for the derived ALU peak below)
    fp32_meas = doa.probe_fma_tflops(False, device=str(dev))
    fp64_meas = doa.probe_fma_tflops(True, device=str(dev), iters=1 << 10)

    # ---- roofline of the dominant stage
    peaks_json = load_peaks()
    hbm_peak = peaks_json.get("hbm_gbs", 6800.0)
    # one shared contraction per problem: E_n (M - D columns) read by PHD / MUSIC / EV, plus the
    # MN column; per point 8M + 4 flops per column (complex MACs and |y|^2) and 3 per E_n column
    # for the MUSIC sum and the EV weighted sum (steering generation not counted)
    Kf = (M - D) + 1
    scan_flops = B * L * (Kf * (8 * M + 4) + 3 * (M - D))
    cov_bytes = B * (8 * M * N_SNAP + 16 * M * M)
    stage_info = {}
    names = doa.STAGE_NAMES
    for i, name in enumerate(names):
        stage_info[name] = {"ms": round(stage_ms[i], 4)}
    stage_info["scan"].update(bound="alu", achieved=scan_flops / (stage_ms[3] / 1e3) / 1e12, unit="TFLOP/s",
                              peak=FP32_PEAK_TFLOPS)
    stage_info["covariance"].update(bound="hbm", achieved=cov_bytes / (stage_ms[1] / 1e3) / 1e9, unit="GB/s",
                                    peak=hbm_peak)
    dom = max(range(doa.BATCH_STAGES), key=lambda i: stage_ms[i])
    dname = names[dom]
    if dname == "scan":
        roof = {"bound": "alu", "achieved": round(stage_info["scan"]["achieved"], 3), "peak": round(FP32_PEAK_TFLOPS, 2),
                "unit": "TFLOP/s", "frac": round(stage_info["scan"]["achieved"] / FP32_PEAK_TFLOPS, 4),
                "traffic": TRAFFIC_BYTES.get(f"scan_shared_kernel<16,{plan.scan_pt[1]}>"),
                "kernel": f"scan_shared_kernel<16,{plan.scan_pt[1]}>",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    elif dname == "covariance":
        a = stage_info["covariance"]["achieved"]
        roof = {"bound": "hbm", "achieved": round(a, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(a / hbm_peak, 4), "traffic": TRAFFIC_BYTES.get("covariance_tc_batch_kernel<16>"),
                "kernel": "covariance_tc_batch_kernel<16>",
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": dname, "peak_source": "nominal FP64"}
    for v in stage_info.values():
        if "achieved" in v:
            v["achieved"] = round(v["achieved"], 3)
            v["frac"] = round(v["achieved"] / v["peak"], 4)

    result = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Eq. 1 ULA snapshots, Philox)",
        "config": {"workload": workload_name(B), "batch_per_gpu": B, "M": M, "d": D, "N": N_SNAP, "L": L,
                   "algorithms": ["PHD", "MUSIC", "EV", "MN"], "eig": "double-float Jacobi (FP32 pipe)", "scan": "FP32 FFMA, blocked Horner in z and z^4, grid-shared (32 problems per tile), 4 points per thread", "peaks": "polished (FP64 at peaks +-2)",
                   "l2": f"inputs {Xh.nbytes / 1e9:.2f} GB per step > 129 MB L2 (no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": solves / (ms / 1e3),
        "gpu_launches": launches_per_step * args.steps,
        "stages": stage_info,
        "roofline": roof,
        "alu_peaks_measured": {"fp32_fma_tflops": round(fp32_meas, 2), "fp64_fma_tflops": round(fp64_meas, 3),
                               "how": "doa_probe_fma: 8 independent FMA chains per thread on every SM, best of 5"},
        "e2e": {"value": points / (e2e_ms / 1e3), "unit": "points/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "how": f"pinned host X to device in {B // chunk} chunks of {chunk} problems, uploads and "
                       f"peak downloads overlapped with the solves (two buffer sets, three streams)"},
        "clocks": clk,
    }

    # ---- CPU baseline (oracle) on a bounded sample, rank 0, N = 1; also a parity spot check
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        S = min(args.cpu_sample, B)
        full = min(args.parity_full, S)
        workers = min(os.cpu_count() or 1, 16)
        res, dt = oracle_sample(Xh, S, workers, full=full)
        pts = S * nalg * L
        result["cpu_baseline"] = {"value": pts / dt, "unit": "points/s", "cores": workers, "kind": "oracle",
                                  "sample": f"first {S} problems of the batch x 4 algorithms ({pts} points)",
                                  "seconds": round(dt, 3)}
        result["parity"] = parity_summary(res, idx[:S].cpu().numpy(), cnt[:S].cpu().numpy(),
                                          P[:full].cpu().numpy(), Xh, L)

    # ---- the same batch with the scan on the tensor cores (FP16x3 split operands) and with the
    # FP64 Jacobi: time, stage times and the same parity check against the oracle
    if rank == 0 and world == 1 and not args.no_forms:
        forms = {}
        for name, prec, eprec, polish in (("fp16x3_scan", doa.FP16X3, doa.EIG_DOUBLE_FLOAT, True),
                                          ("fp64_jacobi", doa.FP32, doa.EIG_FP64, True),
                                          ("no_peak_polish", doa.FP32, doa.EIG_DOUBLE_FLOAT, False)):
            fprobs = [doa.make_problem(X[i], D, 0xF, g, P[i], idx[i], val[i], cnt[i], prec=prec, eig_prec=eprec,
                                       polish=polish) for i in range(B)]
            fplan = doa.BatchPlan(fprobs, device=str(dev))
            fws = doa.workspace(fplan, device=str(dev))
            for _ in range(args.warmup):
                doa.doa_solve_batch(fplan, fws, status, stream=stream)
            fev = [[torch.cuda.Event(enable_timing=True) for _ in range(nst)] for _ in range(args.steps)]
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            f0.record(stream)
            for k in range(args.steps):
                doa.doa_solve_batch(fplan, fws, status, stage_events=fev[k], stream=stream)
            f1.record(stream)
            torch.cuda.synchronize(dev)
            fms = f0.elapsed_time(f1) / args.steps
            fst = [statistics.fmean(fev[k][i].elapsed_time(fev[k][i + 1]) for k in range(args.steps))
                   for i in range(doa.BATCH_STAGES)]
            info = {"ms_per_step": fms, "points_per_s": points / (fms / 1e3), "solves_per_s": solves / (fms / 1e3),
                    "stages_ms": {n: round(v, 4) for n, v in zip(doa.STAGE_NAMES, fst)},
                    "status_ok": bool(np.all(status.cpu().numpy() == 0))}
            if "parity" in result:
                S = min(args.cpu_sample, B)
                full = min(args.parity_full, S)
                info["parity"] = parity_summary(res, idx[:S].cpu().numpy(), cnt[:S].cpu().numpy(),
                                                P[:full].cpu().numpy(), Xh, L)
            forms[name] = info
            del fplan, fws, fprobs
        result["forms"] = forms
        result["refinement"] = refinement_form(args, doa, torch, X, P, idx, val, cnt, status, g, meta, stream, dev,
                                               points, solves)
        result["root_and_order"] = root_order_form(args, doa, torch, X, P, idx, val, cnt, status, g, meta, stream,
                                                   dev, points, solves)
        if not args.no_workload_forms:
            result["workloads"] = workload_forms(args)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def workload_forms(args):
    """The other configurations as compact forms of the default line, each with its own parity
    against the oracle and its roofline: the uneven batch (1024 problems, CUDA graph, autotuned),
    the large array (32 replicas, FP32 / FP16x3 contractions, double-float and FP64 Jacobi), the
    learned proposal (a smaller training set, 65536 test instances, judged) and the paper's UCA
    scenario. Each runs with 3 timed steps after 3 warm-up steps."""
    import copy
    base = {"steps": 3, "warmup": 3, "cpu_sample": 256, "parity_full": 16, "no_cpu_baseline": False}
    specs = (("uneven_batch", run_uneven, {"batch": 1024}),
             ("large_array", run_large_array, {"batch": 32, "la_forms": "fp32,fp16x3,fp16x3_fp64_jacobi"}),
             ("learned_proposal", run_learned, {"batch": 65536, "train": 1 << 18, "epochs": 16, "lr_decay": 0.85}),
             ("paper_uca", run_uca, {"batch": 4096, "uca_rows": 90}))
    drop = ("autotune", "clocks", "table10", "single")
    out = {}
    for name, fn, kw in specs:
        a = copy.copy(args)
        a.__dict__.update(base)
        a.__dict__.update(kw)
        t0 = time.perf_counter()
        try:
            r = fn(a, emit=False)
        except Exception as e:   # a failed form is reported, not hidden
            out[name] = {"error": repr(e)[:400]}
            continue
        r = {k: v for k, v in r.items() if k not in drop}
        r["wall_s"] = round(time.perf_counter() - t0, 1)
        out[name] = r
    return out


def refinement_form(args, doa, torch, X, P, idx, val, cnt, status, g, meta, stream, dev, points, solves):
    """The same batch with sub-grid refinement (FP64 Newton next to every picked peak): step time,
    and the error against the true angles of the grid estimates and of the refined ones (problems
    whose algorithm found all d peaks; peaks and truths paired in sorted order)."""
    B = X.shape[0]
    ang = torch.full((B, len(ALGS), D), float("nan"), dtype=torch.float64, device=dev)
    rprobs = [doa.make_problem(X[i], D, 0xF, g, P[i], idx[i], val[i], cnt[i], polish=True, peak_angle=ang[i])
              for i in range(B)]
    rplan = doa.BatchPlan(rprobs, device=str(dev))
    rws = doa.workspace(rplan, device=str(dev))
    for _ in range(args.warmup):
        doa.doa_solve_batch(rplan, rws, status, stream=stream)
    nst = doa.BATCH_STAGES + 1
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    r0.record(stream)
    for _ in range(args.steps):
        doa.doa_solve_batch(rplan, rws, status, stream=stream)
    r1.record(stream)
    torch.cuda.synchronize(dev)
    rms = r0.elapsed_time(r1) / args.steps
    ih, ch, ah = idx.cpu().numpy(), cnt.cpu().numpy(), ang.cpu().numpy()
    names = {0: "PHD", 1: "MUSIC", 2: "EV", 3: "MN"}
    err = {}
    for a in ALGS:
        eg, er = [], []
        for i in range(B):
            if ch[i, a] != D:
                continue
            truth = np.sort(meta[i].angles)
            eg.append(np.sort(LO + ih[i, a] * STEP) - truth)
            er.append(np.sort(ah[i, a]) - truth)
        eg, er = np.concatenate(eg), np.concatenate(er)
        err[names[a]] = {"solves": len(eg) // D, "rmse_grid_deg": float(np.sqrt(np.mean(eg ** 2))),
                         "rmse_refined_deg": float(np.sqrt(np.mean(er ** 2))),
                         "max_abs_refined_deg": float(np.max(np.abs(er)))}
    del rplan, rws, rprobs
    return {"ms_per_step": rms, "points_per_s": points / (rms / 1e3), "solves_per_s": solves / (rms / 1e3),
            "status_ok": bool(np.all(status.cpu().numpy() == 0)), "error_vs_truth": err,
            "how": "FP64 bracketed Newton on den' next to every peak (all four algorithms), after peak polish"}


def root_order_form(args, doa, torch, X, P, idx, val, cnt, status, g, meta, stream, dev, points, solves):
    """The same batch with the root form of the scan (Aberth roots of each algorithm's polynomial) and
    the MDL / AIC source-count estimates: step time, the root estimates' error against the true
    angles beside the grid peaks', and how often each criterion returns the true d."""
    B = X.shape[0]
    ra = torch.full((B, len(ALGS), D), float("nan"), dtype=torch.float64, device=dev)
    oe = torch.full((B, 2), -1, dtype=torch.int32, device=dev)
    probs = [doa.make_problem(X[i], D, 0xF, g, P[i], idx[i], val[i], cnt[i], polish=True, root_angle=ra[i],
                              order_est=oe[i]) for i in range(B)]
    plan = doa.BatchPlan(probs, device=str(dev))
    ws = doa.workspace(plan, device=str(dev))
    for _ in range(args.warmup):
        doa.doa_solve_batch(plan, ws, status, stream=stream)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    r0.record(stream)
    for _ in range(args.steps):
        doa.doa_solve_batch(plan, ws, status, stream=stream)
    r1.record(stream)
    torch.cuda.synchronize(dev)
    ms = r0.elapsed_time(r1) / args.steps
    ih, ch, rh, oh = idx.cpu().numpy(), cnt.cpu().numpy(), ra.cpu().numpy(), oe.cpu().numpy()
    names = {0: "PHD", 1: "MUSIC", 2: "EV", 3: "MN"}
    err = {}
    for a in ALGS:
        eg, er = [], []
        for i in range(B):
            truth = np.sort(meta[i].angles)
            if ch[i, a] == D:
                eg.append(np.sort(LO + ih[i, a] * STEP) - truth)
            if np.all(np.isfinite(rh[i, a])):
                er.append(np.sort(rh[i, a]) - truth)
        eg, er = np.concatenate(eg), np.concatenate(er)
        err[names[a]] = {"rmse_grid_deg": float(np.sqrt(np.mean(eg ** 2))),
                         "rmse_root_deg": float(np.sqrt(np.mean(er ** 2))), "root_solves": len(er) // D}
    st = status.cpu().numpy()
    del plan, ws, probs
    return {"ms_per_step": ms, "points_per_s": points / (ms / 1e3), "solves_per_s": solves / (ms / 1e3),
            "status_ok": int(np.sum(st == 0)), "error_vs_truth": err,
            "order_estimates": {"mdl_equals_d": float(np.mean(oh[:, 0] == D)), "aic_equals_d": float(np.mean(oh[:, 1] == D)),
                                "d": D},
            "how": "Aberth-Ehrlich roots (FP64) of each algorithm's scan polynomial; MDL / AIC from the sorted "
                   "eigenvalues after the Jacobi sweeps"}


def run_uneven(args, emit=True):
    """Uneven batch: 4096 problems, M in {8,12,16,32}, d in U{1..M/2}, N in U{256..8192}, grid step in
    {0.1, 0.01, 0.001} deg, one algorithm each, solved by one doa_solve_batch replayed from a CUDA
    graph, with scan tiles from the autotuner."""
    import torch
    from paper_2007_14135_gb300 import synth
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    specs = synth.uneven_specs(args.batch, seed=20071415 + rank)
    buf, offs = synth.uneven_batch_parallel(specs)
    torch.cuda.set_device(local)
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2007_14135_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2007_14135_gb300 import autotune, doa, shard
    dev = torch.device("cuda", local)
    Xd = torch.from_numpy(buf).to(dev)
    Ls = np.array([s.L for s in specs], dtype=np.int64)
    p_off = np.concatenate([[0], np.cumsum(Ls)[:-1]])
    P = torch.empty(int(Ls.sum()), dtype=torch.float32, device=dev)
    dmax = max(s.d for s in specs)
    idx = torch.empty((len(specs), dmax), dtype=torch.int32, device=dev)
    val = torch.empty((len(specs), dmax), dtype=torch.float32, device=dev)
    cnt = torch.empty(len(specs), dtype=torch.int32, device=dev)
    probs = []
    for i, s in enumerate(specs):
        X = Xd[int(offs[i]):int(offs[i]) + s.M * s.N].view(s.M, s.N)
        prec = doa.FP16X3 if (args.tc_min_m and s.M >= args.tc_min_m and s.M <= 32) else doa.FP32
        probs.append(doa.make_problem(X, s.d, 1 << s.alg, doa.grid(LO, s.step, s.L), P[int(p_off[i]):int(p_off[i] + s.L)],
                                      idx[i], val[i], cnt[i:i + 1], prec=prec))
    tune_log = []
    scan_pt, eig_mats = (autotune.tune(probs, device=str(dev), log=tune_log) if not args.no_tune
                         else (list(autotune.DEFAULT), [0, 0, 0, 0]))
    plan = doa.BatchPlan(probs, device=str(dev), scan_pt=scan_pt, eig_mats=eig_mats)
    ws = doa.workspace(plan, device=str(dev))
    status = torch.empty(len(specs), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # per-stage breakdown from instrumented (non-graph) solves
    nst = doa.BATCH_STAGES + 1
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst)] for _ in range(3)]
    for k in range(3):
        doa.doa_solve_batch(plan, ws, status, stage_events=evs[k], stream=stream)
    torch.cuda.synchronize(dev)
    st = status.cpu().numpy()
    if np.any(st != 0):
        raise RuntimeError(f"device status errors: {np.unique(st, return_counts=True)}")
    stage_ms = [statistics.fmean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(1, 3))
                for i in range(doa.BATCH_STAGES)]
    # graph capture of the whole solve, replayed in the timed region
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        doa.doa_solve_batch(plan, ws, status, stream=side)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        doa.doa_solve_batch(plan, ws, status)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    if world > 1:
        ms = shard.max_over_ranks(ms, device=dev)
    points = int(Ls.sum()) * world
    # end to end: pinned H2D of all snapshots + graph + D2H of peaks and status
    Xpin = torch.from_numpy(buf).pin_memory()
    outs = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (idx, val, cnt, status)]
    h2d = Xpin.numel() * Xpin.element_size()
    d2h = sum(t.numel() * t.element_size() for t in outs)

    def e2e_step():
        Xd.copy_(Xpin, non_blocking=True)
        graph.replay()
        for o, t in zip(outs, (idx, val, cnt, status)):
            o.copy_(t, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / args.steps
    # FP32 ALU roofline of the scan stage: per problem L K (8M + 4) flops for its K factor columns
    # (one algorithm each: K = 1 for PHD and MN, M - d for MUSIC and EV)
    scan_flops = sum(s.L * (1 if s.alg in (0, 3) else s.M - s.d) * (8 * s.M + 4) for s in specs)
    a_tf = scan_flops / (stage_ms[3] / 1e3) / 1e12
    scan_roof = {"bound": "alu", "achieved": round(a_tf, 3), "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
                 "frac": round(a_tf / FP32_PEAK_TFLOPS, 4), "traffic": None, "kernel": "scan stage (all buckets)",
                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}
    result = {
        "metric": METRIC, "value": points / (ms / 1e3), "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded Eq. 1 ULA snapshots, Philox)",
        "config": {"workload": f"uneven batch: {len(specs)} problems, M in {{8,12,16,32}}, d in U{{1..M/2}}, "
                               f"N in U{{256..8192}}, step in {{0.1,0.01,0.001}} deg, one algorithm each",
                   "batch_per_gpu": len(specs), "points_per_gpu": int(Ls.sum()), "graph": True,
                   "scan_pt": scan_pt, "eig_mats": plan.eig_mats,
                   "tensor_scan": (f"FP16x3 for M >= {args.tc_min_m}" if args.tc_min_m else "none"),
                   "l2": f"inputs {buf.nbytes / 1e9:.2f} GB > 129 MB L2 (no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": len(specs) * world / (ms / 1e3),
        "gpu_launches": plan.launches() * args.steps,
        "stages": {n: {"ms": round(v, 4)} for n, v in zip(doa.STAGE_NAMES, stage_ms)},
        "roofline": scan_roof,
        "autotune": tune_log,
        "e2e": {"value": points / (e2e_ms / 1e3), "unit": "points/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # stratified sample: the first problem of every (M, algorithm, grid) class
        seen, pick = set(), []
        for i, s in enumerate(specs):
            key = (s.M, s.alg, s.L)
            if key not in seen:
                seen.add(key)
                pick.append(i)
        tasks = [(buf[int(offs[i]):int(offs[i]) + specs[i].M * specs[i].N].reshape(specs[i].M, specs[i].N),
                  specs[i].d, specs[i].alg, specs[i].step, specs[i].L) for i in pick]
        res, dt = oracle_tasks(tasks, min(os.cpu_count() or 1, 16))
        pts = int(sum(specs[i].L for i in pick))
        result["cpu_baseline"] = {"value": pts / dt, "unit": "points/s", "cores": min(os.cpu_count() or 1, 16),
                                  "kind": "oracle", "seconds": round(dt, 3),
                                  "sample": f"{len(pick)} problems, one per (M, algorithm, grid) class ({pts} points)"}
        Ph = P.cpu().numpy()
        ih, ch = idx.cpu().numpy(), cnt.cpu().numpy()
        worst, agree = 0.0, 0
        for i, (io, Po, sto) in zip(pick, res):
            Pg = Ph[int(p_off[i]):int(p_off[i] + specs[i].L)].astype(np.float64)
            worst = max(worst, float(np.max(np.abs(10 * np.log10(Pg / Po)))))
            agree += list(ih[i, :ch[i]]) == list(io)
        result["parity"] = {"sampled_solves": len(pick), "peak_index_agreement": agree, "max_db_err": worst}
    if rank == 0 and emit:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return result


def run_large_array(args, emit=True):
    """Large array: M=64, d=8 (1 deg separation), N=16384, 360001-point grid (0.0005 deg), MUSIC.
    Each form (FP32 plain, one BF16 product, BF16x3 and FP16x3 split) runs covariance, FP64
    Jacobi, scan and peaks for `batch` replicas (spread over streams); the scan stage is also
    timed alone. Accuracy: replicas 0..3 against the oracle's full spectrum and peaks."""
    import torch
    from paper_2007_14135_gb300 import build, synth
    reps = args.batch
    insts = [synth.large_array(i) for i in range(reps)]
    torch.cuda.set_device(0)
    build.build()
    from paper_2007_14135_gb300 import doa
    dev = torch.device("cuda", 0)
    M, d, L = insts[0].M, insts[0].d, insts[0].L
    g = doa.grid(insts[0].lo, insts[0].step, L)
    X = [torch.from_numpy(i.X).to(dev) for i in insts]
    R = [torch.empty((M, M), dtype=torch.complex128, device=dev) for _ in insts]
    B = [torch.zeros(M * M, dtype=torch.complex128, device=dev) for _ in insts]
    info = torch.zeros(reps, dtype=torch.int32, device=dev)
    P = torch.empty((reps, L), dtype=torch.float32, device=dev)
    idx = torch.zeros((reps, d), dtype=torch.int32, device=dev)
    val = torch.zeros((reps, d), dtype=torch.float32, device=dev)
    cnt = torch.zeros(reps, dtype=torch.int32, device=dev)
    K = M - d
    nstreams = min(reps, 32)
    streams = [torch.cuda.Stream(dev) for _ in range(nstreams)]
    main = torch.cuda.current_stream(dev)
    # (contraction precision, Jacobi arithmetic); the double-float Jacobi spreads each M=64 matrix
    # over a four-CTA cluster on the FP32 pipe, the FP64 form (one CTA) is kept beside it
    forms = {"fp32": (doa.FP32, doa.EIG_DOUBLE_FLOAT), "bf16": (doa.BF16, doa.EIG_DOUBLE_FLOAT),
             "bf16x3": (doa.BF16X3, doa.EIG_DOUBLE_FLOAT), "fp16x3": (doa.FP16X3, doa.EIG_DOUBLE_FLOAT),
             "fp16x3_fp64_jacobi": (doa.FP16X3, doa.EIG_FP64)}
    if args.la_forms:
        forms = {k: v for k, v in forms.items() if k in args.la_forms.split(",")}
    stage_names = ("covariance", "eig_noise_subspace", "scan", "peaks")

    def solve(form, events=None):
        # one stage at a time over all replicas, the replicas of a stage spread over the streams
        # (the Jacobi of one replica per four-SM cluster; the tensor kernels fill the GPU)
        prec, eprec = form
        calls = (lambda r, st: doa.doa_covariance(X[r], R64=R[r], prec=prec, stream=st),
                 lambda r, st: doa.doa_noise_subspace_prec(R[r], d, doa.MUSIC, eprec, B[r], info[r:r + 1],
                                                           stream=st),
                 lambda r, st: doa.doa_scan(B[r], M, K, g, P[r], prec=prec, stream=st),
                 lambda r, st: doa.doa_peaks(P[r], d, idx[r], val[r], cnt[r:r + 1], stream=st))
        for si, call in enumerate(calls):
            if events is not None:
                events[si].record(main)
            for st in streams:
                st.wait_stream(main)
            for r in range(reps):
                call(r, streams[r % nstreams])
            for st in streams:
                main.wait_stream(st)
        if events is not None:
            events[len(calls)].record(main)

    def scans(prec):
        for r in range(reps):
            doa.doa_scan(B[r], M, K, g, P[r], prec=prec)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for _ in range(steps):
            fn()
        e1.record(main)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    nchk = min(4, reps)
    ref = oracle_tasks([(insts[i].X, d, doa.MUSIC, insts[i].step, L) for i in range(nchk)],
                       min(os.cpu_count() or 1, 16))[0] if not args.no_cpu_baseline else None
    out = {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, form in forms.items():
        prec = form[0]
        ms_solve = timed(lambda: solve(form), args.steps)
        st_info = info.cpu().numpy()
        sev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        solve(form, sev)
        torch.cuda.synchronize(dev)
        stage_ms = {n: round(sev[i].elapsed_time(sev[i + 1]), 3) for i, n in enumerate(stage_names)}
        ms_scan = timed(lambda: scans(prec), args.steps)
        solve(form)
        torch.cuda.synchronize(dev)
        res = {"ms_per_step": ms_solve, "solves_per_s": reps / (ms_solve / 1e3), "stages_ms": stage_ms,
               "scan_ms": ms_scan, "scan_points_per_s": reps * L / (ms_scan / 1e3),
               "scan_tflops_algorithmic": reps * L * K * (8 * M + 4) / (ms_scan / 1e3) / 1e12,
               "eig": "fp64" if form[1] == doa.EIG_FP64 else "double-float", "eig_status_ok": bool(np.all(st_info > 0))}
        if ref is not None:
            Pg = P[:nchk].cpu().numpy().astype(np.float64)
            ig, cg = idx[:nchk].cpu().numpy(), cnt[:nchk].cpu().numpy()
            res["max_db_err"] = float(max(np.max(np.abs(10 * np.log10(Pg[i] / ref[i][1]))) for i in range(nchk)))
            res["peak_index_agreement"] = f"{sum(list(ig[i, :cg[i]]) == list(ref[i][0]) for i in range(nchk))}/{nchk}"
        out[name] = res
    clk = clocks.stop()
    head = "fp16x3" if "fp16x3" in out else next(iter(out))
    fp = out[head]
    # tensor roofline of the split-operand scan: three real GEMMs of the steering block (L x 2M)
    # against the real embedding of B (2M x 2K), 8 L M K flops each
    peaks_json = load_peaks()
    bf16_peak = peaks_json.get("bf16_tflops", 1899.9)
    tc_tf = 3 * 8 * reps * L * M * K / (fp["scan_ms"] / 1e3) / 1e12
    roof = ({"bound": "tensor", "achieved": round(tc_tf, 2), "peak": bf16_peak, "unit": "TFLOP/s",
             "frac": round(tc_tf / bf16_peak, 4), "traffic": None, "kernel": "scan_tc_kernel (FP16x3)",
             "peak_source": "measured bf16 burst (MEASURED_PEAKS.json); FP16 runs at the BF16 rate"}
            if head == "fp16x3" else None)
    result = {
        "metric": METRIC, "value": fp["scan_points_per_s"], "unit": "points/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": fp["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": head, "data": "synthetic (seeded Eq. 1 ULA snapshots, Philox)",
        "config": {"workload": f"large array: {reps} replicas of M=64, d=8 (1 deg separation), N=16384, "
                               f"grid -90:0.0005:90 (L=360001), MUSIC", "replicas": reps,
                   "value_is": f"{head} scan points/s (scan stage alone)"},
        "forms": out, "roofline": roof, "clocks": clk,
    }
    if emit:
        print(json.dumps(result), flush=True)
    return result


def run_learned(args, emit=True):
    """Learned proposal: train the network on 1M method-generated instances (M=16, d in U{1..6},
    SNR U[-5,20] dB, angles U[-80,80] with 3 deg separation, N=2048), then solve a batch of
    test instances two ways at the 0.001 deg resolution: covariance + Jacobi + network + windowed
    fine scan + full-grid fallback, against the plain full-grid method (the arbiter). Step times
    are wall clock around synchronised GPU work (the pipeline reads the fallback flags back)."""
    import torch
    from paper_2007_14135_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    from paper_2007_14135_gb300 import doa, proposal
    t0 = time.perf_counter()
    feats, labels = proposal.make_training_set(args.train, seed=proposal.TRAIN_SEED)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    net = doa.Mlp(seed=1)
    t0 = time.perf_counter()
    hist = proposal.train(net, feats, labels, epochs=args.epochs, batch=4096, lr=2e-3, decay=args.lr_decay)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    steps_train = args.epochs * (args.train // 4096)
    del feats, labels
    ts = proposal.TestSet(args.batch)
    fg = proposal.fine_grid()

    def learned():
        ts.solve()
        return proposal.infer(net, ts.solved(), extra=1)

    def plain():
        ts.solve()
        return proposal.full_grid(ts.solved())

    for _ in range(max(1, args.warmup)):
        inf = learned()
        ji, jc, _ = plain()
    clocks = ClockSampler(0)
    clocks.start()
    tl, tp = [], []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        a = time.perf_counter()
        inf = learned()
        torch.cuda.synchronize()
        tl.append(time.perf_counter() - a)
        a = time.perf_counter()
        ji, jc, _ = plain()
        torch.cuda.synchronize()
        tp.append(time.perf_counter() - a)
    clk = clocks.stop()
    n = ts.n
    same = np.array([list(inf.idx[i, :inf.count[i]]) == list(ji[i, :jc[i]]) for i in range(n)])
    ms_l, ms_p = 1e3 * statistics.median(tl), 1e3 * statistics.median(tp)
    full_pts = n * fg.L
    result = {
        "metric": METRIC, "value": full_pts / (ms_l / 1e3), "unit": "points/s (effective: full-grid points covered)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_l, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 scan, bf16 network", "data": "synthetic (GPU Philox, Eq. 1)",
        "config": {"workload": f"learned proposal: {n} test instances M=16, d in U{{1..6}}, SNR U[-5,20] dB, "
                               f"angles U[-80,80] sep 3 deg, N=2048, 0.001 deg grid (L=180001), MUSIC; +-2 deg "
                               f"windows (d+1 proposals), judge on the 0.1 deg full-grid spectrum, full-grid "
                               f"fallback", "train_instances": args.train,
                   "epochs": args.epochs},
        "solves_per_s": n / (ms_l / 1e3),
        "plain": {"ms_per_step": ms_p, "points_per_s": full_pts / (ms_p / 1e3), "solves_per_s": n / (ms_p / 1e3)},
        "speedup_vs_plain": ms_p / ms_l,
        "agreement_with_full_grid": float(same.mean()), "fallback_rate": float(inf.fallback.mean()),
        "judge_fallback_rate": float(inf.judged.mean()),
        "points_evaluated_ratio": full_pts / inf.points,
        "training": {"data_s": t_gen, "train_s": t_train, "adam_steps": steps_train,
                     "loss_first_last": [hist[0], hist[-1]]},
        "clocks": clk,
    }
    if emit:
        print(json.dumps(result), flush=True)
    return result


def run_uca(args, emit=True):
    """The paper's own scenario (Sec. 4.2, Tables 8 and 10): a batch of 8-element uniform circular
    arrays (radius 10 m at 15 MHz), two uncorrelated sources at 15 dB SNR, N=1024 snapshots, MUSIC
    over azimuth 0:1:359 x elevation angle 1:1:90 (32 400 points) with the steering vector of Eq. 2
    as printed, solved by one doa_solve_batch replayed from a CUDA graph. Also times one solve at a
    time (the paper's single-problem latency, with its host copies) and the four scan sizes of
    Table 10 (360 x 1, 30, 60, 90)."""
    import torch
    from paper_2007_14135_gb300 import synth
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    B, Le = args.batch, args.uca_rows
    insts = [synth.paper_uca(rank * B + i, Le=Le) for i in range(B)]
    Xh = np.stack([g.X for g in insts])
    g0 = insts[0]
    torch.cuda.set_device(local)
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2007_14135_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2007_14135_gb300 import autotune, doa, shard
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    Mu, du = g0.M, g0.d
    tune_log = []
    pos = torch.from_numpy(np.ascontiguousarray(g0.pos)).to(dev)
    az = doa.grid(g0.az_lo, g0.az_step, g0.La)

    def build_batch(X, rows, tuning=None):
        npts = g0.La * rows
        P = torch.empty((X.shape[0], npts), dtype=torch.float32, device=dev)
        idx = torch.empty((X.shape[0], du), dtype=torch.int32, device=dev)
        val = torch.empty((X.shape[0], du), dtype=torch.float32, device=dev)
        cnt = torch.empty(X.shape[0], dtype=torch.int32, device=dev)
        geom = doa.geometry(pos, float(91 - rows), 1.0, rows, True)
        probs = [doa.make_problem(X[i], du, 1 << doa.MUSIC, az, P[i], idx[i], val[i], cnt[i:i + 1], geom=geom)
                 for i in range(X.shape[0])]
        if tuning == "tune":
            tuning = autotune.tune(probs, device=str(dev), log=tune_log)
        sp, em = tuning if tuning else (None, None)
        plan = doa.BatchPlan(probs, device=str(dev), scan_pt=sp, eig_mats=em)
        ws = doa.workspace(plan, device=str(dev))
        status = torch.empty(X.shape[0], dtype=torch.int32, device=dev)
        return dict(P=P, idx=idx, val=val, cnt=cnt, plan=plan, ws=ws, status=status, probs=probs)

    def capture(bt):
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            doa.doa_solve_batch(bt["plan"], bt["ws"], bt["status"], stream=side)
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            doa.doa_solve_batch(bt["plan"], bt["ws"], bt["status"])
        return graph

    def time_graph(graph, steps):
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    X = torch.from_numpy(Xh).to(dev)
    if args.scan_pt:
        fixed = ([int(v) for v in args.scan_pt.split(",")], None)
        bt = build_batch(X, Le, fixed)
    else:
        bt = build_batch(X, Le, None if args.no_tune else "tune")
    nst = doa.BATCH_STAGES + 1
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nst)] for _ in range(3)]
    for k in range(3):
        doa.doa_solve_batch(bt["plan"], bt["ws"], bt["status"], stage_events=evs[k], stream=stream)
    torch.cuda.synchronize(dev)
    st = bt["status"].cpu().numpy()
    if np.any(st != 0):
        raise RuntimeError(f"device status errors: {np.unique(st, return_counts=True)}")
    stage_ms = [statistics.fmean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(1, 3))
                for i in range(doa.BATCH_STAGES)]
    graph = capture(bt)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    if world > 1:
        ms = shard.max_over_ranks(ms, device=dev)
    npts = g0.La * Le
    points = B * npts * world
    # end to end: pinned H2D of the snapshots, the graph, D2H of the peaks and status
    Xpin = torch.from_numpy(Xh).pin_memory()
    outs = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (bt["idx"], bt["val"], bt["cnt"], bt["status"])]
    h2d = Xpin.numel() * Xpin.element_size()
    d2h = sum(t.numel() * t.element_size() for t in outs)

    def e2e_step():
        X.copy_(Xpin, non_blocking=True)
        graph.replay()
        for o, t in zip(outs, (bt["idx"], bt["val"], bt["cnt"], bt["status"])):
            o.copy_(t, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / args.steps

    # one problem at a time: the paper's per-solve latency (Table 10 includes its host copies)
    single = {}
    if rank == 0:
        X1 = torch.from_numpy(Xh[:1].copy()).to(dev)
        b1 = build_batch(X1, Le)
        g1 = capture(b1)
        lat = time_graph(g1, 200)
        X1pin = torch.from_numpy(Xh[:1].copy()).pin_memory()
        o1 = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (b1["idx"], b1["val"], b1["cnt"])]
        for _ in range(args.warmup):
            X1.copy_(X1pin, non_blocking=True)
            g1.replay()
        wall = []
        for _ in range(200):
            torch.cuda.synchronize(dev)
            a = time.perf_counter()
            X1.copy_(X1pin, non_blocking=True)
            g1.replay()
            for o, t in zip(o1, (b1["idx"], b1["val"], b1["cnt"])):
                o.copy_(t, non_blocking=True)
            torch.cuda.synchronize(dev)
            wall.append(time.perf_counter() - a)
        sev = [[torch.cuda.Event(enable_timing=True) for _ in range(nst)] for _ in range(20)]
        for k in range(20):
            doa.doa_solve_batch(b1["plan"], b1["ws"], b1["status"], stage_events=sev[k], stream=stream)
        torch.cuda.synchronize(dev)
        sstage = {n: round(statistics.median(sev[k][i].elapsed_time(sev[k][i + 1]) for k in range(5, 20)), 4)
                  for i, n in enumerate(doa.STAGE_NAMES)}
        single = {"device_ms": lat, "host_to_host_ms_median": 1e3 * statistics.median(wall),
                  "stages_ms_eager": sstage,
                  "paper_table10_ms": {"GTX 1660 Ti (Config-1)": 0.924, "GTX 1050 (Config-2)": 1.447},
                  "launches": b1["plan"].launches()}
        del b1, g1
    # sub-grid refinement of the 2-D peaks (damped Newton in azimuth and elevation): step time and
    # the error against the true source angles, grid peaks beside refined ones
    refine2d = {}
    if rank == 0 and not args.no_forms:
        ang = torch.full((B, du, 2), float("nan"), dtype=torch.float64, device=dev)
        geom = doa.geometry(pos, float(91 - Le), 1.0, Le, True)
        rprobs = [doa.make_problem(X[i], du, 1 << doa.MUSIC, az, bt["P"][i], bt["idx"][i], bt["val"][i],
                                   bt["cnt"][i:i + 1], geom=geom, peak_angle=ang[i]) for i in range(B)]
        rplan = doa.BatchPlan(rprobs, device=str(dev), scan_pt=bt["plan"].scan_pt, eig_mats=bt["plan"].eig_mats)
        rws = doa.workspace(rplan, device=str(dev))
        for _ in range(args.warmup):
            doa.doa_solve_batch(rplan, rws, bt["status"], stream=stream)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        r0.record(stream)
        for _ in range(args.steps):
            doa.doa_solve_batch(rplan, rws, bt["status"], stream=stream)
        r1.record(stream)
        torch.cuda.synchronize(dev)
        ih, ch, ah = bt["idx"].cpu().numpy(), bt["cnt"].cpu().numpy(), ang.cpu().numpy()
        eg, er = [], []
        for i in range(B):
            if ch[i] != du:
                continue
            truth = sorted(zip(insts[i].az, insts[i].el))
            grid_pts = sorted(((int(k) % g0.La) * g0.az_step + g0.az_lo, (int(k) // g0.La) * 1.0 + (91 - Le))
                              for k in ih[i, :du])
            ref_pts = sorted((float(a), float(e)) for a, e in ah[i, :du])
            for (ta, te), (ga, ge), (ra, re_) in zip(truth, grid_pts, ref_pts):
                da = lambda x: (x - ta + 180.0) % 360.0 - 180.0
                eg.append((da(ga), ge - te))
                er.append((da(ra), re_ - te))
        eg, er = np.array(eg), np.array(er)
        refine2d = {"ms_per_step": r0.elapsed_time(r1) / args.steps, "solves": len(eg) // du,
                    "rmse_grid_deg": {"azimuth": float(np.sqrt(np.mean(eg[:, 0] ** 2))),
                                      "elevation": float(np.sqrt(np.mean(eg[:, 1] ** 2)))},
                    "rmse_refined_deg": {"azimuth": float(np.sqrt(np.mean(er[:, 0] ** 2))),
                                         "elevation": float(np.sqrt(np.mean(er[:, 1] ** 2)))},
                    "how": "FP64 damped Newton in (azimuth, elevation) inside one grid step around each peak; "
                           "peaks and true sources paired in sorted order"}
        del rplan, rws, rprobs
    # the four scan sizes of Table 10 (360 x {1, 30, 60, 90}), batched and single
    table10 = {}
    if rank == 0 and not args.no_forms:
        for rows in (1, 30, 60, 90):
            bt_r = build_batch(X, rows)
            gr = capture(bt_r)
            ms_r = time_graph(gr, args.steps)
            X1 = X[:1]
            b1 = build_batch(X1, rows)
            g1 = capture(b1)
            lat = time_graph(g1, 100)
            table10[f"360x{rows}"] = {"batch_ms": ms_r, "solves_per_s": B / (ms_r / 1e3),
                                      "points_per_s": B * 360 * rows / (ms_r / 1e3), "single_solve_device_ms": lat}
            del bt_r, gr, b1, g1
    # roofline of the scan stage: one factor column per noise eigenvector (M - d = 6), 8M + 4 flops
    # per column and point (complex MACs and |y|^2) and 1 for the MUSIC sum (steering not counted)
    Kn = Mu - du
    scan_flops = B * npts * (Kn * (8 * Mu + 4) + Kn)
    stage_info = {n: {"ms": round(v, 4)} for n, v in zip(doa.STAGE_NAMES, stage_ms)}
    stage_info["scan"].update(bound="alu", achieved=round(scan_flops / (stage_ms[3] / 1e3) / 1e12, 3),
                              unit="TFLOP/s", peak=round(FP32_PEAK_TFLOPS, 2))
    stage_info["scan"]["frac"] = round(stage_info["scan"]["achieved"] / FP32_PEAK_TFLOPS, 4)
    dom = max(range(doa.BATCH_STAGES), key=lambda i: stage_ms[i])
    result = {
        "metric": METRIC, "value": points / (ms / 1e3), "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded Eq. 1 snapshots of an 8-element UCA, Philox)",
        "config": {"workload": f"paper-uca batch: {B} problems, 8-element UCA r=10 m at 15 MHz, d=2, SNR 15 dB, "
                               f"N=1024, MUSIC, azimuth 0:1:359 x elevation {91 - Le}:1:90 ({npts} points)",
                   "batch_per_gpu": B, "graph": True, "scan_pt": bt["plan"].scan_pt, "eig_mats": bt["plan"].eig_mats,
                   "steering_tables": int(bt["plan"].host[:512].view(np.int32)[doa.BatchPlan.header_index("ngeo_steer")]),
                   "steering": "one FP32 table per (array, grid, M), written each step from FP64 phases, shared by "
                               "the problems that pass the same positions",
                   "l2": f"inputs {Xh.nbytes / 1e9:.2f} GB > 129 MB L2 (no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "solves_per_s": B * world / (ms / 1e3),
        "gpu_launches": bt["plan"].launches() * args.steps,
        "stages": stage_info,
        "dominant_stage": doa.STAGE_NAMES[dom],
        "roofline": {"bound": "alu", "achieved": stage_info["scan"]["achieved"], "peak": round(FP32_PEAK_TFLOPS, 2),
                     "unit": "TFLOP/s", "frac": stage_info["scan"]["frac"],
                     "traffic": (TRAFFIC_BYTES.get(f"scan_geometry_batch_kernel<8,{bt['plan'].scan_pt[0]}>") or 0) * B / 4096
                     or None,
                     "kernel": f"scan_geometry_batch_kernel<8,{bt['plan'].scan_pt[0]}>",
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"},
        "single_solve": single,
        "table10": table10,
        "refinement_2d": refine2d,
        "autotune": tune_log,
        "e2e": {"value": points / (e2e_ms / 1e3), "unit": "points/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        S = min(args.cpu_sample, B)
        workers = min(os.cpu_count() or 1, 16)
        tasks = [(Xh[i], du, 1, g0.pos, g0.az_lo, g0.az_step, g0.La, float(91 - Le), 1.0, Le) for i in range(S)]
        import multiprocessing as mp
        import oracle
        oracle.build()
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_oracle_task_uca, tasks[:workers])
            a = time.perf_counter()
            res = pool.map(_oracle_task_uca, tasks, chunksize=8)
            dt = time.perf_counter() - a
        result["cpu_baseline"] = {"value": S * npts / dt, "unit": "points/s", "cores": workers, "kind": "oracle",
                                  "seconds": round(dt, 3), "sample": f"first {S} problems of the batch ({S * npts} points)"}
        ih, ch = bt["idx"].cpu().numpy(), bt["cnt"].cpu().numpy()
        Pg = bt["P"][:min(S, args.parity_full)].cpu().numpy()
        agree, worst = 0, 0.0
        for i, (io, Po) in enumerate(res):
            agree += list(ih[i, :ch[i]]) == list(io)
            if i < len(Pg):
                worst = max(worst, float(np.max(np.abs(10 * np.log10(Pg[i].astype(np.float64) / Po)))))
        result["parity"] = {"sampled_solves": S, "peak_index_agreement": agree, "max_db_err": worst,
                            "spectra_compared": len(Pg)}
    if rank == 0 and emit:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return result


def _oracle_task_uca(args):
    X, d, alg, pos, az_lo, az_step, La, el_lo, el_step, Le = args
    import oracle
    r = oracle.solve_geometry(X, d, alg, pos, az_lo, az_step, La, el_lo, el_step, Le, True)
    return r["idx"], r["P"].reshape(-1)


def _oracle_task_generic(args):
    X, d, alg, step, L = args
    import oracle
    r = oracle.solve(X, d, alg, LO, step, L)
    return r["idx"], r["P"], r["status"]


def oracle_tasks(tasks, workers):
    import multiprocessing as mp
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map(_oracle_task_generic, tasks[:1])
        t0 = time.perf_counter()
        res = pool.map(_oracle_task_generic, tasks)
        dt = time.perf_counter() - t0
    return res, dt


def run_reference(args):
    """The FP64 CPU oracle on host cores, on a bounded sample of the same workload per step."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2007_14135_gb300 import synth
    S = args.reference_sample
    Xh, _ = synth.paper_density_batch(S)
    workers = min(os.cpu_count() or 1, 16)
    L = grid_L()
    times = []
    for k in range(args.warmup + args.steps):
        _, dt = oracle_sample(Xh, S, workers)
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.fmean(times)
    pts = S * len(ALGS) * L
    value = pts / (ms / 1e3)
    result = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Eq. 1 ULA snapshots, Philox)",
        "config": {"workload": workload_name(args.batch), "batch_per_gpu": args.batch, "M": M, "d": D,
                   "N": N_SNAP, "L": L, "algorithms": ["PHD", "MUSIC", "EV", "MN"],
                   "parallelism": "oracle on host cores (rank 0)"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": workers, "kind": "oracle",
                         "sample": f"each step: the first {S} of the {args.batch} problems x 4 algorithms"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--batch", type=int, default=None,
                    help="problems per GPU per step (default: 4096; large-array 32 replicas; learned 65536 instances)")
    ap.add_argument("--cpu-sample", type=int, default=3072,
                    help="problems timed on the oracle for cpu_baseline (peak indices compared on all)")
    ap.add_argument("--parity-full", type=int, default=48,
                    help="problems whose whole spectra are compared with the oracle (dB, Eq. 4)")
    ap.add_argument("--reference-sample", type=int, default=256, help="--impl reference: problems per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-chunk", type=int, default=1024, help="problems per streamed chunk in the e2e leg")
    ap.add_argument("--no-forms", action="store_true", help="skip the tensor-core scan and FP64-Jacobi forms")
    ap.add_argument("--no-workload-forms", action="store_true",
                    help="skip the compact uneven / large-array / learned / UCA forms of the default line")
    ap.add_argument("--workload", choices=["paper-density", "uneven", "large-array", "learned", "paper-uca"],
                    default="paper-density")
    ap.add_argument("--uca-rows", type=int, default=90, help="paper-uca workload: elevation rows (360 x rows grid)")
    ap.add_argument("--scan-pt", default="", help="paper-uca workload: fixed scan points per thread per M bucket, "
                                                  "e.g. 2,2,1,1 (no autotuning)")
    ap.add_argument("--train", type=int, default=1 << 20, help="learned workload: training instances")
    ap.add_argument("--epochs", type=int, default=40, help="learned workload: training epochs")
    ap.add_argument("--lr-decay", type=float, default=0.92, help="learned workload: learning-rate factor per epoch")
    ap.add_argument("--no-tune", action="store_true", help="uneven and paper-uca workloads: default launch shapes")
    ap.add_argument("--la-forms", default="", help="large-array workload: comma list of forms (default all)")
    ap.add_argument("--tc-min-m", type=int, default=0,
                    help="uneven workload: problems with M >= this (<= 32) scan on the tensor cores (FP16x3)")
    ap.add_argument("--grid-step", type=float, default=None,
                    help="paper-density workload: scan grid step in degrees (default 0.01; a coarser grid keeps "
                         "profiles of the stages before the scan small at the full batch)")
    args = ap.parse_args()
    if args.grid_step is not None:
        global STEP
        STEP = float(args.grid_step)
    if args.batch is None:
        args.batch = {"large-array": 32, "learned": 65536}.get(args.workload, 4096)
    if args.warmup < 3 and args.impl == "gpu":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "large-array":
        run_large_array(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "paper-uca":
        run_uca(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
