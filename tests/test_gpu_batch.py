"""Batched solve: tile shapes, CUDA-graph replay and the autotuner (GPU, through the C ABI)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import DB_TOL, compare_peaks, db_error, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _uneven(torch, doa, n=48, thin=True):
    specs = [s for s in synth.uneven_specs(4096) if not thin or s.step >= 0.01][:n]
    insts = [synth.uneven_instance(s) for s in specs]
    tensors, probs = [], []
    for inst in insts:
        X = torch.from_numpy(inst.X).cuda()
        P = torch.empty(inst.L, dtype=torch.float32, device="cuda")
        idx = torch.full((inst.d,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(inst.d, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        tensors.append((X, P, idx, val, cnt))
        probs.append(doa.make_problem(X, inst.d, 1 << inst.alg, doa.grid(inst.lo, inst.step, inst.L), P, idx, val, cnt))
    return insts, tensors, probs


def test_tile_shapes_give_identical_spectra(env):
    """The points-per-thread and matrices-per-warp knobs change the launch shape only: every
    point is bit-identical."""
    torch, doa = env
    insts, tensors, probs = _uneven(torch, doa, n=40)
    outs = []
    for pts, em in [((1, 1, 1, 1), (1, 1, 1, 1)), ((4, 2, 1, 1), (8, 4, 2, 1)), ((2, 4, 2, 1), (2, 2, 1, 1))]:
        plan = doa.BatchPlan(probs, scan_pt=pts, eig_mats=em)
        assert plan.eig_mats == list(em)
        ws = doa.workspace(plan)
        status = torch.full((plan.nprob,), -1, dtype=torch.int32, device="cuda")
        doa.doa_solve_batch(plan, ws, status)
        torch.cuda.synchronize()
        assert np.all(status.cpu().numpy() == 0)
        outs.append([t[1].cpu().numpy().copy() for t in tensors])
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a, b)


def test_grid_shared_scan_is_bit_identical(env):
    """Problems that share a grid are scanned in groups (one steering generation per tile for the
    whole group). Every M bucket, every algorithm subset, groups of 2 and 32 with ragged last
    groups and a grid used by one problem only: each spectrum and peak set is bit for bit the one
    of the per-problem scan (groups of 1), which the parity tests hold to the oracle."""
    torch, doa = env
    Ms = [4, 8, 12, 16, 24, 32, 40, 64]
    tensors, probs = [], []
    for i in range(70):
        M = Ms[i % len(Ms)]
        step = 0.1 if i % 5 else 0.25            # two shared grids ...
        if i == 69:
            step = 0.3                           # ... and one grid of a single problem
        inst = synth.custom(M, 1 + i % 3, 700 + 13 * i, None, 10.0, step, seed=7300 + i)
        mask = 1 + i % 15
        nalg = bin(mask).count("1")
        X = torch.from_numpy(inst.X).cuda()
        P = torch.empty(nalg * inst.L, dtype=torch.float32, device="cuda")
        idx = torch.full((nalg * inst.d,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(nalg * inst.d, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(nalg, dtype=torch.int32, device="cuda")
        tensors.append((X, P, idx, val, cnt))
        probs.append(doa.make_problem(X, inst.d, mask, doa.grid(inst.lo, inst.step, inst.L), P, idx, val, cnt))
    outs = []
    for group in (1, 2, 32):
        plan = doa.BatchPlan(probs, scan_group=[group] * 4)
        assert plan.scan_group == [group] * 4
        ws = doa.workspace(plan)
        status = torch.full((plan.nprob,), -1, dtype=torch.int32, device="cuda")
        doa.doa_solve_batch(plan, ws, status)
        torch.cuda.synchronize()
        assert np.all(status.cpu().numpy() == 0)
        outs.append([[t[k].cpu().numpy().copy() for k in (1, 2, 4)] for t in tensors])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_graph_replay_matches_direct_call_and_oracle(env):
    torch, doa = env
    insts, tensors, probs = _uneven(torch, doa, n=32)
    plan = doa.BatchPlan(probs)
    ws = doa.workspace(plan)
    status = torch.full((plan.nprob,), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    direct = [t[1].cpu().numpy().copy() for t in tensors]
    for t in tensors:
        t[1].fill_(float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        doa.doa_solve_batch(plan, ws, status, stream=s)     # warm-up off the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        doa.doa_solve_batch(plan, ws, status)
    for t in tensors:
        t[1].fill_(float("nan"))
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for a, t in zip(direct, tensors):
        assert np.array_equal(a, t[1].cpu().numpy())
    for inst, t in zip(insts[:12], tensors[:12]):
        ref = oracle.solve(inst.X, inst.d, inst.alg, inst.lo, inst.step, inst.L)
        assert db_error(t[1].cpu().numpy(), ref["P"]) < DB_TOL
        n = t[4].item()
        ok, ties = compare_peaks(t[2].cpu().numpy()[:n], ref["idx"], ref["P"], 1e-4)
        assert ok, ties


def test_autotuner_picks_allowed_tiles_and_persists(env, tmp_path):
    torch, doa = env
    from paper_2007_14135_gb300 import autotune
    insts, tensors, probs = _uneven(torch, doa, n=24)
    path = str(tmp_path / "tune.json")
    log = []
    pts, em = autotune.tune(probs, path=path, log=log, reps=1)
    assert len(pts) == 4 and len(em) == 4
    for b, p in enumerate(pts):
        assert p in autotune.CANDIDATES[b]
    table = json.load(open(path))
    assert len(table) == len(log) >= 1
    for entry in log:
        b = entry["bucket"]
        assert set(entry["scan_ms"]) == set(autotune.CANDIDATES[b])
        assert set(entry["eig_ms"]) == set(autotune.EIG_CANDIDATES[b])
        assert em[b] in autotune.EIG_CANDIDATES[b]
    assert autotune.tune(probs, path=path) == (pts, em)    # second call: from the table, no timing


def test_streamed_batch_matches_resident_solve(env):
    """Chunks streamed through two buffer sets (upload, solve and download on three streams) give
    the peaks and status of one resident doa_solve_batch over the same problems."""
    torch, doa = env
    from paper_2007_14135_gb300 import streamed
    B, M, N, d, L = 48, 16, 1024, 4, 1801
    insts = [synth.custom(M, d, N, None, 10.0, 0.1, seed=500 + i) for i in range(B)]
    Xh = np.stack([inst.X for inst in insts]).astype(np.complex64)
    g = doa.grid(-90.0, 0.1, L)
    X = torch.from_numpy(Xh).cuda()
    P = torch.empty((B, 4, L), dtype=torch.float32, device="cuda")
    idx = torch.full((B, 4, d), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros((B, 4, d), dtype=torch.float32, device="cuda")
    cnt = torch.zeros((B, 4), dtype=torch.int32, device="cuda")
    st = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    probs = [doa.make_problem(X[i], d, 0xF, g, P[i], idx[i], val[i], cnt[i]) for i in range(B)]
    plan = doa.BatchPlan(probs)
    doa.doa_solve_batch(plan, doa.workspace(plan), st)
    torch.cuda.synchronize()
    sb = streamed.StreamedBatch(M, N, d, 0xF, g, 16)
    Xpin = torch.from_numpy(Xh).pin_memory()
    oi = torch.full((B, 4, d), -7, dtype=torch.int32).pin_memory()
    ov = torch.zeros((B, 4, d), dtype=torch.float32).pin_memory()
    oc = torch.zeros((B, 4), dtype=torch.int32).pin_memory()
    os_ = torch.full((B,), -7, dtype=torch.int32).pin_memory()
    for _ in range(2):
        ev = sb.enqueue(Xpin, oi, ov, oc, os_)
    ev.synchronize()
    assert np.array_equal(os_.numpy(), st.cpu().numpy()) and np.all(os_.numpy() == 0)
    assert np.array_equal(oc.numpy(), cnt.cpu().numpy())
    assert np.array_equal(oi.numpy(), idx.cpu().numpy()) and np.array_equal(ov.numpy(), val.cpu().numpy())
    assert np.array_equal(sb.spectra(2).cpu().numpy(), P[32:48].cpu().numpy())


def test_launch_count_matches_captured_graph(env):
    """BatchPlan.launches() (the bench's gpu_launches figure) equals the number of kernel nodes that
    a CUDA graph capture of one doa_solve_batch records (driver API through ctypes), for a plan
    with grid-shared FP32 groups, per-problem FP32, grid-shared and per-problem tensor-core scans,
    peak polish, tensor-core and CUDA-core covariances."""
    import ctypes
    torch, doa = env
    cu = ctypes.CDLL("libcuda.so.1")
    probs, keep = [], []

    def add(inst, prec=0, polish=False):
        X = torch.from_numpy(inst.X).cuda()
        P = torch.empty(inst.L, dtype=torch.float32, device="cuda")
        idx = torch.full((max(inst.d, 1),), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(max(inst.d, 1), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        keep.append((X, P, idx, val, cnt))
        probs.append(doa.make_problem(X, inst.d, 1 << doa.MUSIC, doa.grid(inst.lo, inst.step, inst.L), P, idx, val,
                                      cnt, prec=prec, polish=polish))

    for i in range(6):
        add(synth.custom(16, 3, 700 + i, None, 10.0, 0.1, seed=2200 + i), polish=(i % 2 == 0))
    for i in range(3):
        add(synth.custom(16, 3, 800 + i, None, 10.0, 0.1, seed=2210 + i), prec=doa.FP16X3)
    add(synth.custom(8, 2, 900, None, 10.0, 1.0, seed=2220), prec=doa.BF16X3)      # its own grid: alone
    add(synth.custom(64, 6, 2000, None, 10.0, 0.5, seed=2221))                       # CUDA-core covariance
    status = torch.zeros(len(probs), dtype=torch.int32, device="cuda")
    plan = doa.BatchPlan(probs)
    ws = doa.workspace(plan)
    s = torch.cuda.Stream()
    doa.doa_solve_batch(plan, ws, status, stream=s)     # first call outside the capture
    torch.cuda.synchronize()
    graph = ctypes.c_void_p()
    assert cu.cuStreamBeginCapture_v2(ctypes.c_void_p(s.cuda_stream), 0) == 0
    doa.doa_solve_batch(plan, ws, status, stream=s)
    assert cu.cuStreamEndCapture(ctypes.c_void_p(s.cuda_stream), ctypes.byref(graph)) == 0
    n = ctypes.c_size_t(0)
    assert cu.cuGraphGetNodes(graph, None, ctypes.byref(n)) == 0
    nodes = (ctypes.c_void_p * n.value)()
    assert cu.cuGraphGetNodes(graph, nodes, ctypes.byref(n)) == 0
    kinds = []
    for k in range(n.value):
        t = ctypes.c_int(-1)
        assert cu.cuGraphNodeGetType(ctypes.c_void_p(nodes[k]), ctypes.byref(t)) == 0
        kinds.append(t.value)
    cu.cuGraphDestroy(graph)
    torch.cuda.synchronize()
    assert kinds.count(0) == plan.launches(), (kinds, plan.launches())   # CU_GRAPH_NODE_TYPE_KERNEL = 0
