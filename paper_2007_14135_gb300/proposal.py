"""Learned angle proposal (not in the paper): orchestration of the library's kernels.

Training data: instances of the proposal workload (M=16, d in U{1..6}, SNR U[-5,20] dB, angles
U[-80,80] with 3 deg separation, N=2048) are generated on the GPU (doa_synth_ula, Philox), solved
by the plain method (doa_solve_batch: covariance, Jacobi, MUSIC scan on a 0.1 deg grid, peaks),
which also writes the network input (trace-normalised upper triangle of R). The label of an
instance is the set of 1-degree bins that contain the plain method's d peaks, so the network
imitates the method and the method remains the arbiter.

Inference: covariance + Jacobi + features + MUSIC factor for the batch, with the plain MUSIC scan
on the coarse 0.1 deg full grid, network forward, doa_proposal_windows (the d best bins with
1-bin suppression -> +-2 deg windows on the 0.001 deg grid), doa_scan_windows over the windows,
then the judge (doa_proposal_judge): every coarse local maximum that no window covers gets a
+-0.2 deg judge window on the fine grid, and a row falls back to the plain full-grid scan when a
judge window reaches its weakest selected peak, when it has fewer than d window peaks, or when a
window maximum lies on a window edge above that peak.
This module only marshals arguments and loops over chunks; all arithmetic runs in libdoa.so.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Optional

import numpy as np
import torch

from . import doa, synth

M, N_SNAP, DMAX = 16, 2048, 6
WMAX = 8                                # windows per instance (d plus up to EXTRA more proposals)
EXTRA = 2
COARSE_STEP = 0.1                       # label grid
FINE_STEP = 0.001                       # fine grid of the windows and of the full-grid arbiter
WIDTH = 4001                            # +-2 deg at 0.001 deg
JUDGE_WIDTH = 401                       # +-0.2 deg judge windows around uncovered coarse maxima
TRAIN_SEED, TEST_SEED = 20071417, 20071418


def fine_grid() -> doa.Grid:
    return doa.grid(-90.0, FINE_STEP, synth.grid_size(FINE_STEP))


@dataclasses.dataclass
class Solved:
    """Per-instance outputs of the plain method on one chunk."""
    features: torch.Tensor   # (n, 272) float32
    B: torch.Tensor          # (n, M*M) complex128 MUSIC factor
    K: torch.Tensor          # (n,) int32
    d: torch.Tensor          # (n,) int32
    idx: torch.Tensor        # (n, DMAX) int32 peak indices on the solve grid
    count: torch.Tensor      # (n,) int32
    coarse: Optional[torch.Tensor] = None   # (n, 1801) coarse full-grid MUSIC spectra (the judge's input)


def solve_chunk(d: np.ndarray, ang: np.ndarray, snr: np.ndarray, seed: int, first: int, step: float,
                device: str = "cuda") -> Solved:
    """Generates the chunk's snapshots on the GPU and runs the plain MUSIC method on `step` grid."""
    n = len(d)
    dt = torch.from_numpy(d).to(device)
    X = torch.empty((n, M, N_SNAP), dtype=torch.complex64, device=device)
    doa.doa_synth_ula(dt, torch.from_numpy(ang).to(device), torch.from_numpy(snr).to(device), M, N_SNAP, seed,
                      first, X)
    L = synth.grid_size(step)
    g = doa.grid(-90.0, step, L)
    P = torch.empty((n, L), dtype=torch.float32, device=device)
    idx = torch.full((n, DMAX), -1, dtype=torch.int32, device=device)
    val = torch.zeros((n, DMAX), dtype=torch.float32, device=device)
    cnt = torch.zeros(n, dtype=torch.int32, device=device)
    feats = torch.empty((n, M * (M + 1)), dtype=torch.float32, device=device)
    B = torch.zeros((n, M * M), dtype=torch.complex128, device=device)
    probs = [doa.make_problem(X[i], int(d[i]), 1 << doa.MUSIC, g, P[i], idx[i], val[i], cnt[i:i + 1],
                              features=feats[i], B_out=B[i]) for i in range(n)]
    plan = doa.BatchPlan(probs, device=device)
    ws = doa.workspace(plan, device=device)
    status = torch.empty(n, dtype=torch.int32, device=device)
    doa.doa_solve_batch(plan, ws, status)
    K = torch.from_numpy((M - d).astype(np.int32)).to(device)
    del X, ws
    # on the coarse grid the spectra are the judge's input
    return Solved(feats, B, K, dt, idx, cnt, P if step == COARSE_STEP else None)


def labels_from_peaks(idx: np.ndarray, count: np.ndarray, step: float) -> np.ndarray:
    """Multi-hot 1-degree bins (centres -90..90) containing the method's peaks."""
    n = idx.shape[0]
    Y = np.zeros((n, doa.MLP_DIMS[-1]), dtype=np.float32)
    for j in range(idx.shape[1]):
        ok = j < count
        ang = -90.0 + idx[:, j].astype(np.float64) * step
        b = np.clip(np.rint(ang).astype(np.int64) + 90, 0, 180)
        Y[np.nonzero(ok)[0], b[ok]] = 1.0
    return Y


def make_training_set(count: int, seed: int = TRAIN_SEED, chunk: int = 8192, device: str = "cuda"):
    """Features and labels of `count` method-generated instances (kept on the device)."""
    d, ang, snr = synth.proposal_params(count, seed)
    feats = torch.empty((count, 272), dtype=torch.float32, device=device)
    labels = torch.empty((count, 181), dtype=torch.float32, device=device)
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        sol = solve_chunk(d[s:e], ang[s:e], snr[s:e], seed, s, COARSE_STEP, device)
        feats[s:e] = sol.features
        Y = labels_from_peaks(sol.idx.cpu().numpy(), sol.count.cpu().numpy(), COARSE_STEP)
        labels[s:e] = torch.from_numpy(Y).to(device)
    return feats, labels


def train(net: doa.Mlp, feats: torch.Tensor, labels: torch.Tensor, epochs: int = 3, batch: int = 4096,
          lr: float = 1e-3, seed: int = 0, log: Optional[list] = None, decay: float = 1.0) -> list:
    """Adam on shuffled minibatches (the permutation is drawn on the host and passed in); the
    learning rate is multiplied by `decay` after every epoch."""
    n = (feats.shape[0] // batch) * batch
    ws = net.workspace(batch)
    loss = torch.zeros(1, dtype=torch.float32, device=feats.device)
    rng = np.random.Generator(np.random.Philox(key=seed))
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(feats.shape[0])[:n].astype(np.int64)).to(feats.device)
        fb = feats[perm]
        lb = labels[perm]
        for s in range(0, n, batch):
            net.backward(fb[s:s + batch], lb[s:s + batch], ws, loss=loss)
            net.adam(lr * decay ** ep)
        hist.append(float(loss.item()))
        if log is not None:
            log.append({"epoch": ep, "loss": hist[-1]})
    return hist


@dataclasses.dataclass
class Inference:
    idx: np.ndarray          # (n, DMAX) fine-grid peak indices, ascending (first count valid)
    count: np.ndarray
    fallback: np.ndarray     # rows rescanned on the full grid
    judged: np.ndarray       # rows the judge sent to the full grid (a subset of fallback)
    windows: np.ndarray      # (n, DMAX) window starts (-1 unused)
    points: int              # fine-grid points evaluated (windows + fallback rows)
    seconds: float


def infer(net: doa.Mlp, sol: Solved, extra: int = EXTRA, device: str = "cuda", judge: bool = True) -> Inference:
    """Network forward, windows, windowed scan, judge (needs sol.coarse), fallback for the flagged rows."""
    n = sol.features.shape[0]
    nb = (n + 7) // 8 * 8
    fg = fine_grid()
    feats = sol.features if nb == n else torch.cat([sol.features, torch.zeros((nb - n, 272), device=device)])
    ws = net.workspace(nb)
    probs = torch.empty((nb, 181), dtype=torch.float32, device=device)
    win = torch.full((n, WMAX), -1, dtype=torch.int32, device=device)
    S = torch.empty(fg.L, dtype=torch.int32, device=device)
    Pwin = torch.empty((n, WMAX, WIDTH), dtype=torch.float32, device=device)
    idx = torch.full((n, WMAX), -1, dtype=torch.int32, device=device)
    val = torch.zeros((n, WMAX), dtype=torch.float32, device=device)
    cnt = torch.zeros(n, dtype=torch.int32, device=device)
    fb = torch.zeros(n, dtype=torch.int32, device=device)
    use_judge = judge and sol.coarse is not None
    if use_judge:
        jfirst = torch.full((n, doa.JUDGE_MAX), -1, dtype=torch.int32, device=device)
        Pj = torch.empty((n, doa.JUDGE_MAX, JUDGE_WIDTH), dtype=torch.float32, device=device)
        cg = doa.grid(-90.0, COARSE_STEP, synth.grid_size(COARSE_STEP))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.forward(feats, ws, probs=probs)
    doa.doa_proposal_windows(probs, sol.d, fg, WIDTH, win, extra=extra)
    doa.doa_scan_windows(sol.B, M, sol.K, sol.d, fg, S, Pwin, idx, val, cnt, win_first=win, width=WIDTH,
                         fallback=fb)
    fb_windows = fb.clone() if use_judge else fb
    if use_judge:
        doa.doa_proposal_judge(sol.B, M, sol.K, sol.d, sol.coarse, cg, fg, win, WIDTH, val, cnt, JUDGE_WIDTH, jfirst,
                               S, Pj, fb)
    fbh = fb.cpu().numpy()
    rows = np.nonzero(fbh)[0].astype(np.int32)
    if len(rows):
        rt = torch.from_numpy(rows).to(device)
        Pf = torch.empty((len(rows), 1, fg.L), dtype=torch.float32, device=device)
        doa.doa_scan_windows(sol.B, M, sol.K, sol.d, fg, S, Pf, idx, val, cnt, full=True, rows=rt)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    wins = win.cpu().numpy()
    pts = int((wins >= 0).sum()) * WIDTH + len(rows) * fg.L
    judged = np.zeros(n, dtype=bool)
    if use_judge:
        pts += int((jfirst.cpu().numpy() >= 0).sum()) * JUDGE_WIDTH
        judged = (fbh != 0) & (fb_windows.cpu().numpy() == 0)
    return Inference(idx.cpu().numpy()[:, :DMAX], cnt.cpu().numpy(), fbh, judged, wins, pts, dt)


def full_grid(sol: Solved, rows_chunk: int = 8192, device: str = "cuda"):
    """The plain method on the whole 0.001 deg grid (the arbiter): peaks for every row."""
    n = sol.features.shape[0]
    fg = fine_grid()
    S = torch.empty(fg.L, dtype=torch.int32, device=device)
    idx = torch.full((n, DMAX), -1, dtype=torch.int32, device=device)
    val = torch.zeros((n, DMAX), dtype=torch.float32, device=device)
    cnt = torch.zeros(n, dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(0, n, rows_chunk):
        e = min(n, s + rows_chunk)
        rt = torch.arange(s, e, dtype=torch.int32, device=device)
        P = torch.empty((e - s, 1, fg.L), dtype=torch.float32, device=device)
        doa.doa_scan_windows(sol.B, M, sol.K, sol.d, fg, S, P, idx, val, cnt, full=True, rows=rt)
        del P
    torch.cuda.synchronize()
    return idx.cpu().numpy(), cnt.cpu().numpy(), time.perf_counter() - t0


class TestSet:
    """A resident batch of proposal-workload instances with a reusable plan: solve() runs the
    covariance, Jacobi, features and MUSIC factor for every instance and the plain MUSIC scan on
    the coarse 0.1 deg full grid (the judge's input; the fine spectrum is produced later, by the
    windows or by the full-grid scan)."""

    def __init__(self, count: int, seed: int = TEST_SEED, device: str = "cuda"):
        self.d_np, self.ang, self.snr = synth.proposal_params(count, seed)
        n = count
        self.n = n
        self.device = device
        self.d = torch.from_numpy(self.d_np).to(device)
        self.X = torch.empty((n, M, N_SNAP), dtype=torch.complex64, device=device)
        doa.doa_synth_ula(self.d, torch.from_numpy(self.ang).to(device), torch.from_numpy(self.snr).to(device), M,
                          N_SNAP, seed, 0, self.X)
        g = doa.grid(-90.0, COARSE_STEP, synth.grid_size(COARSE_STEP))
        self.P = torch.empty((n, g.L), dtype=torch.float32, device=device)
        self.idx = torch.empty((n, DMAX), dtype=torch.int32, device=device)
        self.val = torch.empty((n, DMAX), dtype=torch.float32, device=device)
        self.cnt = torch.empty(n, dtype=torch.int32, device=device)
        self.features = torch.empty((n, M * (M + 1)), dtype=torch.float32, device=device)
        self.B = torch.zeros((n, M * M), dtype=torch.complex128, device=device)
        probs = [doa.make_problem(self.X[i], int(self.d_np[i]), 1 << doa.MUSIC, g, self.P[i], self.idx[i], self.val[i],
                                  self.cnt[i:i + 1], features=self.features[i], B_out=self.B[i]) for i in range(n)]
        self.plan = doa.BatchPlan(probs, device=device)
        self.ws = doa.workspace(self.plan, device=device)
        self.status = torch.empty(n, dtype=torch.int32, device=device)
        self.K = torch.from_numpy((M - self.d_np).astype(np.int32)).to(device)

    def solve(self):
        doa.doa_solve_batch(self.plan, self.ws, self.status)

    def solved(self) -> Solved:
        return Solved(self.features, self.B, self.K, self.d, self.idx, self.cnt, self.P)
