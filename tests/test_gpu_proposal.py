"""Learned-proposal pipeline on the GPU: snapshot synthesis, features, windows, windowed scan with
fallback, and the trained network's gain over the plain full-grid method it imitates."""
import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import DB_TOL, db_error, require_gpu
from tests.philox_ref import synth_ula as synth_ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def test_synth_matches_reference(env):
    torch, doa = env
    d = np.array([1, 3, 6], np.int32)
    ang = np.zeros((3, 6), np.float32)
    ang[0, :1] = [10.0]
    ang[1, :3] = [-40.0, 0.5, 33.0]
    ang[2, :6] = [-75.0, -50.0, -20.0, 5.0, 40.0, 79.0]
    snr = np.array([0.0, 10.0, -5.0], np.float32)
    X = torch.empty((3, 16, 40), dtype=torch.complex64, device="cuda")
    doa.doa_synth_ula(torch.from_numpy(d).cuda(), torch.from_numpy(ang).cuda(), torch.from_numpy(snr).cuda(),
                      16, 40, 0x1234567890ab, 777, X)
    torch.cuda.synchronize()
    ref = synth_ref(d, ang.astype(np.float64), snr.astype(np.float64), 16, 40, 0x1234567890ab, 777)
    got = X.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 2e-4 * np.max(np.abs(ref))


def test_features_and_factor_outputs(env):
    torch, doa = env
    from paper_2007_14135_gb300 import proposal
    d, ang, snr = synth.proposal_params(24, 5)
    sol = proposal.solve_chunk(d, ang, snr, 99, 0, 0.5)
    X = torch.empty((24, 16, 2048), dtype=torch.complex64, device="cuda")
    doa.doa_synth_ula(torch.from_numpy(d).cuda(), torch.from_numpy(ang).cuda(), torch.from_numpy(snr).cuda(),
                      16, 2048, 99, 0, X)
    Xh = X.cpu().numpy()
    F = sol.features.cpu().numpy()
    Bh = sol.B.cpu().numpy()
    for i in range(24):
        R = oracle.covariance(Xh[i])
        iu = np.triu_indices(16)
        f = np.stack([R[iu].real, R[iu].imag], axis=1).reshape(-1) / np.trace(R).real
        np.testing.assert_allclose(F[i], f, rtol=0, atol=1e-6)
        ev, V, _ = oracle.eigh(R)
        C, _ = oracle.weighting(ev, V, int(d[i]), 1)
        K = 16 - int(d[i])
        Bi = Bh[i][:16 * K].reshape(K, 16).T
        assert np.max(np.abs(Bi @ Bi.conj().T - C)) < 2e-6   # FP32-accurate R (MUSIC-only problem)


def test_windows_decode(env):
    torch, doa = env
    probs = np.full((2, 181), 0.01, np.float32)
    probs[0, [10, 11, 100, 170]] = [0.9, 0.8, 0.7, 0.95]     # bin 11 is suppressed by bin 10
    probs[1, 0] = 0.5
    d = np.array([3, 2], np.int32)
    win = torch.full((2, 6), -9, dtype=torch.int32, device="cuda")
    fg = doa.grid(-90.0, 0.001, 180001)
    doa.doa_proposal_windows(torch.from_numpy(probs).cuda(), torch.from_numpy(d).cuda(), fg, 4001, win, extra=0)
    w = win.cpu().numpy()
    # centres -90 + bin deg -> index (centre + 90) / 0.001, start = centre - 2000
    assert list(w[0, :3]) == [170 * 1000 - 2000, 10 * 1000 - 2000, 100 * 1000 - 2000]
    assert list(w[0, 3:]) == [-1, -1, -1]
    assert w[1, 0] == 0 and w[1, 1] == 2 * 1000 - 2000 and list(w[1, 2:]) == [-1] * 4   # clamped; bin 1 suppressed


def test_windowed_scan_is_the_full_grid_scan_restricted(env):
    """Spectra of windows placed around the full-grid peaks are bit-identical to the full-grid
    spectrum there, the merged peaks equal the full-grid peaks, and a window placed away from a
    peak raises the fallback flag."""
    torch, doa = env
    from paper_2007_14135_gb300 import proposal
    d, ang, snr = synth.proposal_params(16, 6)
    sol = proposal.solve_chunk(d, ang, snr, 7, 0, 0.5)
    fg = proposal.fine_grid()
    n = 16
    S = torch.empty(fg.L, dtype=torch.int32, device="cuda")
    Pf = torch.empty((n, 1, fg.L), dtype=torch.float32, device="cuda")
    fi = torch.full((n, 6), -1, dtype=torch.int32, device="cuda")
    fv = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    fc = torch.zeros(n, dtype=torch.int32, device="cuda")
    doa.doa_scan_windows(sol.B, 16, sol.K, sol.d, fg, S, Pf, fi, fv, fc, full=True)
    fih, fch = fi.cpu().numpy(), fc.cpu().numpy()
    Pfh = Pf.cpu().numpy()[:, 0]
    # oracle check of the full-grid arbiter on two rows
    for r in range(2):
        Xr = torch.empty((1, 16, 2048), dtype=torch.complex64, device="cuda")
        doa.doa_synth_ula(sol.d[r:r + 1], torch.from_numpy(ang[r:r + 1]).cuda(), torch.from_numpy(snr[r:r + 1]).cuda(),
                          16, 2048, 7, r, Xr)
        ref = oracle.solve(Xr.cpu().numpy()[0], int(d[r]), 1, fg.lo_deg, fg.step_deg, fg.L)
        assert db_error(Pfh[r], ref["P"]) < DB_TOL
        assert list(fih[r, :fch[r]]) == list(ref["idx"])
    win = np.full((n, 6), -1, np.int32)
    for r in range(n):
        for j in range(fch[r]):
            win[r, j] = min(max(fih[r, j] - 2000, 0), fg.L - 4001)
    win[3, 0] = max(fih[3, 0] - 4000, 0)          # row 3: the first peak sits on the window edge
    wt = torch.from_numpy(win).cuda()
    Pw = torch.empty((n, 6, 4001), dtype=torch.float32, device="cuda")
    wi = torch.full((n, 6), -1, dtype=torch.int32, device="cuda")
    wv = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    wc = torch.zeros(n, dtype=torch.int32, device="cuda")
    fb = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    doa.doa_scan_windows(sol.B, 16, sol.K, sol.d, fg, S, Pw, wi, wv, wc, win_first=wt, width=4001, fallback=fb)
    Pwh, wih, wch, fbh = Pw.cpu().numpy(), wi.cpu().numpy(), wc.cpu().numpy(), fb.cpu().numpy()
    for r in range(n):
        for j in range(6):
            if win[r, j] >= 0:
                assert np.array_equal(Pwh[r, j], Pfh[r, win[r, j]:win[r, j] + 4001])
        if r != 3:
            assert list(wih[r, :wch[r]]) == list(fih[r, :fch[r]])
            # fewer than d peaks on the full grid: the windows cannot find d either
            assert fbh[r] == (1 if fch[r] < d[r] else 0)
    assert fbh[3] == 1


def test_learned_proposal_gains_over_full_grid(env):
    """Train on 1M method-generated instances, then on 16384 held-out instances the windowed
    pipeline (one extra window, the judge on the coarse full-grid spectrum, fallback to the full
    grid) reproduces the full-grid method's peak indices on every one of them while evaluating
    >= 3x fewer grid points; without the judge some rows differ."""
    torch, doa = env
    from paper_2007_14135_gb300 import proposal
    feats, labels = proposal.make_training_set(1 << 20, seed=proposal.TRAIN_SEED)
    net = doa.Mlp(seed=1)
    hist = proposal.train(net, feats, labels, epochs=12, batch=4096, lr=2e-3, decay=0.85)
    assert hist[-1] < 0.7 * hist[0]
    d, ang, snr = synth.proposal_params(16384, proposal.TEST_SEED)
    sol = proposal.solve_chunk(d, ang, snr, proposal.TEST_SEED, 0, proposal.COARSE_STEP)
    assert sol.coarse is not None
    ji, jc, _ = proposal.full_grid(sol)
    full_pts = len(d) * proposal.fine_grid().L

    def agreement(inf):
        return np.array([list(inf.idx[i, :inf.count[i]]) == list(ji[i, :jc[i]]) for i in range(len(d))])

    bare = proposal.infer(net, sol, extra=1, judge=False)
    judged = proposal.infer(net, sol, extra=1)
    same = agreement(judged)
    print("agreement without / with the judge", agreement(bare).mean(), same.mean(),
          "fallback", bare.fallback.mean(), judged.fallback.mean(), "points ratio", full_pts / judged.points)
    assert same.all(), (np.nonzero(~same)[0][:10], judged.fallback.mean())
    assert set(np.nonzero(~agreement(bare))[0]) <= set(np.nonzero(judged.judged)[0])
    assert full_pts / judged.points >= 3.0, (full_pts / judged.points, judged.fallback.mean())
