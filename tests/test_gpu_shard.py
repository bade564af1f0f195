"""Grid slices on the GPU: the slice scan reproduces the full scan's points bit for bit, and the
slice peak summaries merged on the host reproduce doa_peaks on the whole spectrum (ranks run
one after another on the one GPU; the exchange itself is covered by the gloo test)."""
import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _factor(torch, doa, inst, alg):
    X = torch.from_numpy(inst.X).cuda()
    R64 = torch.empty((inst.M, inst.M), dtype=torch.complex128, device="cuda")
    doa.doa_covariance(X, None, R64)
    B = torch.empty(inst.M * inst.M, dtype=torch.complex128, device="cuda")
    K = torch.zeros(1, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    doa.doa_noise_subspace(R64, inst.d, alg, B, info, K_out=K)
    torch.cuda.synchronize()
    assert info.item() > 0
    return B, int(K.item())


@pytest.mark.parametrize("M,d,alg,step", [(16, 4, 1, 0.01), (8, 2, 0, 0.1), (33, 5, 2, 0.05), (64, 8, 1, 0.02)])
def test_scan_slice_is_the_full_scan_restricted(env, M, d, alg, step):
    torch, doa = env
    inst = synth.custom(M, d, 2000, None, 15.0, step, seed=300 + M)
    B, K = _factor(torch, doa, inst, alg)
    g = doa.grid(inst.lo, inst.step, inst.L)
    full = torch.empty(inst.L, dtype=torch.float32, device="cuda")
    doa.doa_scan(B, M, K, g, full)
    ref = full.cpu().numpy()
    L = inst.L
    for k0, n in [(0, L), (0, 1), (L - 1, 1), (1, L - 2), (L // 3, L // 3 + 7), (777 % L, min(4097, L - 777 % L))]:
        P = torch.empty(n, dtype=torch.float32, device="cuda")
        doa.doa_scan_slice(B, M, K, g, k0, n, P)
        torch.cuda.synchronize()
        assert np.array_equal(P.cpu().numpy(), ref[k0:k0 + n]), (k0, n)


def _slice_peaks(torch, doa, P, d, world):
    from paper_2007_14135_gb300 import shard
    L = len(P)
    Pd = torch.from_numpy(P).cuda()
    sums = []
    for r in range(world):
        k0, k1, b0, b1 = shard.slice_bounds(L, r, world)
        out = torch.zeros(shard.SUMMARY_BYTES, dtype=torch.uint8, device="cuda")
        doa.doa_slice_peaks(Pd[b0:b1], b0, k0, k1, L, d, out)
        torch.cuda.synchronize()
        sums.append(doa.slice_summary_from_bytes(out.cpu().numpy().tobytes()))
    return shard.merge(sums, d)


def _full_peaks(torch, doa, P, d):
    Pd = torch.from_numpy(P).cuda()
    idx = torch.full((max(d, 1),), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros(max(d, 1), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    doa.doa_peaks(Pd, d, idx, val, cnt)
    torch.cuda.synchronize()
    n = cnt.item()
    return idx.cpu().numpy()[:n], val.cpu().numpy()[:n]


def test_slice_summaries_merge_to_doa_peaks(env):
    torch, doa = env
    rng = np.random.default_rng(11)
    spectra = [rng.random(5000).astype(np.float32), np.round(rng.random(3001) * 5).astype(np.float32),
               np.cumsum(rng.choice([-1.0, 0.0, 0.0, 1.0], size=4000)).astype(np.float32),
               np.full(999, 0.25, np.float32)]
    step = np.zeros(800, np.float32)
    step[100:700] = 3.0
    spectra.append(step)
    inst = synth.paper_density(2)
    spectra.append(oracle.solve(inst.X, inst.d, 0, inst.lo, inst.step, inst.L)["P"].astype(np.float32))
    for P in spectra:
        for d in (0, 1, 4, 9):
            want_i, want_v = _full_peaks(torch, doa, P, d)
            ref_i, _ = oracle.peaks(P.astype(np.float64), d)
            assert list(want_i) == list(ref_i)
            for world in (1, 2, 3, 5, 8):
                got_i, got_v = _slice_peaks(torch, doa, P, d, world)
                assert list(got_i) == list(want_i), (len(P), d, world)
                assert np.array_equal(got_v, want_v)


def test_sliced_pipeline_on_one_gpu(env):
    """Every rank of an 8-way split scans its slice with halo and summarises it; the merged peaks
    equal the whole-grid scan + doa_peaks."""
    torch, doa = env
    from paper_2007_14135_gb300 import shard
    inst = synth.custom(16, 4, 3000, None, 12.0, 0.002, seed=77)
    B, K = _factor(torch, doa, inst, 1)
    g = doa.grid(inst.lo, inst.step, inst.L)
    full = torch.empty(inst.L, dtype=torch.float32, device="cuda")
    doa.doa_scan(B, 16, K, g, full)
    want_i, want_v = _full_peaks(torch, doa, full.cpu().numpy(), inst.d)
    sums = []
    for r in range(8):
        P, out, (k0, k1, b0, b1) = shard.scan_slice_summary(B, 16, K, g, inst.d, r, 8)
        torch.cuda.synchronize()
        assert np.array_equal(P.cpu().numpy(), full.cpu().numpy()[b0:b1])
        sums.append(doa.slice_summary_from_bytes(out.cpu().numpy().tobytes()))
    got_i, got_v = shard.merge(sums, inst.d)
    assert list(got_i) == list(want_i) and np.array_equal(got_v, want_v)
