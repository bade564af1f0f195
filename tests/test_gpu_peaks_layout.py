"""Step-6 peak pickers (doa_peaks, doa_peaks2d) on spectra that start at every 4-byte offset from a
16-byte boundary, with plateaus and ties placed across the four-point groups the pickers load
together, rows shorter than four points, nearly flat rows, and d up to 63. Each case is compared
with the oracle's Step-6 on the same float32 values: indices and values bit-exact."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _view(torch, P, off):
    """A device view of P whose first element sits off floats past a 16-byte boundary."""
    buf = torch.zeros(P.size + 8, dtype=torch.float32, device="cuda")
    assert buf.data_ptr() % 16 == 0
    v = buf[off:off + P.size]
    v.copy_(torch.from_numpy(np.ascontiguousarray(P.reshape(-1), dtype=np.float32)))
    return v


def _peaks1d(torch, doa, P, off, d):
    v = _view(torch, P, off)
    idx = torch.full((max(d, 1),), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros(max(d, 1), dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    doa.doa_peaks(v, d, idx, val, cnt)
    torch.cuda.synchronize()
    n = cnt.item()
    return idx.cpu().numpy()[:n], val.cpu().numpy()[:n]


def _peaks2d(torch, doa, P, off, wrap, d):
    Le, La = P.shape
    v = _view(torch, P, off)
    idx = torch.full((max(d, 1),), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros(max(d, 1), dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    doa.doa_peaks2d(v, La, Le, wrap, d, idx, val, cnt)
    torch.cuda.synchronize()
    n = cnt.item()
    return idx.cpu().numpy()[:n], val.cpu().numpy()[:n]


def _plateaus(rng, L):
    """Integer levels with runs of equal values that start and end at every position mod 4."""
    P = rng.integers(0, 6, L).astype(np.float32)
    for start in range(1, max(L - 8, 1), 7):
        n = 1 + (start % 6)
        P[start:start + n] = 9.0 + (start % 3)
    return P


@pytest.mark.parametrize("L", [3, 4, 5, 6, 7, 8, 9, 31, 1023, 1024, 1025, 4097, 18001])
def test_peaks_every_offset(env, L):
    torch, doa = env
    rng = np.random.default_rng(L)
    spectra = [_plateaus(rng, L), rng.random(L).astype(np.float32)]
    x = np.linspace(0.0, 9.0, L)
    spectra.append((np.cos(x) ** 2 + 1e-3 * np.cos(37 * x)).astype(np.float32))   # smooth, few peaks
    for P in spectra:
        for off in range(4):
            for d in (1, 4, 63):
                gi, gv = _peaks1d(torch, doa, P, off, d)
                ri, rv = oracle.peaks(P.astype(np.float64), d)
                assert gi.tolist() == ri.tolist(), (L, off, d)
                assert np.array_equal(gv.astype(np.float64), rv), (L, off, d)


def test_peaks_many_selections(env):
    """d = 63 on noise: the winning threads' four-entry caches run dry and are refilled many times
    inside the warp rounds."""
    torch, doa = env
    rng = np.random.default_rng(63)
    for L in (18001, 360001):
        P = rng.random(L).astype(np.float32)
        P[::97] = 2.0 + rng.integers(0, 3, P[::97].size)          # many equal tall peaks
        for off in range(4):
            gi, gv = _peaks1d(torch, doa, P, off, 63)
            ri, rv = oracle.peaks(P.astype(np.float64), 63)
            assert len(ri) == 63
            assert gi.tolist() == ri.tolist(), (L, off)
            assert np.array_equal(gv.astype(np.float64), rv)


@pytest.mark.parametrize("Le,La", [(5, 1), (3, 2), (7, 3), (4, 4), (3, 5), (2, 6), (9, 7), (6, 13), (90, 360),
                                   (5, 361)])
def test_peaks2d_every_offset(env, Le, La):
    torch, doa = env
    rng = np.random.default_rng(Le * 1000 + La)
    spectra = [rng.integers(0, 4, (Le, La)).astype(np.float32), rng.random((Le, La)).astype(np.float32)]
    # rows that are nearly flat along the azimuth (as near the pole of a circular array), then a lobe
    a = np.arange(La)[None, :]
    e = np.arange(Le)[:, None]
    lobe = np.cos(2 * np.pi * a / max(La, 1)) * np.exp(-0.1 * e) + 0.05 * e
    jitter = rng.integers(0, 3, (Le, La)) * 1e-6
    spectra.append((lobe * (e > Le // 3) + 1.0 + jitter).astype(np.float32))
    for P in spectra:
        for wrap in (False, True):
            for off in range(4):
                for d in (1, 5, 63):
                    gi, gv = _peaks2d(torch, doa, P, off, wrap, d)
                    ri, rv = oracle.peaks2d(P.astype(np.float64), d, wrap)
                    assert gi.tolist() == ri.tolist(), (Le, La, wrap, off, d)
                    assert np.array_equal(gv.astype(np.float64), rv), (Le, La, wrap, off, d)
