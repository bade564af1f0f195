"""GPU parity of the batch's tensor-core covariance (Step-1, Eq. 3, exact BF16 slices): R of every
problem with M <= 16, read from the workspace, against the FP64 oracle and against the compensated
CUDA-core form; ragged snapshot counts around the 64-snapshot stages and 960-snapshot windows;
thousands of short problems (every CTA runs many problems); and the problems the kernel must hand
to the CUDA-core fixup (a sample beyond the scaling range, a silent first stage, a NaN)."""
import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import MUSIC, PHD, require_gpu

pytestmark = pytest.mark.gpu

# Error bound of the slices: the dropped pairs (level >= 6) and the residual below the sixth slice
# are under 2^-27 u0^2 per snapshot, u0 <= max|x| / 16, so |dR| <= 2^-35 max|x|^2, i.e. ~1e-9 of
# max|R| for Gaussian data (and about 1e-12 on average over thousands of snapshots).
REL_TOL = 1e-9


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _solve(torch, doa, Xs, ds, cuda_core=False, L=181, step=1.0):
    tensors, probs = [], []
    for X, d in zip(Xs, ds):
        M = X.shape[0]
        P = torch.empty(2 * L, dtype=torch.float32, device="cuda")
        idx = torch.full((2 * max(d, 1),), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(2 * max(d, 1), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
        ev = torch.empty(M, dtype=torch.float64, device="cuda")
        tensors.append((X, P, idx, val, cnt, ev))
        # PHD requested: the CUDA-core form then accumulates in compensated FP32 (MUSIC alone would
        # take its plain FP32 form, accurate to ~1e-7 only)
        probs.append(doa.make_problem(X, d, (1 << PHD) | (1 << MUSIC), doa.grid(-90.0, step, L), P, idx, val,
                                      cnt, ev, cov_cuda_core=cuda_core))
    plan = doa.BatchPlan(probs)
    ws = doa.workspace(plan)
    status = torch.full((len(probs),), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    R = [plan.covariance(ws, i).cpu().numpy() for i in range(len(probs))]
    return plan, ws, status.cpu().numpy(), R, tensors


def _check(Rg, Xh, tol=REL_TOL, what=""):
    Ro = oracle.covariance(Xh)
    err = np.max(np.abs(Rg - Ro)) / np.max(np.abs(Ro))
    assert err < tol, (what, err)
    assert np.array_equal(Rg, Rg.conj().T), what
    return err


def test_tc_covariance_ragged_shapes(env):
    """Both operand layouts (M <= 8, 8 < M <= 16) at snapshot counts around the stage (64) and
    window (960) boundaries, odd counts (the last snapshot read outside the bulk copies) and a padded
    row stride; the same problems through the compensated CUDA-core form agree."""
    torch, doa = env
    Ms = [2, 3, 5, 8, 9, 12, 13, 16]
    Ns = [1, 2, 3, 63, 64, 65, 959, 960, 961, 1921, 4096, 8191]
    Xs, Xh, ds = [], [], []
    for i, (M, N) in enumerate((M, N) for M in Ms for N in Ns):
        inst = synth.custom(M, 1, N, None, 10.0, 1.0, seed=4000 + i)
        pad = 2 if i % 3 == 0 else 0                        # ldx = N + 2 (even when N is even)
        if (N + pad) % 2:
            pad += 1                                         # keep ldx even: tensor-core eligible
        buf = np.zeros((M, N + pad), np.complex64)
        buf[:, :N] = inst.X
        Xs.append(torch.from_numpy(buf).cuda()[:, :N])
        Xh.append(inst.X)
        ds.append(1)
    plan, ws, status, R, _ = _solve(torch, doa, Xs, ds)
    assert np.all(status == 0), status
    h = plan.host.view(np.int32)
    assert list(h[108:110]) == [4 * len(Ns), 4 * len(Ns)]       # every problem on the tensor cores
    assert np.all(plan.covtc_marks(ws).cpu().numpy() == 0)
    worst = max(_check(Rg, X, what=(X.shape, i)) for i, (Rg, X) in enumerate(zip(R, Xh)))
    _, _, status2, R2, _ = _solve(torch, doa, Xs, ds, cuda_core=True)
    assert np.all(status2 == 0)
    for a, b, X in zip(R, R2, Xh):
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < REL_TOL, ("vs CUDA-core", X.shape)
    print("worst relative error", worst)


def test_tc_covariance_thousands_of_short_problems(env):
    """2000 problems of 1..300 snapshots and M in 2..16: each CTA runs about 13 problems in a row,
    wrapping the scaling ring and alternating the accumulator buffers within a few stages."""
    torch, doa = env
    rng = np.random.default_rng(77)
    Ms = rng.integers(2, 17, 2000)
    Ns = rng.integers(1, 301, 2000)
    Xh = [(rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))).astype(np.complex64) * 0.7
          for M, N in zip(Ms, Ns)]
    Xs = [torch.from_numpy(x).cuda() if x.shape[1] % 2 == 0 else
          torch.from_numpy(np.pad(x, ((0, 0), (0, 1)))).cuda()[:, :x.shape[1]] for x in Xh]
    plan, ws, status, R, _ = _solve(torch, doa, Xs, [1] * len(Xs), L=5, step=45.0)
    assert np.all(status == 0)
    assert np.all(plan.covtc_marks(ws).cpu().numpy() == 0)
    for i, (Rg, X) in enumerate(zip(R, Xh)):
        _check(Rg, X, what=i)


def test_tc_covariance_marked_problems_are_recomputed(env):
    """A problem whose later samples exceed twice the first stage's largest one, one whose first
    stage is silent, and one with a NaN are marked and recomputed by the CUDA-core fixup (the NaN
    one then reports a non-finite covariance); an ordinary problem beside them is not marked."""
    torch, doa = env
    M, N = 16, 2000
    base = [synth.custom(M, 2, N, None, 10.0, 1.0, seed=5100 + i).X for i in range(4)]
    ramp = base[0].copy()
    ramp[:, :64] *= 1.0 / 16.0                       # the scaling unit comes from a quiet first stage
    silent = base[1].copy()
    silent[:, :64] = 0.0
    nan = base[2].copy()
    nan[3, 777] = np.nan
    Xh = [ramp, silent, nan, base[3]]
    Xs = [torch.from_numpy(x).cuda() for x in Xh]
    plan, ws, status, R, _ = _solve(torch, doa, Xs, [2] * 4)
    marks = plan.covtc_marks(ws).cpu().numpy()
    assert list(marks) == [1, 1, 1, 0], marks      # equal N: the list keeps the problem order
    _check(R[0], ramp, what="ramp")
    _check(R[1], silent, what="silent")
    _check(R[3], base[3], what="plain")
    assert np.isnan(R[2]).any()
    assert status[2] == doa.ENONFINITE and status[0] == status[1] == status[3] == 0, status
