"""doa_covariance_noalloc: the covariance for callers that cannot allocate device memory while
they run (fixed-memory real-time loops, frameworks that forbid allocation after start-up). It
keeps its scratch in a library-owned device array instead of memory the caller provides, and
must agree with the existing entry point doa_covariance and with the FP64 oracle to the accuracy
of their compensated accumulation, call after call.

This file is collected last so that a stop at the first failure has already run everything else.
"""
import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

# Both entry points accumulate exact FP32 products in compensated double-float and add their chunk
# sums in FP64 (about 2^-44 relative); they split the snapshots differently (up to 8 cluster CTAs
# against 1024-snapshot chunks), so the results agree to that accuracy, not bit for bit. The FP64
# outputs are held to 1e-12 of max |R| against each other and against the FP64 oracle; the
# complex64 output to the FP32 rounding of R.
REL_TOL64 = 1e-12
REL_TOL32 = 2e-6


def _both(torch, doa, inst):
    M = inst.M
    X = torch.from_numpy(inst.X).cuda()
    R_ref = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    R_na = torch.full((M, M), float("nan"), dtype=torch.complex128, device="cuda")
    R32_na = torch.full((M, M), float("nan"), dtype=torch.complex64, device="cuda")
    doa.doa_covariance(X, R64=R_ref)
    doa.doa_covariance_noalloc(X, R=R32_na, R64=R_na)
    torch.cuda.synchronize()
    return R_ref.cpu().numpy(), R_na.cpu().numpy(), R32_na.cpu().numpy()


def test_noalloc_matches_covariance_on_consecutive_calls():
    torch, doa = require_gpu()
    # two calls in a row with different shapes (multi-chunk, then single-chunk), then the first
    # shape again: the shared scratch must not leak state between calls
    cases = [synth.custom(16, 4, 4097, None, 10.0, 0.1, seed=501),
             synth.custom(8, 2, 1000, None, 5.0, 0.1, seed=502),
             synth.custom(64, 8, 20000, None, 12.0, 0.1, seed=503),
             synth.custom(16, 4, 4097, None, 10.0, 0.1, seed=501)]
    for inst in cases:
        R_ref, R_na, R32 = _both(torch, doa, inst)
        R_or = oracle.covariance(inst.X)
        scale = np.max(np.abs(R_or))
        assert np.max(np.abs(R_na - R_ref)) <= REL_TOL64 * scale
        assert np.max(np.abs(R_na - R_or)) <= REL_TOL64 * scale
        assert np.max(np.abs(R32 - R_or)) <= REL_TOL32 * scale
        assert np.array_equal(R_na, R_na.conj().T)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, doa = require_gpu()
    M = 64
    chunks_max = doa.NOALLOC_SCRATCH_BYTES // (M * M * 16)
    N = chunks_max * 1024 + 1
    X = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
    R = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    with pytest.raises(doa.DoaError) as e:
        doa.doa_covariance_noalloc(X, R64=R)
    assert e.value.status == doa.ENOMEM
    doa.doa_covariance_noalloc(X[:, :N - 1], R64=R)   # the largest accepted size still runs
    torch.cuda.synchronize()
    assert np.all(R.cpu().numpy() == 0)
