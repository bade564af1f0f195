"""GPU parity of Step-2 taken as a one-sided Jacobi SVD of X (doa_svd_data) against the FP64
oracle's oracle.svd_data: sample covariances of the paper's ULA workloads (eigenvalues and the
noise-subspace projector), random complex64 X up to M = 64, the exactly graded X of the oracle's
pins (s = 1 .. 1e-8: every s^2 to 1e-8 relative, where the covariance route loses the smallest),
rank one, a ragged N, a padded row stride, and the sweep cap."""
import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _unitary(rng, n, m=None):
    m = n if m is None else m
    A = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    Q, _ = np.linalg.qr(A)
    return Q


def _svd(torch, doa, X, ldx=None, **kw):
    M, N = X.shape
    if ldx is not None and ldx != N:
        buf = np.zeros((M, ldx), X.dtype)
        buf[:, :N] = X
        Xd = torch.from_numpy(buf).cuda()[:, :N]
    else:
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    ev = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
    U = torch.full((M, M), float("nan"), dtype=torch.complex128, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    doa.doa_svd_data(Xd, ev, U, info, **kw)
    torch.cuda.synchronize()
    return ev.cpu().numpy(), U.cpu().numpy().T.copy(), int(info.item())   # columns = singular vectors


def _check_unitary_and_diagonal(X, ev, U, tol=1e-12):
    M, N = X.shape
    assert np.abs(U.conj().T @ U - np.eye(M)).max() <= tol
    Y = U.conj().T @ X.astype(np.complex128)
    G = Y @ Y.conj().T
    assert np.abs(G - np.diag(np.diag(G))).max() <= tol * np.abs(np.diag(G)).max()
    np.testing.assert_allclose(np.diag(G).real / N, ev, rtol=1e-11, atol=1e-14 * ev[0])


def test_svd_matches_oracle_on_sample_covariances(env):
    """Paper-like ULA snapshots (M = 8, 16 with d sources): eigenvalues to 1e-13 of the largest, the
    sweep count equal to the oracle's, and the noise-subspace projector E_n E_n^H to 1e-10."""
    torch, doa = env
    for k, (M, d, N) in enumerate(((8, 2, 1024), (16, 4, 4096), (16, 6, 2048), (12, 3, 777))):
        inst = synth.custom(M, d, N, None, 10.0, 0.1, seed=900 + k)
        ev, U, info = _svd(torch, doa, inst.X)
        evo, Uo, sw = oracle.svd_data(inst.X)
        assert info > 0 and sw > 0
        assert abs(info - sw) <= 1, (info, sw)
        assert np.abs(ev - evo).max() <= 1e-13 * evo[0], (M, N)
        En, Fn = U[:, d:], Uo[:, d:]
        assert np.abs(En @ En.conj().T - Fn @ Fn.conj().T).max() <= 1e-10
        _check_unitary_and_diagonal(inst.X, ev, U)


def test_svd_random_shapes_and_strides(env):
    """Random complex64 X, M from 2 to 64, N ragged around the 32-snapshot chunks, a padded row
    stride: eigenvalues against the oracle (LAPACK for the largest) and U unitary and diagonalising."""
    torch, doa = env
    rng = np.random.default_rng(17)
    for M, N, ldx in ((2, 1, None), (2, 3, None), (5, 33, 40), (8, 200, None), (16, 1000, 1002), (32, 4097, None),
                      (64, 2048, None)):
        X = (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))).astype(np.complex64)
        ev, U, info = _svd(torch, doa, X, ldx=ldx)
        assert info > 0, (M, N, info)
        if M <= 16:
            evo, _, _ = oracle.svd_data(X)
        else:
            evo = np.linalg.svd(X.astype(np.complex128), compute_uv=False) ** 2 / N
        np.testing.assert_allclose(ev, evo, rtol=1e-12, atol=1e-14 * evo[0])
        _check_unitary_and_diagonal(X, ev, U)


def test_svd_graded_spectrum_relative_accuracy(env):
    """The oracle pin's graded X = U0 diag(s) V0^H (complex128 input), s = 1 .. 1e-8: every s_k^2
    within 1e-8 relative, as the oracle and LAPACK give, while the covariance route through the
    GPU's own doa_covariance + doa_noise_subspace loses the smallest."""
    torch, doa = env
    rng = np.random.default_rng(3)
    M, N = 5, 64
    s = np.array([1.0, 1e-2, 1e-4, 1e-6, 1e-8])
    for trial in range(4):
        X = _unitary(rng, M) @ np.diag(s) @ _unitary(rng, N, M).conj().T
        ev, U, info = _svd(torch, doa, X)
        assert info > 0
        rel = np.abs(ev * N - s ** 2) / s ** 2
        assert np.all(rel <= 1e-8), rel
        evo, _, _ = oracle.svd_data(X)
        assert np.all(np.abs(ev - evo) <= 1e-8 * evo)
    # the covariance route (complex64 snapshots are too coarse here: feed the FP64 R directly)
    R = torch.from_numpy(X @ X.conj().T / N).cuda()
    evc = torch.empty(M, dtype=torch.float64, device="cuda")
    B = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    infc = torch.zeros(1, dtype=torch.int32, device="cuda")
    doa.doa_noise_subspace(R, 1, doa.MUSIC, B, infc, evals=evc)
    torch.cuda.synchronize()
    assert abs(evc.cpu().numpy()[-1] * N - s[-1] ** 2) / s[-1] ** 2 > 1e-3


def test_svd_rank_one_and_sweep_cap(env):
    torch, doa = env
    rng = np.random.default_rng(11)
    M, N = 6, 40
    u = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = np.outer(u, v.conj())
    ev, U, info = _svd(torch, doa, X)
    lam = np.vdot(u, u).real * np.vdot(v, v).real / N
    assert info > 0
    assert abs(ev[0] - lam) <= 1e-13 * lam
    assert np.all(np.abs(ev[1:]) <= 1e-26 * lam)
    assert abs(abs(np.vdot(U[:, 0], u)) - np.linalg.norm(u)) <= 1e-12 * np.linalg.norm(u)
    # one sweep allowed on a general X: not converged, reported as -ENOCONV, outputs still written
    X = (rng.standard_normal((8, 300)) + 1j * rng.standard_normal((8, 300))).astype(np.complex64)
    ev, U, info = _svd(torch, doa, X, max_sweeps=1)
    assert info == -doa.ENOCONV
    assert np.all(np.isfinite(ev)) and np.all(np.isfinite(U))
    A = np.abs(U)                                        # the cap left U a permutation (sorted by the
    assert np.all((A == 0.0) | (A == 1.0)) and np.all(A.sum(0) == 1.0) and np.all(A.sum(1) == 1.0)   # Gram diagonal)
