"""Pins of oracle.svd_data, Step-2 taken as an SVD of the snapshot matrix X itself (one-sided
Jacobi on its rows), against closed forms, exactly constructed spectra, LAPACK's SVD and the
separately pinned covariance + Jacobi eigendecomposition path. No GPU."""
import numpy as np

import oracle


def _unitary(rng, n, m=None):
    m = n if m is None else m
    A = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    Q, _ = np.linalg.qr(A)
    return Q


def test_orthogonal_rows():
    """Rows that are already orthogonal (scaled DFT rows): eigenvalues are the rows' mean squares,
    sorted descending, and U is a permutation up to phases."""
    N = 64
    n = np.arange(N)
    scales = np.array([0.5, 3.0, 1.0, 2.0])
    X = np.stack([s * np.exp(2j * np.pi * k * n / N) for s, k in zip(scales, (1, 5, 9, 13))])
    ev, U, sweeps = oracle.svd_data(X)
    assert sweeps >= 1
    np.testing.assert_allclose(ev, np.sort(scales ** 2)[::-1], rtol=1e-13)
    P = np.abs(U)
    assert np.allclose(np.sort(P, axis=0)[-1], 1.0, atol=1e-12)
    assert np.allclose(np.sort(P, axis=0)[:-1], 0.0, atol=1e-12)
    assert list(np.argmax(P, axis=0)) == list(np.argsort(-scales ** 2, kind="stable"))


def test_rank_one():
    """X = u v^H: one eigenvalue |u|^2 |v|^2 / N with eigenvector u / |u|, the rest zero."""
    rng = np.random.default_rng(11)
    M, N = 6, 40
    u = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = np.outer(u, v.conj())
    ev, U, _ = oracle.svd_data(X)
    lam = np.vdot(u, u).real * np.vdot(v, v).real / N
    assert abs(ev[0] - lam) <= 1e-13 * lam
    assert np.all(np.abs(ev[1:]) <= 1e-26 * lam)
    assert abs(abs(np.vdot(U[:, 0], u)) - np.linalg.norm(u)) <= 1e-12 * np.linalg.norm(u)


def test_graded_spectrum_relative_accuracy():
    """X = U0 diag(s) V0^H with s from 1 to 1e-8: the SVD route recovers every s_k^2 to high
    relative accuracy (as LAPACK's SVD does), while the route through R = X X^H / N loses the
    smallest, whose eigenvalue sits at R's rounding level. This is why the SVD form exists."""
    rng = np.random.default_rng(3)
    M, N = 5, 64
    s = np.array([1.0, 1e-2, 1e-4, 1e-6, 1e-8])
    X = _unitary(rng, M) @ np.diag(s) @ _unitary(rng, N, M).conj().T
    ev, U, _ = oracle.svd_data(X)
    rel = np.abs(ev * N - s ** 2) / s ** 2
    assert np.all(rel <= 1e-8), rel
    lapack = np.linalg.svd(X, compute_uv=False) ** 2
    assert np.all(np.abs(ev * N - lapack) <= 1e-8 * lapack)
    e2, _, _ = oracle.eigh(X @ X.conj().T / N)
    assert abs(e2[-1] * N - s[-1] ** 2) / s[-1] ** 2 > 1e-3


def test_matches_lapack_and_is_unitary():
    rng = np.random.default_rng(5)
    for M, N in ((2, 3), (8, 200), (16, 1000), (16, 4096)):
        X = (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))).astype(np.complex64)
        ev, U, sweeps = oracle.svd_data(X)
        assert sweeps > 0
        s2 = np.linalg.svd(X.astype(np.complex128), compute_uv=False) ** 2 / N
        np.testing.assert_allclose(ev, s2, rtol=1e-12, atol=1e-14 * s2[0])
        assert np.abs(U.conj().T @ U - np.eye(M)).max() <= 1e-13
        Y = U.conj().T @ X.astype(np.complex128)
        G = Y @ Y.conj().T
        off = np.abs(G - np.diag(np.diag(G)))
        assert off.max() <= 1e-12 * np.abs(np.diag(G)).max()
        np.testing.assert_allclose(np.diag(G).real / N, ev, rtol=1e-12)


def test_matches_covariance_eig_path():
    """On ordinary sample covariances the two oracle routes agree: eigenvalues to ~1e-13 of the
    largest and the noise-subspace projectors (which fix what Steps 3-5 see) to 1e-10."""
    from paper_2007_14135_gb300 import synth
    for seed in range(3):
        inst = synth.custom(16, 4, 2048, None, 10.0, 0.1, seed=500 + seed)
        ev, U, _ = oracle.svd_data(inst.X)
        e2, V, _ = oracle.eigh(oracle.covariance(inst.X))
        assert np.abs(ev - e2).max() <= 1e-13 * e2[0]
        En, Fn = U[:, inst.d:], V[:, inst.d:]
        assert np.abs(En @ En.conj().T - Fn @ Fn.conj().T).max() <= 1e-10


def test_rank_deficient_rows_converge():
    """N < M: X has rank N, so M - N rows end at the rounding level; the zero-row floor (squared
    norm below 1e-30 of the largest) stops the iteration, the N nonzero eigenvalues match LAPACK's
    singular values and the rest are zero to rounding, U stays unitary."""
    rng = np.random.default_rng(23)
    for M, N in ((2, 1), (5, 3), (8, 4), (16, 7)):
        X = (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))).astype(np.complex64)
        ev, U, sweeps = oracle.svd_data(X)
        assert sweeps > 0, (M, N, sweeps)
        s2 = np.linalg.svd(X.astype(np.complex128), compute_uv=False) ** 2 / N
        np.testing.assert_allclose(ev[:N], s2, rtol=1e-12)
        assert np.all(np.abs(ev[N:]) <= 1e-28 * ev[0])
        assert np.abs(U.conj().T @ U - np.eye(M)).max() <= 1e-13
