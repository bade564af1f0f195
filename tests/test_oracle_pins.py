"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it pins. The expected values come from closed forms, hand
derivations (tests/golden), invariants and special cases, never from the oracle itself.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2007_14135_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PHD, MUSIC, EV, MN = 0, 1, 2, 3


def _ula(M, theta_deg):
    """Half-wavelength ULA response written out for the checks: exp(j pi m sin theta)."""
    m = np.arange(M)
    return np.exp(1j * math.pi * m * math.sin(math.radians(theta_deg)))


def _rand_unitary(M, rng):
    Z = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    Q, Rr = np.linalg.qr(Z)
    return Q * (np.diag(Rr) / np.abs(np.diag(Rr)))


def _proj(V):
    return V @ V.conj().T


# ------------------------------------------------------------------------------ Step-1, Eq. 3
def test_covariance_hand_values(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "covariance_2x3.json")))
    X = (np.array(g["X_re"]) + 1j * np.array(g["X_im"])).astype(np.complex64)
    R = oracle_mod.covariance(X)
    R_exp = np.array(g["R_re"]) + 1j * np.array(g["R_im"])
    np.testing.assert_allclose(R, R_exp, rtol=0, atol=1e-15)


def test_covariance_invariants(oracle_mod):
    inst = synth.custom(7, 2, 333, [-10.0, 25.0], 5.0, 0.1, seed=11)
    R = oracle_mod.covariance(inst.X)
    X64 = inst.X.astype(np.complex128)
    np.testing.assert_allclose(R, R.conj().T, rtol=0, atol=0)            # Hermitian
    assert np.all(np.real(np.diag(R)) >= 0) and np.all(np.imag(np.diag(R)) == 0)
    assert abs(np.trace(R).real - np.sum(np.abs(X64) ** 2) / inst.N) < 1e-12 * np.trace(R).real
    # row/column orientation: R[a, b] pairs x_a with conj(x_b)
    a, b = 1, 4
    manual = np.sum(X64[a] * np.conj(X64[b])) / inst.N
    assert abs(R[a, b] - manual) < 1e-13 * abs(manual)


# ------------------------------------------------------------------------------ Step-2
def test_eig_2x2_closed_form(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "covariance_2x3.json")))
    R = np.array(g["R_re"]) + 1j * np.array(g["R_im"])
    ev, V, sweeps = oracle_mod.eigh(R)
    assert sweeps > 0
    np.testing.assert_allclose(ev, g["evals_desc"], rtol=1e-14)
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, c = rng.uniform(-3, 3, 2)
        b = complex(*rng.uniform(-2, 2, 2))
        R = np.array([[a, b], [np.conj(b), c]])
        ev, V, _ = oracle_mod.eigh(R)
        disc = math.sqrt(((a - c) / 2) ** 2 + abs(b) ** 2)
        lam = [(a + c) / 2 + disc, (a + c) / 2 - disc]
        np.testing.assert_allclose(ev, lam, rtol=1e-13, atol=1e-14)
        for i in range(2):   # v proportional to [b, lambda - a]^T
            v = np.array([b, lam[i] - a])
            v /= np.linalg.norm(v)
            assert abs(abs(np.vdot(v, V[:, i])) - 1) < 1e-12


def _cubic_eigs(A):
    """Eigenvalues of a 3x3 Hermitian matrix from the trigonometric solution of its
    characteristic cubic (Smith, CACM 4(4):168, 1961)."""
    q = np.trace(A).real / 3
    p1 = abs(A[0, 1]) ** 2 + abs(A[0, 2]) ** 2 + abs(A[1, 2]) ** 2
    p2 = sum((A[i, i].real - q) ** 2 for i in range(3)) + 2 * p1
    p = math.sqrt(p2 / 6)
    B = (A - q * np.eye(3)) / p
    r = np.linalg.det(B).real / 2
    phi = math.acos(min(1.0, max(-1.0, r))) / 3
    l1 = q + 2 * p * math.cos(phi)
    l3 = q + 2 * p * math.cos(phi + 2 * math.pi / 3)
    return [l1, 3 * q - l1 - l3, l3]


def test_eig_3x3_trigonometric(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(20):
        Z = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        A = Z + Z.conj().T
        lam = _cubic_eigs(A)
        if min(lam[0] - lam[1], lam[1] - lam[2]) < 1e-2:
            continue
        ev, V, _ = oracle_mod.eigh(A)
        np.testing.assert_allclose(ev, lam, rtol=1e-12, atol=1e-12)
        for i in range(3):
            Bm = A - lam[i] * np.eye(3)
            v = np.cross(Bm[0], Bm[1])   # (A - lambda I) v = 0 for the bilinear rows
            v /= np.linalg.norm(v)
            assert abs(abs(np.vdot(v, V[:, i])) - 1) < 1e-9


@pytest.mark.parametrize("M", [2, 5, 8, 16, 33, 64])
def test_eig_residual_orthonormality_and_lapack(oracle_mod, M):
    rng = np.random.default_rng(100 + M)
    Z = rng.standard_normal((M, 3 * M)) + 1j * rng.standard_normal((M, 3 * M))
    R = Z @ Z.conj().T / (3 * M)
    ev, V, sweeps = oracle_mod.eigh(R)
    assert 0 < sweeps < 100
    # Eq. 5 analogue: residual of the reconstruction, and FP64 orthonormality
    res = np.linalg.norm(R - V @ np.diag(ev) @ V.conj().T) / np.linalg.norm(R)
    assert res < 1e-13
    assert np.max(np.abs(V.conj().T @ V - np.eye(M))) < 1e-13
    assert np.all(np.diff(ev) <= 0)
    lap = np.linalg.eigvalsh(R)[::-1]                  # LAPACK, used only as a checker
    np.testing.assert_allclose(ev, lap, rtol=1e-12, atol=1e-13 * lap[0])


def test_eig_known_decomposition(oracle_mod):
    rng = np.random.default_rng(3)
    M = 10
    U = _rand_unitary(M, rng)
    lam = np.sort(rng.uniform(0.1, 10, M))[::-1]
    R = U @ np.diag(lam) @ U.conj().T
    ev, V, _ = oracle_mod.eigh(R)
    np.testing.assert_allclose(ev, lam, rtol=1e-12)
    for i in range(M):
        assert abs(abs(np.vdot(U[:, i], V[:, i])) - 1) < 1e-10


def test_eig_degenerate_and_diagonal(oracle_mod):
    R = np.diag([3.0, 1.0, 2.0, 1.0]).astype(np.complex128)
    ev, V, sweeps = oracle_mod.eigh(R)
    assert sweeps == 1
    np.testing.assert_array_equal(ev, [3.0, 2.0, 1.0, 1.0])
    # stable order for the equal eigenvalues: original index 1 before index 3
    assert abs(V[1, 2]) == 1.0 and abs(V[3, 3]) == 1.0


# ------------------------------------------------------------------------------ Steps 3-4
@pytest.mark.parametrize("M,D", [(6, 2), (9, 4)])
def test_weighting_closed_forms_from_known_decomposition(oracle_mod, M, D):
    rng = np.random.default_rng(M * 10 + D)
    U = _rand_unitary(M, rng)
    lam = np.sort(rng.uniform(0.2, 5, M))[::-1]
    R = U @ np.diag(lam) @ U.conj().T
    ev, V, _ = oracle_mod.eigh(R)
    Un = U[:, D:]
    expect = {
        PHD: np.outer(U[:, -1], U[:, -1].conj()),
        MUSIC: Un @ Un.conj().T,
        EV: Un @ np.diag(1.0 / lam[D:]) @ Un.conj().T,
    }
    Pn = Un @ Un.conj().T
    valph = Pn[:, 0] / Pn[0, 0].real
    expect[MN] = np.outer(valph, valph.conj())
    for alg, Cx in expect.items():
        C, st = oracle_mod.weighting(ev, V, D, alg)
        assert st == 0
        np.testing.assert_allclose(C, Cx, rtol=0, atol=1e-11 * np.max(np.abs(Cx)))


def test_weighting_rank_errors(oracle_mod):
    M = 4
    ev = np.array([3.0, 1.0, 0.0, -1e-3])
    V = np.eye(M, dtype=np.complex128)
    assert oracle_mod.weighting(ev, V, 1, EV)[1] == 5
    # MN: u^H P_n u = 0 when the noise subspace is orthogonal to e_1
    ev = np.array([3.0, 2.0, 1.0, 0.5])
    assert oracle_mod.weighting(ev, V, 1, MN)[1] == 5
    assert oracle_mod.weighting(ev, V, 4, MUSIC)[1] == 1


# ------------------------------------------------------------------------------ Step-5, Eq. 2
def test_scan_steering_sign_and_index(oracle_mod):
    """C = u u^H with u = e_0 + j e_r gives a^H C a = |1 - j a_r|^2 = 2 + 2 sin(pi r sin theta):
    pins the +j sign of Eq. 2, the element index r and the conjugation order."""
    M, L, lo, step = 6, 37, -90.0, 5.0
    th = lo + np.arange(L) * step
    for r in (1, 3, 5):
        u = np.zeros(M, complex)
        u[0], u[r] = 1.0, 1j
        C = np.outer(u, u.conj())
        P, rel = oracle_mod.scan(C, lo, step, L)
        invp = 2 + 2 * np.sin(np.pi * r * np.sin(np.radians(th)))
        ok = invp > 1e-9
        np.testing.assert_allclose(1 / P[ok], invp[ok], rtol=1e-12, atol=1e-13)
        assert rel < 1e-12


def test_scan_dirichlet_kernel(oracle_mod):
    """C = a(t0) a(t0)^H / M: a^H C a = |sum_m exp(j pi m (s - s0))|^2 / M (Dirichlet kernel)."""
    M, L, lo, step, t0 = 8, 181, -90.0, 1.0, 17.0
    a0 = _ula(M, t0)
    C = np.outer(a0, a0.conj()) / M
    P, _ = oracle_mod.scan(C, lo, step, L)
    s = np.sin(np.radians(lo + np.arange(L) * step))
    x = np.pi * (s - math.sin(math.radians(t0))) / 2
    with np.errstate(invalid="ignore", divide="ignore"):
        dk = np.where(np.abs(np.sin(x)) < 1e-12, M * M, (np.sin(M * x) / np.sin(x)) ** 2) / M
    ok = dk > 1e-8
    np.testing.assert_allclose(1 / P[ok], dk[ok], rtol=1e-9)


def test_scan_identity_and_endpoint_symmetry(oracle_mod):
    M = 12
    P, _ = oracle_mod.scan(np.eye(M, dtype=complex), -90.0, 0.1, 1801)
    np.testing.assert_allclose(P, 1.0 / M, rtol=1e-14)
    rng = np.random.default_rng(1)
    Z = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    P, _ = oracle_mod.scan(Z @ Z.conj().T, -90.0, 0.1, 1801)
    assert abs(P[0] - P[-1]) <= 1e-12 * P[0]   # a(-90) == a(+90) for half-wavelength spacing


def test_grid_definition():
    th = synth.GRID_LO + np.arange(synth.grid_size(0.01)) * 0.01
    assert synth.grid_size(0.1) == 1801 and synth.grid_size(0.01) == 18001
    assert synth.grid_size(0.001) == 180001 and synth.grid_size(0.0005) == 360001
    assert th[0] == -90.0 and abs(th[-1] - 90.0) < 1e-9


# ------------------------------------------------------------------------------ Step-6
def test_peaks_hand_cases(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "peaks_cases.json")))
    for c in g["cases"]:
        idx, val = oracle_mod.peaks(np.array(c["P"], dtype=np.float64), c["d"])
        assert list(idx) == c["idx"], c["name"]
        np.testing.assert_array_equal(val, np.array(c["P"], float)[c["idx"]])


def test_peaks_brute_force_random(oracle_mod):
    """Brute force: enumerate every interior plateau by run-length, keep strict local maxima."""
    rng = np.random.default_rng(9)
    for trial in range(200):
        L = int(rng.integers(3, 40))
        P = rng.integers(0, 5, L).astype(np.float64)
        d = int(rng.integers(0, 6))
        runs, i = [], 0
        while i < L:
            j = i
            while j + 1 < L and P[j + 1] == P[i]:
                j += 1
            runs.append((i, j))
            i = j + 1
        cands = [i for (i, j) in runs if i >= 1 and j <= L - 2 and P[i - 1] < P[i] and P[j + 1] < P[j]]
        cands.sort(key=lambda k: (-P[k], k))
        exp = sorted(cands[:d])
        idx, _ = oracle_mod.peaks(P, d)
        assert list(idx) == exp, (P, d)


# ------------------------------------------------------------------------------ whole method
def _exact_cov(M, angles, sigma2, powers=None):
    A = np.stack([_ula(M, t) for t in angles], axis=1)
    p = np.ones(len(angles)) if powers is None else np.asarray(powers)
    return A @ np.diag(p) @ A.conj().T + sigma2 * np.eye(M), A


def test_exact_covariance_noise_eigs_and_nulls(oracle_mod):
    """R = A P A^H + sigma^2 I: noise eigenvalues = sigma^2, E_n^H a(theta_i) = 0, and the MUSIC
    spectrum has its nulls exactly at the true on-grid angles (-20, 35 deg on the 0.1 deg grid)."""
    M, angles, sigma2 = 8, [-20.0, 35.0], 0.1
    R, A = _exact_cov(M, angles, sigma2)
    ev, V, _ = oracle_mod.eigh(R)
    np.testing.assert_allclose(ev[2:], sigma2, rtol=1e-12)
    En = V[:, 2:]
    for i in range(2):
        assert np.linalg.norm(En.conj().T @ A[:, i]) < 1e-12
    C, st = oracle_mod.weighting(ev, V, 2, MUSIC)
    assert st == 0
    P, _ = oracle_mod.scan(C, -90.0, 0.1, 1801)
    invp = 1.0 / P
    for k in (700, 1250):
        assert abs(invp[k]) < 1e-12 or np.isinf(P[k])
    others = np.ones(1801, bool)
    others[[700, 1250]] = False
    assert np.min(invp[others]) > 1e-6
    # closed-form noise projector I - A (A^H A)^-1 A^H
    Pn = np.eye(M) - A @ np.linalg.solve(A.conj().T @ A, A.conj().T)
    np.testing.assert_allclose(C, Pn, atol=1e-12)
    # EV with equal noise eigenvalues: C_EV = C_MUSIC / sigma^2
    Cev, _ = oracle_mod.weighting(ev, V, 2, EV)
    np.testing.assert_allclose(Cev, Pn / sigma2, atol=1e-10)
    # MN: valph = P_n e_1 / (e_1^H P_n e_1)
    Cmn, _ = oracle_mod.weighting(ev, V, 2, MN)
    va = Pn[:, 0] / Pn[0, 0].real
    np.testing.assert_allclose(Cmn, np.outer(va, va.conj()), atol=1e-10)


def test_one_noise_vector_coincidence(oracle_mod):
    """M - d = 1: P_PHD = P_MUSIC, P_EV = lambda_min P_MUSIC, P_MN = |e_n[0]|^2 P_MUSIC."""
    inst = synth.custom(6, 5, 2000, [-50.0, -20.0, 0.0, 20.0, 50.0], 10.0, 0.1, seed=21)
    R = oracle_mod.covariance(inst.X)
    ev, V, _ = oracle_mod.eigh(R)
    Ps = {}
    for alg in (PHD, MUSIC, EV, MN):
        C, st = oracle_mod.weighting(ev, V, 5, alg)
        assert st == 0
        Ps[alg], _ = oracle_mod.scan(C, inst.lo, inst.step, inst.L)
    np.testing.assert_allclose(Ps[PHD], Ps[MUSIC], rtol=1e-10)
    np.testing.assert_allclose(Ps[EV], ev[-1] * Ps[MUSIC], rtol=1e-10)
    np.testing.assert_allclose(Ps[MN], abs(V[0, -1]) ** 2 * Ps[MUSIC], rtol=1e-10)
    pk = [list(oracle_mod.peaks(Ps[a], 5)[0]) for a in (PHD, MUSIC, EV, MN)]
    assert pk[0] == pk[1] == pk[2] == pk[3]


def test_no_sources_flat_music(oracle_mod):
    inst = synth.custom(8, 0, 512, [], 0.0, 0.5, seed=4)
    res = oracle_mod.solve(inst.X, 0, MUSIC, inst.lo, inst.step, inst.L)
    assert res["status"] == 0
    np.testing.assert_allclose(res["P"], 1.0 / 8, rtol=1e-12)
    assert len(res["idx"]) == 0


def test_music_lower_bound_and_estimates(oracle_mod):
    """MUSIC: den = ||E_n^H a||^2 <= ||a||^2 = M, so P >= 1/M; the peaks land on the sources."""
    inst = synth.single_c1()
    for alg in (PHD, MUSIC, EV, MN):
        res = oracle_mod.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
        assert res["status"] == 0
        if alg == MUSIC:
            assert np.min(res["P"]) >= 1.0 / inst.M * (1 - 1e-12)
        est = inst.lo + res["idx"] * inst.step
        assert len(est) == 2
        np.testing.assert_allclose(est, inst.angles, atol=1.0 if alg == PHD else 0.3)


def test_solve_matches_stepwise(oracle_mod):
    inst = synth.custom(9, 3, 700, None, 12.0, 0.05, seed=33)
    R = oracle_mod.covariance(inst.X)
    ev, V, _ = oracle_mod.eigh(R)
    for alg in (PHD, MUSIC, EV, MN):
        C, _ = oracle_mod.weighting(ev, V, inst.d, alg)
        P, _ = oracle_mod.scan(C, inst.lo, inst.step, inst.L)
        res = oracle_mod.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
        np.testing.assert_array_equal(res["P"], P)
        np.testing.assert_array_equal(res["idx"], oracle_mod.peaks(P, inst.d)[0])
