"""Pins of the oracle's arbitrary-geometry azimuth x elevation scan (Eq. 2 as printed, Sec. 4.2's
circular array) and of its 2-D peak picking, against closed forms, symmetries and brute force.
"""
import math

import numpy as np
import pytest
from scipy import special

PHD, MUSIC, EV, MN = 0, 1, 2, 3


def _pair_C(M, i, j, kind):
    """Hermitian C with one pair of elements: 'diff' -> (e_i - e_j)(e_i - e_j)^H, 'sin' -> the
    imaginary antisymmetric pair j e_i e_j^H - j e_j e_i^H."""
    C = np.zeros((M, M), dtype=np.complex128)
    if kind == "diff":
        C[i, i] = C[j, j] = 1.0
        C[i, j] = C[j, i] = -1.0
    else:
        C[i, j] = 1j
        C[j, i] = -1j
    return C


def test_pair_differences_fix_each_axis(oracle_mod):
    """With C = (e_0 - e_1)(e_0 - e_1)^H, a^H C a = |a_0 - a_1|^2 = 4 sin^2(dphase / 2), where the phase
    difference is 2 pi h times the direction cosine of the axis the two elements differ along: x ->
    sin(theta) sin(phi), y -> cos(theta) sin(phi), z -> cos(phi) (Eq. 2)."""
    h = 0.37
    az = np.arange(-170.0, 180.0, 7.0)
    el = np.arange(3.0, 178.0, 11.0)
    T, F = np.meshgrid(np.deg2rad(az), np.deg2rad(el))
    cosines = {0: np.sin(T) * np.sin(F), 1: np.cos(T) * np.sin(F), 2: np.cos(F)}
    for axis, dc in cosines.items():
        pos = np.zeros((2, 3))
        pos[1, axis] = h
        P = oracle_mod.scan_geometry(_pair_C(2, 0, 1, "diff"), pos, az[0], 7.0, len(az), el[0], 11.0, len(el))
        want = 1.0 / (4.0 * np.sin(math.pi * h * dc) ** 2)
        np.testing.assert_allclose(P, want, rtol=1e-9)


def test_pair_sign_of_phase(oracle_mod):
    """C = j e_0 e_1^H - j e_1 e_0^H gives a^H C a = -2 sin(p_1 - p_0), so P is finite exactly where
    the second element leads in phase by less than pi, which pins the +j sign of Eq. 2: element 1 at
    +x h, phase p_1 - p_0 = +2 pi h sin(theta) sin(phi)."""
    h = 0.2
    pos = np.array([[0.0, 0.0, 0.0], [h, 0.0, 0.0]])
    az = np.arange(-179.0, 180.0, 2.0)
    P = oracle_mod.scan_geometry(_pair_C(2, 0, 1, "sin"), pos, az[0], 2.0, len(az), 90.0, 1.0, 1)[0]
    s = np.sin(2 * math.pi * h * np.sin(np.deg2rad(az)))
    for k in range(len(az)):
        if s[k] < -1e-12:
            assert P[k] == pytest.approx(1.0 / (-2.0 * s[k]), rel=1e-9)
        elif s[k] > 1e-12:
            assert P[k] == math.inf


@pytest.mark.parametrize("M,r", [(8, 0.5), (5, 0.83), (12, 0.31)])
def test_uca_sum_beam_is_the_jacobi_anger_series(oracle_mod, M, r):
    """For a uniform circular array (element m at angle 2 pi m / M from +y toward +x, radius r in
    wavelengths) the phase of element m is z cos(alpha_m - theta), z = 2 pi r sin(phi). With C = 1 1^H,
    a^H C a = |sum_m exp(j z cos(alpha_m - theta))|^2 and the Jacobi-Anger expansion collapses the sum
    to M sum_q j^(qM) J_(qM)(z) exp(-j q M theta)."""
    pos = oracle_mod.uca_positions(M, r)
    C = np.ones((M, M), dtype=np.complex128)
    az = np.arange(0.0, 360.0, 5.0)
    el = np.arange(1.0, 91.0, 8.0)
    P = oracle_mod.scan_geometry(C, pos, 0.0, 5.0, len(az), 1.0, 8.0, len(el))
    for l, phi in enumerate(el):
        z = 2 * math.pi * r * math.sin(math.radians(phi))
        th = np.deg2rad(az)
        s = np.zeros(len(az), dtype=np.complex128)
        for q in range(-6, 7):
            n = q * M
            s += (1j ** (n % 4)) * special.jv(n, z) * np.exp(-1j * n * th)
        want = 1.0 / np.abs(M * s) ** 2
        np.testing.assert_allclose(P[l], want, rtol=1e-9)


def test_uca_positions_are_a_regular_polygon(oracle_mod):
    pos = oracle_mod.uca_positions(8, 0.5)
    assert np.allclose(pos[:, 2], 0.0)
    assert np.allclose(np.hypot(pos[:, 0], pos[:, 1]), 0.5)
    assert np.allclose(pos[0], [0.0, 0.5, 0.0]) and np.allclose(pos[2], [0.5, 0.0, 0.0], atol=1e-15)
    d = np.linalg.norm(pos - np.roll(pos, 1, axis=0), axis=1)
    assert np.allclose(d, 2 * 0.5 * math.sin(math.pi / 8))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_line_array_reduces_to_the_ula_scan(oracle_mod, axis):
    """A half-wavelength line along x, seen in the plane phi = 90, is the ULA of Step-5 (phase
    pi m sin(theta)); along y at azimuth theta it is the ULA at 90 - theta; along z at elevation phi
    it is the ULA at 90 - phi, for any azimuth."""
    M = 6
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    C = Z @ Z.conj().T + np.eye(M)
    pos = np.zeros((M, 3))
    pos[:, axis] = 0.5 * np.arange(M)
    if axis == 0:
        P = oracle_mod.scan_geometry(C, pos, -60.0, 0.5, 241, 90.0, 1.0, 1)[0]
        ref, _ = oracle_mod.scan(C, -60.0, 0.5, 241)
    elif axis == 1:
        P = oracle_mod.scan_geometry(C, pos, 30.0, 0.5, 241, 90.0, 1.0, 1)[0]
        ref, _ = oracle_mod.scan(C, 60.0, -0.5, 241)
    else:
        P = oracle_mod.scan_geometry(C, pos, 17.0, 1.0, 1, 10.0, 0.5, 161)[:, 0]
        ref, _ = oracle_mod.scan(C, 80.0, -0.5, 161)
    np.testing.assert_allclose(P, ref, rtol=1e-10)


def test_uca_rotation_by_one_element(oracle_mod):
    """Rotating an M-element UCA by one element (360/M degrees of azimuth) permutes its steering
    vector cyclically: a(theta + 360/M) = S a(theta) with (S a)_m = a_(m-1). So the spectrum of
    S^H C S equals the spectrum of C shifted by 360/M degrees."""
    M = 8
    pos = oracle_mod.uca_positions(M, 0.5)
    rng = np.random.default_rng(9)
    Z = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    C = Z @ Z.conj().T + 0.1 * np.eye(M)
    S = np.roll(np.eye(M), 1, axis=0)          # S e_m = e_(m+1): (S a)_m = a_(m-1)
    P = oracle_mod.scan_geometry(C, pos, 0.0, 1.0, 360, 10.0, 10.0, 9)
    Q = oracle_mod.scan_geometry(S.conj().T @ C @ S, pos, 0.0, 1.0, 360, 10.0, 10.0, 9)
    np.testing.assert_allclose(Q, np.roll(P, -45, axis=1), rtol=1e-9)


def test_uca_plane_symmetry_in_elevation(oracle_mod):
    """A planar array in z = 0 cannot tell phi from 180 - phi: the spectrum is symmetric about 90."""
    M = 8
    pos = oracle_mod.uca_positions(M, 0.5)
    rng = np.random.default_rng(2)
    Z = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    C = Z @ Z.conj().T
    P = oracle_mod.scan_geometry(C, pos, 0.0, 3.0, 120, 10.0, 1.0, 161)   # phi = 10 .. 170
    np.testing.assert_allclose(P, P[::-1], rtol=1e-10)


@pytest.mark.parametrize("alg", [PHD, MUSIC, EV, MN])
def test_uca_exact_covariance_nulls_at_the_sources(oracle_mod, alg):
    """R = A diag(p) A^H + sigma^2 I for two sources on grid points of the 8-element UCA (radius
    lambda/2): the noise subspace is orthogonal to both steering vectors, so invP vanishes there up
    to rounding (P above 1e10 against an O(1) background) and the two largest 2-D peaks are exactly
    the two source cells."""
    M = 8
    pos = oracle_mod.uca_positions(M, 0.5)
    src = [(37.0, 61.0), (250.0, 25.0)]
    A = np.stack([oracle_mod.steering_geometry(pos, t, f) for t, f in src], axis=1)
    R = A @ np.diag([1.0, 0.6]) @ A.conj().T + 0.05 * np.eye(M)
    ev, V, sweeps = oracle_mod.eigh(R)
    assert sweeps > 0
    C, st = oracle_mod.weighting(ev, V, 2, alg)
    assert st == 0
    P = oracle_mod.scan_geometry(C, pos, 0.0, 1.0, 360, 1.0, 1.0, 90)
    cells = sorted((int(round(f - 1.0)) * 360 + int(round(t))) for t, f in src)
    for c in cells:
        assert P.flat[c] > 1e10
    idx, val = oracle_mod.peaks2d(P, 2, wrap_az=True)
    if alg == PHD:
        # one noise vector: a^H v = 0 is two real equations in (theta, phi), so it can vanish at
        # other isolated directions too; both source cells must still be strict 2-D maxima
        idx_all, _ = oracle_mod.peaks2d(P, 1000, wrap_az=True)
        assert set(cells) <= set(idx_all)
    else:
        assert list(idx) == cells


# ------------------------------------------------------------------------------ 2-D Step-6
def _brute_peaks2d(P, D, wrap):
    Le, La = P.shape
    cand = []
    for l in range(Le):
        for k in range(La):
            nb = []
            for dl in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    if dl == 0 and dk == 0:
                        continue
                    ll, kk = l + dl, k + dk
                    if not 0 <= ll < Le:
                        continue
                    if not 0 <= kk < La:
                        if not wrap:
                            continue
                        kk %= La
                    nb.append(P[ll, kk])
            if nb and all(x < P[l, k] for x in nb):
                cand.append((-P[l, k], l * La + k))
    cand.sort()
    pick = sorted(c[1] for c in cand[:D])
    return pick


def test_peaks2d_hand_cases(oracle_mod):
    P = np.zeros((3, 5))
    P[1, 1] = 5.0
    P[0, 4] = 4.0         # corner: neighbours (0,3), (1,3), (1,4) and, wrapped, (0,0), (1,0)
    P[2, 3] = 3.0         # bottom row: only the rows that exist are compared
    idx, val = oracle_mod.peaks2d(P, 5, wrap_az=False)
    assert list(idx) == [4, 6, 13] and list(val) == [4.0, 5.0, 3.0]
    assert list(oracle_mod.peaks2d(P, 2, wrap_az=False)[0]) == [4, 6]
    P2 = P.copy()
    P2[1, 0] = 4.5        # next to (1,1) = 5, and (wrapped) next to the corner (0,4) = 4
    idx, _ = oracle_mod.peaks2d(P2, 5, wrap_az=True)
    assert list(idx) == [6, 13]
    idx, _ = oracle_mod.peaks2d(P2, 5, wrap_az=False)
    assert list(idx) == [4, 6, 13]
    # plateau of two equal cells: neither is strictly larger than the other
    Q = np.zeros((3, 5))
    Q[1, 2] = Q[1, 3] = 2.0
    assert len(oracle_mod.peaks2d(Q, 3, wrap_az=False)[0]) == 0
    # a flat spectrum has no peak, a single point has no neighbour, D = 0 selects nothing
    assert len(oracle_mod.peaks2d(np.ones((4, 4)), 3, True)[0]) == 0
    assert len(oracle_mod.peaks2d(np.ones((1, 1)), 3, True)[0]) == 0
    assert len(oracle_mod.peaks2d(P, 0, False)[0]) == 0
    # one row with wrap is the circular 1-D rule
    row = np.array([[3.0, 1.0, 2.0, 1.0, 2.5]])
    assert list(oracle_mod.peaks2d(row, 4, True)[0]) == [0, 2]
    assert list(oracle_mod.peaks2d(row, 4, False)[0]) == [0, 2, 4]
    # equal peaks: the lower flat index wins the last slot
    T = np.zeros((3, 7))
    T[0, 1] = T[2, 5] = T[1, 3] = 1.0
    assert list(oracle_mod.peaks2d(T, 2, False)[0]) == [1, 10]


@pytest.mark.parametrize("seed", range(12))
def test_peaks2d_brute_force_random(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    Le, La = rng.integers(1, 9), rng.integers(1, 13)
    P = rng.integers(0, 4, size=(Le, La)).astype(np.float64)   # many ties
    for wrap in (False, True):
        for D in (0, 1, 3, 50):
            idx, val = oracle_mod.peaks2d(P, D, wrap)
            assert list(idx) == _brute_peaks2d(P, D, wrap)
            assert np.array_equal(val, P.flat[idx])


def test_solve_geometry_matches_steps(oracle_mod):
    from paper_2007_14135_gb300 import synth
    M = 8
    pos = oracle_mod.uca_positions(M, 0.5)
    rng = np.random.default_rng(4)
    X = (rng.standard_normal((M, 300)) + 1j * rng.standard_normal((M, 300))).astype(np.complex64)
    out = oracle_mod.solve_geometry(X, 2, MUSIC, pos, 0.0, 4.0, 90, 5.0, 10.0, 9, True)
    R = oracle_mod.covariance(X)
    ev, V, _ = oracle_mod.eigh(R)
    C, _ = oracle_mod.weighting(ev, V, 2, MUSIC)
    P = oracle_mod.scan_geometry(C, pos, 0.0, 4.0, 90, 5.0, 10.0, 9)
    assert np.array_equal(out["P"], P)
    assert list(out["idx"]) == list(oracle_mod.peaks2d(P, 2, True)[0])
    del synth
