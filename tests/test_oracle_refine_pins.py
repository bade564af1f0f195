"""Pins of the oracle's sub-grid peak refinement (the local minimiser of a^H C a next to a picked
grid peak), against closed forms and exact covariances with off-grid sources."""
import math

import numpy as np
import pytest

PHD, MUSIC, EV, MN = 0, 1, 2, 3


def _ula(M, theta_deg):
    m = np.arange(M)
    return np.exp(1j * math.pi * m * math.sin(math.radians(theta_deg)))


@pytest.mark.parametrize("M,ang,step", [(8, [-20.137, 35.4219], 0.1), (16, [-41.3, -7.77, 12.05, 50.5], 0.05),
                                        (5, [10.123], 1.0), (12, [-60.01, 0.003, 44.444], 0.2)])
@pytest.mark.parametrize("alg", [PHD, MUSIC, EV, MN])
def test_refine_recovers_off_grid_sources_of_an_exact_covariance(oracle_mod, M, ang, step, alg):
    """R = A P A^H + s^2 I: the noise subspace is orthogonal to every a(theta_i), so den vanishes
    (a double zero) exactly at the true angles, which lie between grid points; the refinement
    from the grid peak next to each must land on the true angle to 1e-9 degree."""
    d = len(ang)
    A = np.stack([_ula(M, t) for t in ang], axis=1)
    R = A @ np.diag(np.linspace(1.0, 0.5, d)) @ A.conj().T + 0.1 * np.eye(M)
    ev, V, _ = oracle_mod.eigh(R)
    C, st = oracle_mod.weighting(ev, V, d, alg)
    assert st == 0
    L = int(round(180.0 / step)) + 1
    P, _ = oracle_mod.scan(C, -90.0, step, L)
    idx, _ = oracle_mod.peaks(P, d)
    if alg == PHD and M - d > 1:
        # one noise vector also vanishes elsewhere: check only the peaks next to the sources
        idx = [k for k in oracle_mod.peaks(P, M - 1)[0] if min(abs(-90.0 + k * step - t) for t in ang) < step]
    got = sorted(oracle_mod.refine_peak(C, -90.0, step, int(k))[0] for k in idx)
    assert len(got) == d
    np.testing.assert_allclose(got, sorted(ang), rtol=0, atol=1e-9)


def test_refine_two_element_closed_form(oracle_mod):
    """M = 2, C = u u^H with u = (1, -e^{j psi}): a^H C a = 4 sin^2((pi sin(theta) - psi) / 2), whose
    minimiser is theta* = asin(psi / pi) (pins the steering sign, the chain rule through sin theta
    and the Newton update)."""
    for psi in (-2.1, -0.4, 0.3, 1.234, 2.9):
        u = np.array([1.0, -np.exp(1j * psi)])
        C = np.outer(u, u.conj())
        want = math.degrees(math.asin(psi / math.pi))
        step = 0.5
        k = int(round((want + 90.0) / step))
        got, it = oracle_mod.refine_peak(C, -90.0, step, k)
        assert abs(got - want) < 1e-10, (psi, got, want)
        assert it <= 10


def test_refine_is_a_stationary_point_inside_its_bracket(oracle_mod):
    """On a noisy covariance the refined angle is where den' = 0 (central difference), lies within
    one grid step of the peak, and has den no larger than at the grid peak."""
    rng = np.random.default_rng(3)
    M = 10
    X = (rng.standard_normal((M, 300)) + 1j * rng.standard_normal((M, 300))).astype(np.complex64)
    A = np.stack([_ula(M, t) for t in (-30.3, 22.2)], axis=1)
    X = (X + 3 * A @ (rng.standard_normal((2, 300)) + 1j * rng.standard_normal((2, 300)))).astype(np.complex64)
    R = oracle_mod.covariance(X)
    ev, V, _ = oracle_mod.eigh(R)
    C, _ = oracle_mod.weighting(ev, V, 2, MUSIC)
    step = 0.1
    P, _ = oracle_mod.scan(C, -90.0, step, 1801)
    idx, _ = oracle_mod.peaks(P, 2)

    def den(t):
        a = _ula(M, t)
        return float(np.real(a.conj() @ C @ a))

    for k in idx:
        th, _ = oracle_mod.refine_peak(C, -90.0, step, int(k))
        grid = -90.0 + k * step
        assert abs(th - grid) <= step
        h = 1e-6
        deriv = (den(th + h) - den(th - h)) / (2 * h)
        curv = (den(th + h) - 2 * den(th) + den(th - h)) / h ** 2
        assert abs(deriv) < 1e-6 * curv
        assert den(th) <= den(grid)


@pytest.mark.parametrize("alg", [MUSIC, EV])
@pytest.mark.parametrize("geometry", ["uca8", "random3d"])
def test_refine2d_recovers_off_grid_sources(oracle_mod, alg, geometry):
    rng = np.random.default_rng(12)
    pos = oracle_mod.uca_positions(8, 0.5) if geometry == "uca8" else rng.uniform(-1, 1, size=(9, 3))
    M = pos.shape[0]
    src = [(37.3, 61.7), (250.6, 25.2)]
    A = np.stack([oracle_mod.steering_geometry(pos, t, f) for t, f in src], axis=1)
    R = A @ np.diag([1.0, 0.6]) @ A.conj().T + 0.05 * np.eye(M)
    ev, V, _ = oracle_mod.eigh(R)
    C, _ = oracle_mod.weighting(ev, V, 2, alg)
    P = oracle_mod.scan_geometry(C, pos, 0.0, 1.0, 360, 1.0, 1.0, 90)
    idx, _ = oracle_mod.peaks2d(P, 2, True)
    got = sorted(oracle_mod.refine_peak2d(C, pos, 0.0, 1.0, 360, 1.0, 1.0, int(i))[0] for i in idx)
    np.testing.assert_allclose(np.array(got), np.array(sorted(src)), rtol=0, atol=1e-9)


def test_refine2d_closed_form_three_elements(oracle_mod):
    """Elements at the origin, at +x h and at +y h, C = u1 u1^H + u2 u2^H with u1 = e0 - e^{j psi1} e1,
    u2 = e0 - e^{j psi2} e2: den = 4 sin^2((2 pi h u_x - psi1)/2) + 4 sin^2((2 pi h u_y - psi2)/2)
    vanishes where h sin(theta) sin(phi) = psi1 / 2pi and h cos(theta) sin(phi) = psi2 / 2pi."""
    h = 0.45
    pos = np.array([[0.0, 0.0, 0.0], [h, 0.0, 0.0], [0.0, h, 0.0]])
    for psi1, psi2 in [(0.9, 1.3), (-1.1, 0.4), (0.2, -1.7)]:
        u1 = np.array([1.0, -np.exp(1j * psi1), 0.0])
        u2 = np.array([1.0, 0.0, -np.exp(1j * psi2)])
        C = np.outer(u1, u1.conj()) + np.outer(u2, u2.conj())
        th = math.degrees(math.atan2(psi1, psi2)) % 360.0
        ph = math.degrees(math.asin(math.hypot(psi1, psi2) / (2 * math.pi * h)))
        k, l = int(round(th / 2.0)), int(round((ph - 1.0) / 2.0))
        (gt, gp), _ = oracle_mod.refine_peak2d(C, pos, 0.0, 2.0, 180, 1.0, 2.0, l * 180 + k)
        assert abs(gt - th) < 1e-9 and abs(gp - ph) < 1e-9, (psi1, psi2, gt, th, gp, ph)


def test_refine2d_stays_in_its_box(oracle_mod):
    """A minimum outside the box: the result is clamped to the box edge, one step from the start."""
    h = 0.45
    pos = np.array([[0.0, 0.0, 0.0], [h, 0.0, 0.0], [0.0, h, 0.0]])
    u1 = np.array([1.0, -np.exp(0.9j), 0.0])
    u2 = np.array([1.0, 0.0, -np.exp(1.3j)])
    C = np.outer(u1, u1.conj()) + np.outer(u2, u2.conj())
    th_true = math.degrees(math.atan2(0.9, 1.3))
    k = int(round(th_true / 2.0)) + 3          # start three azimuth steps away
    ph = math.degrees(math.asin(math.hypot(0.9, 1.3) / (2 * math.pi * h)))
    l = int(round((ph - 1.0) / 2.0))
    (gt, _), _ = oracle_mod.refine_peak2d(C, pos, 0.0, 2.0, 180, 1.0, 2.0, l * 180 + k)
    assert abs(gt - (2.0 * k - 2.0)) < 1e-12
