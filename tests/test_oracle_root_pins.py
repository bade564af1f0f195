"""Pins of the oracle's root form of the ULA scan (root-MUSIC): the polynomial reproduces the scan's
denominator on the unit circle, its roots pair up as z, 1/conj(z), and the selected roots recover
the sources of exact covariances and the two-element closed form."""
import math

import numpy as np
import pytest

from paper_2007_14135_gb300 import synth

PHD, MUSIC, EV, MN = 0, 1, 2, 3


def _ula(M, theta_deg):
    return np.exp(1j * math.pi * np.arange(M) * math.sin(math.radians(theta_deg)))


@pytest.mark.parametrize("alg", [PHD, MUSIC, EV, MN])
def test_polynomial_is_the_scan_denominator(oracle_mod, alg):
    inst = synth.custom(12, 3, 2000, None, 10.0, 0.37, seed=91)
    ev, V, _ = oracle_mod.eigh(oracle_mod.covariance(inst.X))
    C, _ = oracle_mod.weighting(ev, V, 3, alg)
    coef = oracle_mod.root_polynomial(C)
    P, _ = oracle_mod.scan(C, inst.lo, inst.step, inst.L)
    th = np.radians(inst.lo + np.arange(inst.L) * inst.step)
    z = np.exp(1j * np.pi * np.sin(th))
    D = np.polyval(coef, z) * z ** (-(12 - 1))
    np.testing.assert_allclose(D.real, 1.0 / P, rtol=1e-9)
    assert np.max(np.abs(D.imag)) < 1e-9 * np.max(np.abs(D.real))


def test_roots_pair_up(oracle_mod):
    inst = synth.custom(10, 2, 500, None, 5.0, 1.0, seed=92)
    ev, V, _ = oracle_mod.eigh(oracle_mod.covariance(inst.X))
    C, _ = oracle_mod.weighting(ev, V, 2, MUSIC)
    r = np.roots(oracle_mod.root_polynomial(C))
    assert len(r) == 18
    partners = 1.0 / np.conj(r)
    for p in partners:
        assert np.min(np.abs(r - p)) < 1e-8 * max(1.0, abs(p))
    assert np.sum(np.abs(r) <= 1.0) == 9


@pytest.mark.parametrize("M,ang", [(8, [-20.137, 35.4219]), (16, [-41.3, -7.77, 12.05, 50.5]), (6, [3.3])])
@pytest.mark.parametrize("alg", [MUSIC, EV, PHD, MN])
def test_exact_covariance_roots_on_the_sources(oracle_mod, M, ang, alg):
    d = len(ang)
    A = np.stack([_ula(M, t) for t in ang], axis=1)
    R = A @ np.diag(np.linspace(1.0, 0.5, d)) @ A.conj().T + 0.1 * np.eye(M)
    ev, V, _ = oracle_mod.eigh(R)
    C, _ = oracle_mod.weighting(ev, V, d, alg)
    got, roots = oracle_mod.root_music(C, d)
    if alg in (PHD, MN) and M - d > 1:
        # one noise vector: its polynomial also has roots off the sources, maybe nearer the circle;
        # every source is still a (double) root on the circle
        r = np.roots(oracle_mod.root_polynomial(C))
        for t in ang:
            zt = np.exp(1j * np.pi * math.sin(math.radians(t)))
            assert np.min(np.abs(r - zt)) < 1e-6
        return
    np.testing.assert_allclose(got, sorted(ang), rtol=0, atol=1e-5)     # double roots: ~sqrt(eps)
    assert np.all(np.abs(np.abs(roots) - 1.0) < 1e-6)


def test_two_element_closed_form(oracle_mod):
    """C = u u^H, u = (1, -e^{j psi}): z D(z) = -e^{-j psi} (z - e^{j psi})^2, a double root at
    e^{j psi}, so theta = asin(psi / pi)."""
    for psi in (-2.5, -0.3, 0.8, 2.2):
        u = np.array([1.0, -np.exp(1j * psi)])
        C = np.outer(u, u.conj())
        coef = oracle_mod.root_polynomial(C)
        np.testing.assert_allclose(coef, [-np.exp(-1j * psi), 2.0, -np.exp(1j * psi)], atol=1e-15)
        got, _ = oracle_mod.root_music(C, 1)
        assert abs(got[0] - math.degrees(math.asin(psi / math.pi))) < 1e-6


def test_root_music_near_the_scan_peaks(oracle_mod):
    """At high SNR the root estimates sit within a grid step of the MUSIC scan's peaks."""
    inst = synth.custom(16, 4, 4096, None, 20.0, 0.01, seed=93)
    ev, V, _ = oracle_mod.eigh(oracle_mod.covariance(inst.X))
    C, _ = oracle_mod.weighting(ev, V, 4, MUSIC)
    P, _ = oracle_mod.scan(C, inst.lo, inst.step, inst.L)
    idx, _ = oracle_mod.peaks(P, 4)
    got, _ = oracle_mod.root_music(C, 4)
    np.testing.assert_allclose(got, np.sort(inst.lo + idx * inst.step), atol=2 * inst.step)
