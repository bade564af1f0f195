"""Pins of the oracle's MDL / AIC model-order estimates (Wax & Kailath's criteria) against
invariants, the AM-GM bound, a product-form restatement and exact-covariance structure."""
import math

import numpy as np
import pytest

from paper_2007_14135_gb300 import synth


def _L_product_form(ev, N, k):
    """The log-likelihood term as the ratio of the noise eigenvalues' determinant to their mean
    raised to their count (equal to N (M-k) log(a/g))."""
    tail = np.asarray(ev[k:], dtype=np.float64)
    n = len(tail)
    return -N * math.log(np.prod(tail / tail.mean()))


@pytest.mark.parametrize("seed", range(6))
def test_criteria_values(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(2, 20))
    N = int(rng.integers(M, 5000))
    ev = np.sort(rng.uniform(0.1, 10.0, size=M))[::-1]
    mdl, aic, mv, av = oracle_mod.model_order(ev, N)
    for k in range(M):
        L = _L_product_form(ev, N, k)
        assert L >= -1e-9                      # AM-GM
        pen = k * (2 * M - k)
        assert mv[k] == pytest.approx(L + 0.5 * pen * math.log(N), rel=1e-10, abs=1e-9)
        assert av[k] == pytest.approx(2 * L + 2 * pen, rel=1e-10, abs=1e-9)
    assert mdl == int(np.argmin(mv)) and aic == int(np.argmin(av))
    assert mv[M - 1] == pytest.approx(0.5 * (M - 1) * (M + 1) * math.log(N))   # one noise eigenvalue: L = 0


def test_scale_invariance_and_equal_tail(oracle_mod):
    ev = np.array([9.0, 4.0, 1.0, 1.0, 1.0, 1.0])
    for c in (1e-6, 1.0, 3.7, 1e5):
        mdl, aic, mv, _ = oracle_mod.model_order(c * ev, 1000)
        assert (mdl, aic) == (2, 2)
        assert mv[2] == pytest.approx(0.5 * 2 * 10 * math.log(1000))            # equal tail: L(2) = 0
    # everything equal: no source
    assert oracle_mod.model_order(np.ones(5), 100)[:2] == (0, 0)


def test_exact_covariance_structure_gives_d(oracle_mod):
    """R = A P A^H + s^2 I has d signal eigenvalues above M - d equal ones; with many snapshots both
    criteria return d."""
    for M, d in [(8, 2), (16, 4), (12, 1), (32, 7)]:
        m = np.arange(M)[:, None]
        ang = np.linspace(-50, 50, d)
        A = np.exp(1j * np.pi * m * np.sin(np.radians(ang))[None, :])
        R = A @ np.diag(np.linspace(1.0, 0.3, d)) @ A.conj().T + 0.1 * np.eye(M)
        ev, _, _ = oracle_mod.eigh(R)
        assert oracle_mod.model_order(ev, 4096)[:2] == (d, d)


def test_nonpositive_noise_eigenvalue(oracle_mod):
    """A zero eigenvalue (rank-deficient R, N < M) is in every noise tail: every criterion is +inf
    and the estimate falls back to the first k, 0."""
    ev = np.array([5.0, 2.0, 1.0, 0.0])
    mdl, aic, mv, av = oracle_mod.model_order(ev, 50)
    assert np.all(np.isinf(mv)) and np.all(np.isinf(av)) and (mdl, aic) == (0, 0)


def test_high_snr_snapshots(oracle_mod):
    """Sample covariances of well separated sources at 20 dB: MDL finds d."""
    for seed, (M, d) in enumerate([(8, 2), (16, 4), (12, 3)]):
        inst = synth.custom(M, d, 4096, None, 20.0, 1.0, seed=700 + seed)
        ev, _, _ = oracle_mod.eigh(oracle_mod.covariance(inst.X))
        assert oracle_mod.model_order(ev, inst.N)[0] == d
