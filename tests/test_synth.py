"""The seeded generator follows the signal model of Eq. 1 (checked on CPU)."""
import numpy as np

from paper_2007_14135_gb300 import synth


def test_separated_angles():
    rng = np.random.default_rng(0)
    for d, sep in [(1, 5.0), (4, 5.0), (16, 5.0), (8, 1.0), (6, 3.0)]:
        for _ in range(50):
            a = synth.draw_angles(rng, d, -60.0, 60.0, sep)
            assert len(a) == d and np.all(a >= -60.0) and np.all(a <= 60.0)
            assert d < 2 or np.min(np.diff(a)) >= sep - 1e-12


def test_reproducible_and_distinct():
    a = synth.paper_density(3).X
    b = synth.paper_density(3).X
    c = synth.paper_density(4).X
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    X, meta = synth.paper_density_batch(3)
    assert np.array_equal(X[2], synth.paper_density(2).X)


def test_snapshot_statistics_match_model():
    """E[X X^H / N] = A A^H + sigma^2 I for unit-power uncorrelated sources (Eq. 1)."""
    M, N, ang, snr = 6, 200000, [-30.0, 10.0], 5.0
    inst = synth.custom(M, 2, N, ang, snr, 1.0, seed=77)
    X = inst.X.astype(np.complex128)
    R = X @ X.conj().T / N
    m = np.arange(M)[:, None]
    A = np.exp(1j * np.pi * m * np.sin(np.radians(ang))[None, :])
    Rt = A @ A.conj().T + 10 ** (-snr / 10) * np.eye(M)
    assert np.max(np.abs(R - Rt)) < 6 * np.sqrt(2.0 / N) * np.max(np.abs(Rt))
