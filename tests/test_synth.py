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


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 published with Random123 (Salmon et al., SC'11)."""
    from tests.philox_ref import philox4x32_10
    assert philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2) == [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]
    assert philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0]) == \
        [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_proposal_params_ranges():
    d, ang, snr = synth.proposal_params(5000, 3)
    assert d.min() >= 1 and d.max() <= 6 and snr.min() >= -5 and snr.max() <= 20
    for i in range(200):
        a = ang[i, :d[i]]
        assert np.all(a >= -80) and np.all(a <= 80) and (d[i] < 2 or np.min(np.diff(a)) >= 3 - 1e-4)
        assert np.all(ang[i, d[i]:] == 0)
