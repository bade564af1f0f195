"""Autotuner cache keys (host logic, no GPU): one key per occupied M bucket, with the size class
and the scan kind, where 2-D problems that share a steering table (one positions pointer, grid
and M, as the plan decides) are their own kind."""
import pytest


@pytest.fixture(scope="module")
def mods():
    from paper_2007_14135_gb300 import autotune, build, doa
    build.build()
    return autotune, doa


def _prob(doa, M=8, L=360, Le=0, pos=0):
    p = doa.Problem()
    p.M, p.N, p.ldx, p.d, p.alg_mask = M, 1024, 1024, 2, 1 << doa.MUSIC
    p.grid = doa.grid(0.0, 1.0, L)
    if pos:
        p.geom = doa.Geometry(pos, 1.0, 1.0, Le, 1)
    return p


def test_keys_scan_kinds(mods):
    autotune, doa = mods
    ula = [_prob(doa, M=16, L=18001) for _ in range(40)]
    k = autotune._keys(ula, None, gpu_name="GB300 test")
    assert k == {1: "GB300_test|M1|n1e2|L1e4|ula"}
    own = [_prob(doa, Le=90, pos=0x1000 + 64 * i) for i in range(4096)]
    assert autotune._keys(own, None, gpu_name="g")[0].endswith("|n1e4|L1e5|geo")      # 32 400 points
    shared = [_prob(doa, Le=90, pos=0x1000) for _ in range(4096)]
    assert autotune._keys(shared, None, gpu_name="g")[0].endswith("|n1e4|L1e5|geotab")
    mixed = shared[:2] + own[:2] + ula[:1]
    k = autotune._keys(mixed, None, gpu_name="g")
    assert k[0].endswith("|geo+geotab") and k[1].endswith("|ula")
    # one pointer, different grids or M: no sharing
    split = [_prob(doa, Le=90, pos=0x1000), _prob(doa, Le=45, pos=0x1000), _prob(doa, M=7, Le=90, pos=0x1000)]
    assert autotune._keys(split, None, gpu_name="g")[0].endswith("|geo")
