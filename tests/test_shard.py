"""Splitting over ranks, on the CPU: partitions, the host merge of grid-slice peak summaries
against the oracle's Step-6 on the whole spectrum, and the exchange over a world of two gloo
ranks. The slice summaries here come from `_summary`, a direct restatement of the slice rule
(the GPU kernel that produces them is compared with doa_peaks in the GPU tests)."""
import os
import socket

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def libdoa():
    from paper_2007_14135_gb300 import build
    build.build()
    from paper_2007_14135_gb300 import doa
    return doa


def _summary(doa, P, k0, k1, d):
    """Peak summary of the slice [k0, k1) of P seen through its halo (doa_slice_peaks' contract)."""
    L = len(P)
    limit = min(k1 + 1, L) - 1
    decided, open_ = [], None
    for i in range(max(k0, 1), min(k1, L - 1)):
        v = P[i]
        if not P[i - 1] < v:
            continue
        j = i
        while j + 1 <= limit and P[j + 1] == v:
            j += 1
        if j + 1 <= limit:
            if P[j + 1] < v:
                decided.append((v, i))
        elif limit < L - 1:
            open_ = (i, v)
    decided.sort(key=lambda c: (-c[0], c[1]))
    decided = decided[:d]
    s = doa.SliceSummary()
    s.count = len(decided)
    for q, (v, i) in enumerate(decided):
        s.idx[q] = i
        s.val[q] = v
    s.open_idx, s.open_val = (open_[0], open_[1]) if open_ else (-1, 0.0)
    v0, k = P[k0], k0
    while k + 1 <= limit and P[k + 1] == v0:
        k += 1
    s.first_val = v0
    s.first_run_to_end = int(k + 1 > limit)
    s.first_next_val = P[k + 1] if k + 1 <= limit else 0.0
    return s


def _spectra():
    rng = np.random.default_rng(7)
    out = []
    for L in (3, 4, 9, 40, 257):
        out.append(rng.random(L).astype(np.float32))
        out.append(np.round(rng.random(L) * 4).astype(np.float32))              # many plateaus
    walk = np.cumsum(rng.choice([-1.0, 0.0, 0.0, 1.0], size=600)).astype(np.float32)
    out.append(walk)                                                            # long plateaus
    out.append(np.full(100, 0.0625, np.float32))                                # flat: no peak
    step = np.zeros(120, np.float32)
    step[30:90] = 2.0                                                           # one wide plateau
    out.append(step)
    tri = np.concatenate([np.arange(50), np.arange(50)[::-1]]).astype(np.float32)
    out.append(tri)
    return out


def test_shard_range_partitions():
    from paper_2007_14135_gb300.shard import shard_range, slice_bounds
    for n in (0, 1, 5, 17, 18001):
        for world in (1, 2, 3, 7, 8):
            parts = [shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1
    assert slice_bounds(10, 0, 2) == (0, 5, 0, 6) and slice_bounds(10, 1, 2) == (5, 10, 4, 10)
    with pytest.raises(ValueError):
        shard_range(5, 2, 2)


@pytest.mark.parametrize("d", [0, 1, 3, 8])
def test_merge_of_slices_equals_whole_spectrum_peaks(libdoa, d):
    from paper_2007_14135_gb300.shard import shard_range
    for P in _spectra():
        L = len(P)
        want_i, want_v = oracle.peaks(P.astype(np.float64), d)
        for world in range(1, min(L, 7) + 1):
            sums = []
            for r in range(world):
                k0, k1 = shard_range(L, r, world)
                sums.append(_summary(libdoa, P, k0, k1, d))
            got_i, got_v = libdoa.doa_merge_slices(sums, d)
            assert list(got_i) == list(want_i), (L, world, d, got_i, want_i)
            assert np.array_equal(got_v.astype(np.float64), want_v)


def test_merge_rejects_broken_chain(libdoa):
    P = np.array([0, 1, 2, 2, 2, 2, 1, 0], np.float32)
    a = _summary(libdoa, P, 0, 3, 2)
    assert a.open_idx == 2
    b = _summary(libdoa, P, 3, 8, 2)
    b.first_val = 5.0
    with pytest.raises(libdoa.DoaError):
        libdoa.doa_merge_slices([a, b], 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, P, d, want):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2007_14135_gb300 import doa, shard
        k0, k1 = shard.shard_range(len(P), rank, world)
        s = _summary(doa, P, k0, k1, d)
        raw = bytes(memoryview(s))
        local = torch.frombuffer(bytearray(raw), dtype=torch.uint8).clone()
        sums = shard.gather_summaries(local)
        assert len(sums) == world
        idx, val = shard.merge(sums, d)
        assert list(idx) == list(want), (rank, idx, want)
        assert shard.max_over_ranks(rank + 1.5) == world + 0.5
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_merge(libdoa):
    import torch.multiprocessing as mp
    rng = np.random.default_rng(3)
    P = np.round(rng.random(301) * 6).astype(np.float32)
    d = 5
    want, _ = oracle.peaks(P.astype(np.float64), d)
    mp.start_processes(_rank_main, args=(2, _free_port(), P, d, list(want)), nprocs=2, join=True,
                       start_method="spawn")
