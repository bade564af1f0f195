"""Seeded synthetic array snapshots (the signal model of Sec. 3.1, Eq. 1 and Table 1).

This module only generates inputs; it holds none of the estimation method's arithmetic
(no covariance, decomposition, spectrum or peak code). Both the CUDA path and the FP64
oracle consume exactly the complex64 bytes produced here.

Model (Eq. 1): X(t) = A(theta) S(t) + W(t) for a half-wavelength uniform linear array of M
omnidirectional elements on the x axis (Eq. 2 with x_m = m lambda/2, y = z = 0, phi = 90 deg),
so the array response of source i is exp(+j pi m sin(theta_i)), m = 0..M-1.
Sources are unit-power circular complex Gaussian, s ~ CN(0, 1) = (g1 + j g2)/sqrt(2), mutually
independent (uncorrelated narrowband sources); noise is white CN(0, sigma^2) per element with
sigma^2 = 10^(-SNR/10), one SNR per instance shared by all sources.

Other geometries (Sec. 4.2's uniform circular array) use Eq. 2 as printed: element positions
(x_m, y_m, z_m) in wavelengths and a source at azimuth theta, elevation angle phi has response
exp{j 2 pi (x_m sin(theta) sin(phi) + y_m cos(theta) sin(phi) + z_m cos(phi))}.

Random numbers come from NumPy's Philox4x32-10 counter-based generator (Salmon et al.,
SC'11) keyed by the instance seed, so every instance is reproducible on any machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GRID_LO = -90.0
GRID_HI = 90.0


def grid_size(step: float, lo: float = GRID_LO, hi: float = GRID_HI) -> int:
    """Number of points of the grid lo:step:hi (inclusive)."""
    return int(round((hi - lo) / step)) + 1


@dataclasses.dataclass
class Instance:
    """One snapshot matrix with its ground truth and its scan grid."""
    X: np.ndarray            # complex64 (M, N), row-major: row m = time series of element m
    M: int
    d: int
    N: int
    angles: np.ndarray       # true DOAs in degrees, ascending
    snr_db: float
    lo: float                # scan grid theta_k = lo + k*step, k = 0..L-1
    step: float
    L: int
    seed: int
    alg: int = 1             # algorithm for single-algorithm workloads (0 PHD, 1 MUSIC, 2 EV, 3 MN)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _source_response(M: int, angles_deg: Sequence[float]) -> np.ndarray:
    """Array response of the sources, (M, d) complex128: exp(j pi m sin(theta_i))."""
    m = np.arange(M, dtype=np.float64)[:, None]
    s = np.sin(np.deg2rad(np.asarray(angles_deg, dtype=np.float64)))[None, :]
    return np.exp(1j * np.pi * m * s)


def draw_angles(rng: np.random.Generator, d: int, lo: float, hi: float, min_sep: float) -> np.ndarray:
    """d angles uniform over {theta in [lo, hi]^d : sorted gaps >= min_sep}: sorted uniforms on
    [lo, hi - (d-1) min_sep] shifted by i*min_sep (a bijection onto the separated set that keeps
    the distribution uniform)."""
    if d == 0:
        return np.zeros(0)
    span = hi - lo - (d - 1) * min_sep
    if span < 0:
        raise ValueError("cannot place d separated angles in the range")
    u = np.sort(rng.uniform(0.0, span, size=d))
    return lo + u + min_sep * np.arange(d)


def snapshots(rng: np.random.Generator, M: int, N: int, angles_deg: Sequence[float],
              snr_db: float) -> np.ndarray:
    """X = A S + W as complex64 (M, N)."""
    d = len(angles_deg)
    sigma = math.sqrt(10.0 ** (-snr_db / 10.0))
    inv_sqrt2 = 1.0 / math.sqrt(2.0)
    if d > 0:
        g = rng.standard_normal((2, d, N), dtype=np.float32)
        S = (g[0].astype(np.float64) + 1j * g[1].astype(np.float64)) * inv_sqrt2
        X = _source_response(M, angles_deg) @ S
    else:
        X = np.zeros((M, N), dtype=np.complex128)
    w = rng.standard_normal((2, M, N), dtype=np.float32)
    X += (w[0].astype(np.float64) + 1j * w[1].astype(np.float64)) * (sigma * inv_sqrt2)
    return X.astype(np.complex64)


# ---------------------------------------------------------------------------------------------
# Workload recipes. Each one is a seeded function of the instance number.
# ---------------------------------------------------------------------------------------------

def single_c1(seed: int = 20071413) -> Instance:
    """M=8 ULA, two unit-power sources at -20 and 35 deg, SNR 10 dB, N=1024, 0.1 deg grid."""
    M, N, snr, step = 8, 1024, 10.0, 0.1
    ang = np.array([-20.0, 35.0])
    X = snapshots(_rng(seed), M, N, ang, snr)
    return Instance(X, M, 2, N, ang, snr, GRID_LO, step, grid_size(step), seed)


def paper_density(i: int, base_seed: int = 20071414, N: int = 4096) -> Instance:
    """M=16, d=4 in U[-60,60] with 5 deg separation, SNR U[0,20] dB, N=4096, 0.01 deg grid."""
    seed = base_seed + i
    rng = _rng(seed)
    M, d, step = 16, 4, 0.01
    ang = draw_angles(rng, d, -60.0, 60.0, 5.0)
    snr = float(rng.uniform(0.0, 20.0))
    X = snapshots(rng, M, N, ang, snr)
    return Instance(X, M, d, N, ang, snr, GRID_LO, step, grid_size(step), seed)


def paper_density_batch(count: int, base_seed: int = 20071414, N: int = 4096):
    """`count` independent replicas of paper_density as one contiguous complex64 (count, M, N)."""
    M = 16
    X = np.empty((count, M, N), dtype=np.complex64)
    meta = []
    for i in range(count):
        inst = paper_density(i, base_seed, N)
        X[i] = inst.X
        inst.X = None
        meta.append(inst)
    return X, meta


@dataclasses.dataclass
class ProblemSpec:
    """Shape and truth of one problem of the uneven batch (X generated on demand)."""
    index: int
    M: int
    d: int
    N: int
    step: float
    L: int
    alg: int
    angles: np.ndarray
    snr_db: float
    seed: int


def uneven_specs(count: int = 4096, seed: int = 20071415) -> List[ProblemSpec]:
    """Uneven batch: M in {8,12,16,32}, d in U{1..M/2}, N in U{256..8192}, step in
    {0.1, 0.01, 0.001} deg, algorithm uniform over PHD/MUSIC/EV/MN, angles U[-60,60] with
    5 deg separation, SNR U[0,20] dB."""
    rng = _rng(seed)
    specs = []
    for i in range(count):
        M = int(rng.choice([8, 12, 16, 32]))
        d = int(rng.integers(1, M // 2 + 1))
        N = int(rng.integers(256, 8193))
        step = float(rng.choice([0.1, 0.01, 0.001]))
        alg = int(rng.integers(0, 4))
        ang = draw_angles(rng, d, -60.0, 60.0, 5.0)
        snr = float(rng.uniform(0.0, 20.0))
        specs.append(ProblemSpec(i, M, d, N, step, grid_size(step), alg, ang, snr,
                                 seed * 100003 + i))
    return specs


def uneven_instance(spec: ProblemSpec) -> Instance:
    X = snapshots(_rng(spec.seed), spec.M, spec.N, spec.angles, spec.snr_db)
    return Instance(X, spec.M, spec.d, spec.N, spec.angles, spec.snr_db, GRID_LO, spec.step,
                    spec.L, spec.seed, spec.alg)


def large_array(i: int, base_seed: int = 20071416) -> Instance:
    """M=64, d=8 in U[-60,60] with 1 deg separation, SNR U[0,15] dB, N=16384, 0.0005 deg grid."""
    seed = base_seed + i
    rng = _rng(seed)
    M, d, N, step = 64, 8, 16384, 0.0005
    ang = draw_angles(rng, d, -60.0, 60.0, 1.0)
    snr = float(rng.uniform(0.0, 15.0))
    X = snapshots(rng, M, N, ang, snr)
    return Instance(X, M, d, N, ang, snr, GRID_LO, step, grid_size(step), seed)


def proposal_instance(i: int, base_seed: int = 20071418, N: int = 2048) -> Instance:
    """M=16, d in U{1..6}, SNR U[-5,20] dB, angles U[-80,80] with 3 deg separation, N=2048,
    0.001 deg fine grid."""
    seed = base_seed * 1000003 + i
    rng = _rng(seed)
    M = 16
    d = int(rng.integers(1, 7))
    ang = draw_angles(rng, d, -80.0, 80.0, 3.0)
    snr = float(rng.uniform(-5.0, 20.0))
    X = snapshots(rng, M, N, ang, snr)
    step = 0.001
    return Instance(X, M, d, N, ang, snr, GRID_LO, step, grid_size(step), seed)


def custom(M: int, d: int, N: int, angles: Optional[Sequence[float]], snr_db: float, step: float,
           seed: int) -> Instance:
    """Arbitrary instance for tests (angles None -> drawn U[-60,60] with 5 deg separation)."""
    rng = _rng(seed)
    ang = (np.sort(np.asarray(angles, dtype=np.float64)) if angles is not None
           else draw_angles(rng, d, -60.0, 60.0, 5.0))
    X = snapshots(rng, M, N, ang, snr_db)
    return Instance(X, M, d, N, ang, snr_db, GRID_LO, step, grid_size(step), seed)


def _fill_paper_density(args):
    shm_name, shape, start, stop, base_seed, N = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        X = np.ndarray(shape, dtype=np.complex64, buffer=shm.buf)
        meta = []
        for i in range(start, stop):
            inst = paper_density(i, base_seed, N)
            X[i] = inst.X
            meta.append((inst.angles, inst.snr_db, inst.seed))
        return meta
    finally:
        shm.close()


def paper_density_batch_parallel(count: int, base_seed: int = 20071414, N: int = 4096,
                                 workers: Optional[int] = None):
    """Same bytes as paper_density_batch, generated by `workers` spawned processes into shared
    memory. Returns (X complex64 (count, 16, N), list of Instance without X)."""
    import multiprocessing as mp
    import os
    from multiprocessing import shared_memory
    workers = workers or min(16, os.cpu_count() or 1)
    M = 16
    shape = (count, M, N)
    nbytes = int(np.prod(shape)) * 8
    if workers <= 1 or count < 64:
        return paper_density_batch(count, base_seed, N)
    shm = shared_memory.SharedMemory(create=True, size=nbytes)
    try:
        per = (count + workers - 1) // workers
        tasks = [(shm.name, shape, s, min(count, s + per), base_seed, N) for s in range(0, count, per)]
        with mp.get_context("spawn").Pool(len(tasks)) as pool:
            metas = pool.map(_fill_paper_density, tasks)
        X = np.ndarray(shape, dtype=np.complex64, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    step = 0.01
    meta = []
    for part in metas:
        for ang, snr, seed in part:
            meta.append(Instance(None, M, 4, N, ang, snr, GRID_LO, step, grid_size(step), seed))
    return X, meta


def _fill_uneven(args):
    shm_name, total, specs, offsets = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        buf = np.ndarray((total,), dtype=np.complex64, buffer=shm.buf)
        for spec, off in zip(specs, offsets):
            X = snapshots(_rng(spec.seed), spec.M, spec.N, spec.angles, spec.snr_db)
            buf[off:off + spec.M * spec.N] = X.reshape(-1)
        return len(specs)
    finally:
        shm.close()


def uneven_batch_parallel(specs: Sequence[ProblemSpec], workers: Optional[int] = None):
    """Snapshots of every spec in one flat complex64 buffer (problem i at offsets[i], shape
    (M_i, N_i) row-major), generated by spawned workers. Same bytes as uneven_instance(spec).X."""
    import multiprocessing as mp
    import os
    from multiprocessing import shared_memory
    sizes = np.array([s.M * s.N for s in specs], dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    # keep every problem 8-complex (64-byte) aligned
    offsets = np.zeros(len(specs), dtype=np.int64)
    at = 0
    for i, sz in enumerate(sizes):
        offsets[i] = at
        at += int((sz + 7) // 8 * 8)
    total = max(at, 8)
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1 or len(specs) < 64:
        buf = np.zeros(total, dtype=np.complex64)
        for spec, off in zip(specs, offsets):
            buf[off:off + spec.M * spec.N] = uneven_instance(spec).X.reshape(-1)
        return buf, offsets
    shm = shared_memory.SharedMemory(create=True, size=total * 8)
    try:
        order = np.argsort(-sizes)          # deal large problems round-robin for balance
        parts = [order[w::workers] for w in range(workers)]
        tasks = [(shm.name, total, [specs[i] for i in part], [int(offsets[i]) for i in part]) for part in parts]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_fill_uneven, tasks)
        buf = np.ndarray((total,), dtype=np.complex64, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return buf, offsets


def proposal_params(count: int, seed: int, dmax: int = 6):
    """Per-instance parameters of the learned-proposal workload, vectorised: d in U{1..6},
    angles U[-80, 80] with 3 deg separation (spacing transform), SNR U[-5, 20] dB.
    Returns (d int32 (count,), angles float32 (count, dmax) zero-padded, snr float32 (count,))."""
    rng = _rng(seed)
    d = rng.integers(1, dmax + 1, size=count).astype(np.int32)
    lo, hi, sep = -80.0, 80.0, 3.0
    u = rng.uniform(0.0, 1.0, size=(count, dmax))
    span = (hi - lo) - (d - 1) * sep                          # per-row room for the sorted uniforms
    mask = np.arange(dmax)[None, :] < d[:, None]
    u = np.where(mask, u * span[:, None], np.inf)
    u = np.sort(u, axis=1)
    ang = np.where(mask, lo + u + sep * np.arange(dmax)[None, :], 0.0).astype(np.float32)
    snr = rng.uniform(-5.0, 20.0, size=count).astype(np.float32)
    return d, ang, snr


# ---------------------------------------------------------------------------------------------
# Arbitrary geometry (Eq. 2 as printed) and the paper's circular-array scenario (Sec. 4.2)
# ---------------------------------------------------------------------------------------------
SPEED_OF_LIGHT = 299792458.0


def uca_positions(M: int, radius_wl: float) -> np.ndarray:
    """(M, 3) float64 positions in wavelengths of a uniform circular array in the plane z = 0,
    element m at angle 2 pi m / M from the +y axis towards +x."""
    ang = 2.0 * np.pi * np.arange(M, dtype=np.float64) / M
    pos = np.zeros((M, 3), dtype=np.float64)
    pos[:, 0] = radius_wl * np.sin(ang)
    pos[:, 1] = radius_wl * np.cos(ang)
    return pos


def _geometry_response(pos: np.ndarray, az_deg: Sequence[float], el_deg: Sequence[float]) -> np.ndarray:
    """(M, d) complex128 responses of sources at (azimuth, elevation angle) pairs (Eq. 2)."""
    t, p = np.deg2rad(np.asarray(az_deg, np.float64)), np.deg2rad(np.asarray(el_deg, np.float64))
    u = np.stack([np.sin(t) * np.sin(p), np.cos(t) * np.sin(p), np.cos(p)])     # (3, d)
    return np.exp(2j * np.pi * (np.asarray(pos, np.float64) @ u))


def snapshots_geometry(rng: np.random.Generator, pos: np.ndarray, N: int, az_deg: Sequence[float],
                       el_deg: Sequence[float], snr_db: float) -> np.ndarray:
    """X = A S + W as complex64 (M, N) for an arbitrary geometry (same source and noise model as
    `snapshots`)."""
    M, d = pos.shape[0], len(az_deg)
    sigma = math.sqrt(10.0 ** (-snr_db / 10.0))
    inv_sqrt2 = 1.0 / math.sqrt(2.0)
    if d > 0:
        g = rng.standard_normal((2, d, N), dtype=np.float32)
        S = (g[0].astype(np.float64) + 1j * g[1].astype(np.float64)) * inv_sqrt2
        X = _geometry_response(pos, az_deg, el_deg) @ S
    else:
        X = np.zeros((M, N), dtype=np.complex128)
    w = rng.standard_normal((2, M, N), dtype=np.float32)
    X += (w[0].astype(np.float64) + 1j * w[1].astype(np.float64)) * (sigma * inv_sqrt2)
    return X.astype(np.complex64)


@dataclasses.dataclass
class GeoInstance:
    """One snapshot matrix of an arbitrary geometry with its azimuth x elevation scan grid."""
    X: np.ndarray            # complex64 (M, N)
    M: int
    d: int
    N: int
    pos: np.ndarray          # (M, 3) float64, wavelengths
    az: np.ndarray           # true azimuths (deg)
    el: np.ndarray           # true elevation angles (deg)
    snr_db: float
    az_lo: float             # columns theta_k = az_lo + k az_step, k < La
    az_step: float
    La: int
    el_lo: float             # rows phi_l = el_lo + l el_step, l < Le
    el_step: float
    Le: int
    wrap_az: bool            # the azimuth grid closes the circle
    seed: int


def paper_uca(i: int, base_seed: int = 20071420, N: int = 1024, Le: int = 90) -> GeoInstance:
    """The paper's scenario (Sec. 4.2): 8 omnidirectional elements on a circle of radius 10 m at
    15 MHz (radius 10 f / c = 0.5003 wavelengths), two uncorrelated unit-power sources, SNR 15 dB.
    The source angles of its Fig. 4 are not given: azimuths are drawn U[0, 360) at least 30 deg
    apart on the circle, elevation angles U[10, 90]. N is not given either (1024 here). Scan:
    azimuth 0:1:359 (closing the circle) x elevation angle (91 - Le):1:90, the Le rows ending at the
    array plane (Le = 1 is the single row at 90 deg of Sec. 5.1, Le = 90 the 360 x 90 scan of
    Tables 8 and 10)."""
    seed = base_seed + i
    rng = _rng(seed)
    M, d, snr = 8, 2, 15.0
    radius = 10.0 * 15e6 / SPEED_OF_LIGHT
    a0 = float(rng.uniform(0.0, 360.0))
    a1 = (a0 + float(rng.uniform(30.0, 330.0))) % 360.0
    az = np.array([a0, a1])
    el = rng.uniform(10.0, 90.0, size=2)
    pos = uca_positions(M, radius)
    X = snapshots_geometry(rng, pos, N, az, el, snr)
    return GeoInstance(X, M, d, N, pos, az, el, snr, 0.0, 1.0, 360, float(91 - Le), 1.0, Le, True, seed)


def geometry_custom(pos: np.ndarray, d: int, N: int, snr_db: float, az_lo: float, az_step: float, La: int,
                    el_lo: float, el_step: float, Le: int, wrap_az: bool, seed: int) -> GeoInstance:
    """Arbitrary-geometry instance for tests: d sources at azimuth U[0, 360), elevation U[5, 85]."""
    rng = _rng(seed)
    az = rng.uniform(0.0, 360.0, size=d)
    el = rng.uniform(5.0, 85.0, size=d)
    X = snapshots_geometry(rng, np.asarray(pos, np.float64), N, az, el, snr_db)
    return GeoInstance(X, pos.shape[0], d, N, np.asarray(pos, np.float64), az, el, snr_db, az_lo, az_step, La, el_lo,
                       el_step, Le, wrap_az, seed)
