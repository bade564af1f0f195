"""GPU parity of the arbitrary-geometry azimuth x elevation path (Eq. 2 as printed; the circular
array of Sec. 4.2): doa_scan_geometry and doa_peaks2d through the C ABI, and geometry problems in
doa_solve_batch, against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import (DB_TOL, EV, MN, MUSIC, PHD, compare_peaks2d, db_error, factor_from_decomposition,
                              require_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _planar_grid(nx, ny, spacing):
    xs, ys = np.meshgrid(np.arange(nx) * spacing, np.arange(ny) * spacing)
    return np.stack([xs.ravel(), ys.ravel(), np.zeros(nx * ny)], axis=1)


def _geometries():
    rng = np.random.default_rng(41)
    return {
        "uca8": synth.uca_positions(8, 10.0 * 15e6 / synth.SPEED_OF_LIGHT),
        "uca16_far": synth.uca_positions(16, 1.3) + np.array([5.0, -3.0, 0.25]),    # off-centre: centroid shift
        "random3d_12": rng.uniform(-1.0, 1.0, size=(12, 3)),
        "line_z_5": np.stack([np.zeros(5), np.zeros(5), 0.5 * np.arange(5)], axis=1),
        "random_33": rng.uniform(-2.0, 2.0, size=(33, 3)),
        "planar_8x8": _planar_grid(8, 8, 0.5),
    }


# (name, d, az grid, el grid, wrap)
GRIDS = [
    ("uca8", 2, (0.0, 1.0, 360), (1.0, 1.0, 90), True),
    ("uca8", 2, (0.0, 1.0, 360), (90.0, 1.0, 1), True),
    ("uca8", 1, (-37.5, 0.37, 97), (12.0, 0.9, 13), False),      # ragged tile tail, rows split across tiles
    ("uca16_far", 3, (0.0, 2.0, 180), (0.0, 3.0, 31), True),     # includes the zenith row
    ("random3d_12", 4, (10.0, 1.5, 211), (-30.0, 2.5, 81), False),
    ("line_z_5", 1, (5.0, 45.0, 1), (0.0, 0.25, 721), False),     # one column
    ("random_33", 5, (0.0, 3.0, 120), (20.0, 5.0, 14), True),
    ("planar_8x8", 6, (0.0, 0.5, 720), (60.0, 0.5, 61), True),
]


def _factor_inputs(g, d, N=4096, snr=12.0, seed=0):
    pos = _geometries()[g]
    inst = synth.geometry_custom(pos, d, N, snr, 0.0, 1.0, 2, 90.0, 1.0, 1, False, seed)
    R = oracle.covariance(inst.X)
    ev, V, sweeps = oracle.eigh(R)
    assert sweeps > 0
    return pos, ev, V


@pytest.mark.parametrize("case", range(len(GRIDS)))
def test_scan_geometry_matches_oracle(env, case):
    torch, doa = env
    name, d, (alo, ast, La), (elo, est, Le), wrap = GRIDS[case]
    pos, ev, V = _factor_inputs(name, d, seed=500 + case)
    M = pos.shape[0]
    posd = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    geom = doa.geometry(posd, elo, est, Le, wrap)
    for alg in (PHD, MUSIC, EV, MN):
        Co, st = oracle.weighting(ev, V, d, alg)
        assert st == 0
        Bf = factor_from_decomposition(ev, V, d, alg)
        K = Bf.shape[1]
        Po = oracle.scan_geometry(Co, pos, alo, ast, La, elo, est, Le)
        B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
        P = torch.empty(La * Le + 1, dtype=torch.float32, device="cuda")[1:]
        doa.doa_scan_geometry(B, M, K, doa.grid(alo, ast, La), geom, P)
        torch.cuda.synchronize()
        Pg = P.cpu().numpy().reshape(Le, La)
        err = db_error(Pg, Po)
        assert err < DB_TOL, (name, alg, err)


def test_line_array_matches_the_ula_scan(env):
    """A half-wavelength line on x scanned in the plane phi = 90 is the 1-D ULA scan: the 2-D path
    and doa_scan agree with the oracle (and so with each other) on the same factor."""
    torch, doa = env
    M, d, L, lo, step = 16, 4, 1801, -90.0, 0.1
    inst = synth.custom(M, d, 2048, None, 15.0, step, seed=77)
    R = oracle.covariance(inst.X)
    ev, V, _ = oracle.eigh(R)
    pos = np.stack([0.5 * np.arange(M), np.zeros(M), np.zeros(M)], axis=1)
    posd = torch.from_numpy(pos).cuda()
    Bf = factor_from_decomposition(ev, V, d, MUSIC)
    B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
    P2 = torch.empty(L, dtype=torch.float32, device="cuda")
    doa.doa_scan_geometry(B, M, Bf.shape[1], doa.grid(lo, step, L), doa.geometry(posd, 90.0, 1.0, 1, False), P2)
    P1 = torch.empty(L, dtype=torch.float32, device="cuda")
    doa.doa_scan(B, M, Bf.shape[1], doa.grid(lo, step, L), P1)
    torch.cuda.synchronize()
    Co, _ = oracle.weighting(ev, V, d, MUSIC)
    Po, _ = oracle.scan(Co, lo, step, L)
    assert db_error(P2.cpu().numpy(), Po) < DB_TOL
    assert db_error(P1.cpu().numpy(), Po) < DB_TOL


def _peaks2d_gpu(torch, doa, P, wrap, d):
    Le, La = P.shape
    Pd = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda()
    idx = torch.full((max(d, 1),), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros(max(d, 1), dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    doa.doa_peaks2d(Pd, La, Le, wrap, d, idx, val, cnt)
    torch.cuda.synchronize()
    n = cnt.item()
    return idx.cpu().numpy()[:n], val.cpu().numpy()[:n]


def test_peaks2d_matches_oracle(env):
    """Same float32 values on both sides: the flat indices must be identical, with ties (integer
    spectra), wrap on and off, edge rows and columns, one row, one column, one point."""
    torch, doa = env
    rng = np.random.default_rng(8)
    spectra = [rng.integers(0, 5, size=(Le, La)).astype(np.float32)
               for Le, La in [(1, 1), (1, 7), (9, 1), (3, 3), (17, 300), (90, 360), (41, 257)]]
    spectra += [rng.random((90, 360)).astype(np.float32), rng.random((7, 1000)).astype(np.float32)]
    g = synth.paper_uca(3)
    spectra.append(oracle.solve_geometry(g.X, 2, MUSIC, g.pos, g.az_lo, g.az_step, g.La, g.el_lo, g.el_step, g.Le,
                                         True)["P"].astype(np.float32))
    flat = np.zeros((50, 60), np.float32)
    flat[0, 0] = flat[49, 59] = flat[25, 30] = 2.0                 # corners and centre, equal values
    spectra.append(flat)
    for P in spectra:
        for wrap in (False, True):
            for d in (0, 1, 2, 5, 63):
                got_i, got_v = _peaks2d_gpu(torch, doa, P, wrap, d)
                ref_i, ref_v = oracle.peaks2d(P.astype(np.float64), d, wrap)
                assert list(got_i) == list(ref_i), (P.shape, wrap, d)
                assert np.array_equal(got_v.astype(np.float64), ref_v)


def _geo_problem(torch, doa, g, mask, keep):
    nalg = bin(mask).count("1")
    npts = g.La * g.Le
    X = torch.from_numpy(g.X).cuda()
    P = torch.empty(nalg * npts, dtype=torch.float32, device="cuda")
    idx = torch.full((nalg * max(g.d, 1),), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros(nalg * max(g.d, 1), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(nalg, dtype=torch.int32, device="cuda")
    ev = torch.empty(g.M, dtype=torch.float64, device="cuda")
    posd = torch.from_numpy(np.ascontiguousarray(g.pos)).cuda()
    keep.append((X, P, idx, val, cnt, ev, posd))
    geom = doa.geometry(posd, g.el_lo, g.el_step, g.Le, g.wrap_az)
    return doa.make_problem(X, g.d, mask, doa.grid(g.az_lo, g.az_step, g.La), P, idx, val, cnt, ev, geom=geom)


def _check_geo(g, mask, t, worst):
    _, P, idx, _, cnt, ev, _ = t
    npts = g.La * g.Le
    P = P.cpu().numpy().reshape(-1, npts)
    idx = idx.cpu().numpy().reshape(-1, max(g.d, 1))
    cnt = cnt.cpu().numpy()
    slot = 0
    for alg in range(4):
        if not (mask >> alg) & 1:
            continue
        ref = oracle.solve_geometry(g.X, g.d, alg, g.pos, g.az_lo, g.az_step, g.La, g.el_lo, g.el_step, g.Le,
                                    g.wrap_az)
        assert ref["status"] == 0
        err = db_error(P[slot], ref["P"].reshape(-1))
        worst[0] = max(worst[0], err)
        assert err < DB_TOL, (g.seed, alg, err)
        ok, ties = compare_peaks2d(idx[slot][:cnt[slot]], ref["idx"], ref["P"], g.La, g.Le, g.wrap_az, 1e-4)
        assert ok, (g.seed, alg, idx[slot][:cnt[slot]], ref["idx"], ties)
        slot += 1
    np.testing.assert_allclose(ev.cpu().numpy(), ref["evals"], rtol=0, atol=1e-5 * ref["evals"][0])


def test_batch_paper_uca(env):
    """The paper's circular-array scenario through doa_solve_batch: 360 x 90 and 360 x 1 scans, all
    four algorithms, every spectrum within 0.01 dB of the oracle and the same 2-D peaks."""
    torch, doa = env
    insts = [synth.paper_uca(i) for i in range(6)] + [synth.paper_uca(10 + i, Le=1) for i in range(2)]
    keep, probs = [], []
    for g in insts:
        probs.append(_geo_problem(torch, doa, g, 0xF, keep))
    plan = doa.BatchPlan(probs)
    ws = doa.workspace(plan)
    status = torch.full((len(insts),), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    worst = [0.0]
    for g, t in zip(insts, keep):
        _check_geo(g, 0xF, t, worst)


def test_batch_shared_array(env):
    """Problems that pass one positions tensor share an FP32 steering table written once per solve
    (360 x 90 and 360 x 1 grids, four algorithms); a problem with its own copy of the same array
    evaluates its phasors in the scan. All spectra within 0.01 dB of the oracle, same 2-D peaks."""
    torch, doa = env
    insts = [synth.paper_uca(20 + i) for i in range(4)] + [synth.paper_uca(30 + i, Le=1) for i in range(2)]
    posd = torch.from_numpy(np.ascontiguousarray(insts[0].pos)).cuda()
    for g in insts:
        assert np.array_equal(g.pos, insts[0].pos)
    keep, probs = [], []
    for g in insts:
        npts = g.La * g.Le
        X = torch.from_numpy(g.X).cuda()
        P = torch.empty(4 * npts, dtype=torch.float32, device="cuda")
        idx = torch.full((4 * g.d,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(4 * g.d, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
        ev = torch.empty(g.M, dtype=torch.float64, device="cuda")
        keep.append((X, P, idx, val, cnt, ev, posd))
        geom = doa.geometry(posd, g.el_lo, g.el_step, g.Le, g.wrap_az)
        probs.append(doa.make_problem(X, g.d, 0xF, doa.grid(g.az_lo, g.az_step, g.La), P, idx, val, cnt, ev,
                                      geom=geom))
    own, keep_own = synth.paper_uca(40), []
    probs.insert(2, _geo_problem(torch, doa, own, 0xF, keep_own))
    plan = doa.BatchPlan(probs)
    assert int(plan.host[:512].view(np.int32)[doa.BatchPlan.header_index("ngeo_steer")]) == 2
    ws = doa.workspace(plan)
    status = torch.full((len(probs),), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    worst = [0.0]
    for g, t in zip(insts, keep):
        _check_geo(g, 0xF, t, worst)
    _check_geo(own, 0xF, keep_own[0], worst)


def test_batch_mixed_geometry_and_ula(env):
    """Geometry problems of every M bucket next to ULA problems in one plan: both kinds match the
    oracle, so the two scan paths and the two peak rules coexist in the same launches."""
    torch, doa = env
    geos = _geometries()
    ginsts = [
        synth.geometry_custom(geos["uca16_far"], 3, 2000, 10.0, 0.0, 2.0, 180, 0.0, 3.0, 31, True, seed=61),
        synth.geometry_custom(geos["random_33"], 4, 3000, 15.0, 0.0, 3.0, 120, 20.0, 5.0, 14, True, seed=62),
        synth.geometry_custom(geos["planar_8x8"], 5, 5000, 15.0, 0.0, 1.0, 360, 30.0, 1.0, 61, True, seed=63),
        synth.geometry_custom(geos["random3d_12"], 2, 700, 8.0, 10.0, 1.5, 211, -30.0, 2.5, 81, False, seed=64),
    ]
    masks = [0xF, 1 << MUSIC | 1 << MN, 1 << EV, 1 << PHD]
    ulas = [synth.custom(8, 2, 1024, None, 10.0, 0.1, seed=71), synth.custom(16, 4, 4096, None, 12.0, 0.05, seed=72)]
    keep, probs = [], []
    for g, mask in zip(ginsts, masks):
        probs.append(_geo_problem(torch, doa, g, mask, keep))
    ula_t = []
    for inst in ulas:
        X = torch.from_numpy(inst.X).cuda()
        P = torch.empty(4 * inst.L, dtype=torch.float32, device="cuda")
        idx = torch.full((4 * inst.d,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(4 * inst.d, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
        ula_t.append((X, P, idx, val, cnt))
        probs.insert(1, doa.make_problem(X, inst.d, 0xF, doa.grid(inst.lo, inst.step, inst.L), P, idx, val, cnt))
    plan = doa.BatchPlan(probs)
    ws = doa.workspace(plan)
    status = torch.full((len(probs),), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    worst = [0.0]
    for g, mask, t in zip(ginsts, masks, keep):
        _check_geo(g, mask, t, worst)
    from tests.gpu_common import compare_peaks
    for inst, t in zip(ulas, ula_t):
        P = t[1].cpu().numpy().reshape(4, inst.L)
        idx = t[2].cpu().numpy().reshape(4, inst.d)
        for alg in range(4):
            ref = oracle.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
            assert db_error(P[alg], ref["P"]) < DB_TOL
            ok, ties = compare_peaks(idx[alg][:t[4][alg].item()], ref["idx"], ref["P"], 1e-4)
            assert ok, ties


def test_scan_geometry_single_point_and_single_column(env):
    torch, doa = env
    pos, ev, V = _factor_inputs("uca8", 2, seed=9)
    posd = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    Co, _ = oracle.weighting(ev, V, 2, MUSIC)
    Bf = factor_from_decomposition(ev, V, 2, MUSIC)
    B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
    for (alo, ast, La), (elo, est, Le) in [((33.0, 1.0, 1), (45.0, 1.0, 1)), ((200.0, 0.0, 1), (0.0, 0.5, 181))]:
        P = torch.empty(La * Le, dtype=torch.float32, device="cuda")
        doa.doa_scan_geometry(B, 8, Bf.shape[1], doa.grid(alo, ast, La), doa.geometry(posd, elo, est, Le, False), P)
        torch.cuda.synchronize()
        Po = oracle.scan_geometry(Co, pos, alo, ast, La, elo, est, Le)
        assert db_error(P.cpu().numpy(), Po.reshape(-1)) < DB_TOL
