"""GPU parity: every stage of the CUDA path, called through the C ABI, against the FP64 oracle on
the same seeded complex64 inputs."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import (DB_TOL, EV, MN, MUSIC, PHD, compare_peaks, db_error, factor_from_decomposition,
                              percent_error, require_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


# ------------------------------------------------------------------------------ Step-1
@pytest.mark.parametrize("M,N,pad", [(2, 3, 0), (3, 7, 1), (8, 1024, 0), (12, 1000, 3), (16, 4096, 0),
                                     (16, 4097, 5), (32, 3000, 0), (64, 5000, 2), (64, 16384, 0)])
def test_covariance(env, M, N, pad):
    torch, doa = env
    inst = synth.custom(M, min(3, M - 1), N, None, 10.0, 0.1, seed=1000 + M * 7 + N)
    Xh = np.zeros((M, N + pad), np.complex64)
    Xh[:, :N] = inst.X
    X = torch.from_numpy(Xh).cuda()[:, :N]
    R64 = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    R32 = torch.empty((M, M), dtype=torch.complex64, device="cuda")
    doa.doa_covariance(X, R=R32, R64=R64)
    torch.cuda.synchronize()
    Ro = oracle.covariance(inst.X)
    scale = np.max(np.abs(Ro))
    err = np.max(np.abs(R64.cpu().numpy() - Ro)) / scale
    assert err < 2e-6, err
    assert np.max(np.abs(R32.cpu().numpy() - Ro)) / scale < 3e-6
    Rg = R64.cpu().numpy()
    assert np.array_equal(Rg, Rg.conj().T)


# ------------------------------------------------------------------------------ Steps 2-4
@pytest.mark.parametrize("M,d", [(2, 1), (3, 1), (5, 2), (8, 2), (8, 0), (8, 7), (12, 5), (16, 4), (31, 9),
                                 (32, 16), (64, 8)])
def test_noise_subspace(env, M, d):
    torch, doa = env
    ang = None if d <= 8 else np.linspace(-70.0, 70.0, d) + 0.37   # many sources: spread evenly
    inst = synth.custom(M, d, max(4 * M, 256), ang, 12.0, 0.1, seed=2000 + M * 13 + d)
    Ro = oracle.covariance(inst.X)
    ev_o, V_o, _ = oracle.eigh(Ro)
    R = torch.from_numpy(Ro).cuda()
    for alg in (PHD, MUSIC, EV, MN):
        B = torch.zeros(M * M, dtype=torch.complex128, device="cuda")
        ev = torch.empty(M, dtype=torch.float64, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        K = torch.zeros(1, dtype=torch.int32, device="cuda")
        doa.doa_noise_subspace(R, d, alg, B, info, evals=ev, K_out=K)
        torch.cuda.synchronize()
        assert info.item() > 0, info.item()
        Kx = 1 if alg in (PHD, MN) else M - d
        assert K.item() == Kx
        np.testing.assert_allclose(ev.cpu().numpy(), ev_o, rtol=0, atol=1e-12 * ev_o[0])
        Bg = B.cpu().numpy()[:M * Kx].reshape(Kx, M).T
        Cg = Bg @ Bg.conj().T
        Co, st = oracle.weighting(ev_o, V_o, d, alg)
        assert st == 0
        assert np.max(np.abs(Cg - Co)) < 1e-10 * np.max(np.abs(Co)), (alg, np.max(np.abs(Cg - Co)))


@pytest.mark.parametrize("M,d", [(5, 2), (16, 4), (32, 16), (33, 3), (47, 6), (64, 8)])
def test_noise_subspace_double_float(env, M, d):
    """doa_noise_subspace_prec with the double-float Jacobi (~48-bit rotations, FP64 output): the
    same eigenvalues (1e-12 of the largest) and weighting matrices C = B B^H (1e-10) as the FP64
    oracle for all four algorithms, on sample covariances and, at M = 64, on an exact covariance
    A P A^H + sigma^2 I (noise eigenvalues sigma^2 to 1e-13 of the largest, E_n^H a(theta_i) = 0)."""
    torch, doa = env
    ang = None if d <= 8 else np.linspace(-70.0, 70.0, d) + 0.37
    inst = synth.custom(M, d, max(4 * M, 256), ang, 12.0, 0.1, seed=2100 + M * 13 + d)
    Ro = oracle.covariance(inst.X)
    ev_o, V_o, _ = oracle.eigh(Ro)
    R = torch.from_numpy(Ro).cuda()
    for alg in (PHD, MUSIC, EV, MN):
        B = torch.zeros(M * M, dtype=torch.complex128, device="cuda")
        ev = torch.empty(M, dtype=torch.float64, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        doa.doa_noise_subspace_prec(R, d, alg, doa.EIG_DOUBLE_FLOAT, B, info, evals=ev)
        torch.cuda.synchronize()
        assert info.item() > 0, info.item()
        np.testing.assert_allclose(ev.cpu().numpy(), ev_o, rtol=0, atol=1e-12 * ev_o[0])
        Kx = 1 if alg in (PHD, MN) else M - d
        Bg = B.cpu().numpy()[:M * Kx].reshape(Kx, M).T
        Co, st = oracle.weighting(ev_o, V_o, d, alg)
        assert st == 0
        assert np.max(np.abs(Bg @ Bg.conj().T - Co)) < 1e-10 * np.max(np.abs(Co)), alg
    if M == 64:
        m = np.arange(M)[:, None]
        angs = np.linspace(-60.0, 60.0, d) + 0.21
        A = np.exp(1j * np.pi * m * np.sin(np.radians(angs))[None, :])
        s2 = 0.1
        R = torch.from_numpy(A @ A.conj().T + s2 * np.eye(M)).cuda()
        B = torch.zeros(M * M, dtype=torch.complex128, device="cuda")
        ev = torch.empty(M, dtype=torch.float64, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        doa.doa_noise_subspace_prec(R, d, MUSIC, doa.EIG_DOUBLE_FLOAT, B, info, evals=ev)
        torch.cuda.synchronize()
        assert info.item() > 0
        # double-float rotations (~2^-48) leave errors relative to the largest eigenvalue (~M)
        evg = ev.cpu().numpy()
        np.testing.assert_allclose(evg[d:], s2, rtol=0, atol=1e-13 * evg[0])
        En = B.cpu().numpy()[:M * (M - d)].reshape(M - d, M).T
        assert np.linalg.norm(En.conj().T @ A) < 1e-11 * np.linalg.norm(A)
        assert np.max(np.abs(En.conj().T @ En - np.eye(M - d))) < 1e-13


def test_noise_subspace_exact_covariance(env):
    """R = A A^H + sigma^2 I: noise eigenvalues sigma^2 and E_n^H a(theta_i) = 0 on the GPU too."""
    torch, doa = env
    M, ang, s2 = 8, [-20.0, 35.0], 0.1
    m = np.arange(M)[:, None]
    A = np.exp(1j * np.pi * m * np.sin(np.radians(ang))[None, :])
    R = torch.from_numpy(A @ A.conj().T + s2 * np.eye(M)).cuda()
    B = torch.zeros(M * M, dtype=torch.complex128, device="cuda")
    ev = torch.empty(M, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    doa.doa_noise_subspace(R, 2, MUSIC, B, info, evals=ev)
    torch.cuda.synchronize()
    np.testing.assert_allclose(ev.cpu().numpy()[2:], s2, rtol=1e-12)
    En = B.cpu().numpy()[:M * 6].reshape(6, M).T
    assert np.linalg.norm(En.conj().T @ A) < 1e-12
    assert np.max(np.abs(En.conj().T @ En - np.eye(6))) < 1e-13


def test_noise_subspace_status(env):
    torch, doa = env
    M = 6
    R = torch.zeros((M, M), dtype=torch.complex128, device="cuda")
    B = torch.zeros(M * M, dtype=torch.complex128, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    doa.doa_noise_subspace(R, 2, EV, B, info)          # all eigenvalues 0
    assert info.item() == -doa.ERANK
    doa.doa_noise_subspace(R, 2, MN, B, info)          # V = I: e_1 outside the noise subspace
    assert info.item() == -doa.ERANK
    doa.doa_noise_subspace(R, 2, MUSIC, B, info)
    assert info.item() > 0
    R[1, 2] = float("nan")
    doa.doa_noise_subspace(R, 2, MUSIC, B, info)
    assert info.item() == -doa.ENONFINITE


# ------------------------------------------------------------------------------ Step-5
@pytest.mark.parametrize("M,d,step,L", [(8, 2, 0.1, 1801), (16, 4, 0.01, 18001), (12, 3, 0.07, 2573),
                                        (32, 5, 0.05, 3601), (64, 8, 0.01, 18001), (5, 1, 45.0, 5),
                                        (2, 1, 90.0, 3), (16, 0, 1.0, 181)])
def test_scan(env, M, d, step, L):
    torch, doa = env
    inst = synth.custom(M, d, 2048, None, 15.0, step, seed=3000 + M + d)
    Ro = oracle.covariance(inst.X)
    ev_o, V_o, _ = oracle.eigh(Ro)
    lo = -90.0
    for alg in (PHD, MUSIC, EV, MN):
        Co, _ = oracle.weighting(ev_o, V_o, d, alg)
        Bf = factor_from_decomposition(ev_o, V_o, d, alg)
        assert np.max(np.abs(Bf @ Bf.conj().T - Co)) < 1e-12 * np.max(np.abs(Co))
        K = Bf.shape[1]
        Po, _ = oracle.scan(Co, lo, step, L)
        B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
        P = torch.empty(L + 1, dtype=torch.float32, device="cuda")[1:]   # 4-byte aligned, not 8
        doa.doa_scan(B, M, K, doa.grid(lo, step, L), P)
        torch.cuda.synchronize()
        Pg = P.cpu().numpy()
        assert db_error(Pg, Po) < DB_TOL, (alg, db_error(Pg, Po))
        assert percent_error(Pg, Po) < 0.05
        assert Pg[0] == Pg[-1] or abs(step * (L - 1) - 180.0) > 1e-9


# ------------------------------------------------------------------------------ Step-6
def test_peaks_golden(env):
    import json, os
    torch, doa = env
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "peaks_cases.json")))
    for c in g["cases"]:
        P = torch.tensor(c["P"], dtype=torch.float32, device="cuda")
        d = c["d"]
        idx = torch.full((max(d, 1),), -7, dtype=torch.int32, device="cuda")
        val = torch.zeros(max(d, 1), dtype=torch.float32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        doa.doa_peaks(P, d, idx, val, cnt)
        n = cnt.item()
        assert idx.cpu().numpy()[:n].tolist() == c["idx"], c["name"]


@pytest.mark.parametrize("L,d,levels", [(3, 1, 3), (50, 3, 4), (1000, 5, 6), (18001, 4, 1000), (180001, 8, 50),
                                        (360001, 8, 1 << 20)])
def test_peaks_random(env, L, d, levels):
    """Random (often tied) spectra: the GPU picker and the oracle's see the same float32 values."""
    torch, doa = env
    rng = np.random.default_rng(L + d)
    for trial in range(3):
        Ph = (rng.integers(0, levels, L) / levels).astype(np.float32)
        P = torch.from_numpy(Ph).cuda()
        idx = torch.zeros(d, dtype=torch.int32, device="cuda")
        val = torch.zeros(d, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        doa.doa_peaks(P, d, idx, val, cnt)
        n = cnt.item()
        io, vo = oracle.peaks(Ph.astype(np.float64), d)
        assert idx.cpu().numpy()[:n].tolist() == io.tolist()
        assert np.array_equal(val.cpu().numpy()[:n].astype(np.float64), vo)


# ------------------------------------------------------------------------------ Steps 1-6
def _single_pipeline(torch, doa, inst, alg):
    M, d, L = inst.M, inst.d, inst.L
    X = torch.from_numpy(inst.X).cuda()
    R = torch.empty((M, M), dtype=torch.complex128, device="cuda")
    B = torch.zeros(M * M, dtype=torch.complex128, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    K = torch.zeros(1, dtype=torch.int32, device="cuda")
    P = torch.empty(L, dtype=torch.float32, device="cuda")
    idx = torch.zeros(max(d, 1), dtype=torch.int32, device="cuda")
    val = torch.zeros(max(d, 1), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    doa.doa_covariance(X, R64=R)
    doa.doa_noise_subspace(R, d, alg, B, info, K_out=K)
    Kx = 1 if alg in (PHD, MN) else M - d
    doa.doa_scan(B, M, Kx, doa.grid(inst.lo, inst.step, L), P)
    doa.doa_peaks(P, d, idx, val, cnt)
    torch.cuda.synchronize()
    assert info.item() > 0 and K.item() == Kx
    return P.cpu().numpy(), idx.cpu().numpy()[:cnt.item()]


def test_single_calls_c1(env):
    torch, doa = env
    inst = synth.single_c1()
    for alg in (PHD, MUSIC, EV, MN):
        ref = oracle.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
        P, idx = _single_pipeline(torch, doa, inst, alg)
        assert db_error(P, ref["P"]) < DB_TOL
        assert idx.tolist() == ref["idx"].tolist()


def _batch_solve(torch, doa, insts, masks, prec=0, eig_prec=0, polish=False, scan_group=None):
    tensors, probs = [], []
    for inst, mask in zip(insts, masks):
        nalg = bin(mask).count("1")
        X = torch.from_numpy(inst.X).cuda()
        P = torch.empty(nalg * inst.L, dtype=torch.float32, device="cuda")
        idx = torch.full((nalg * max(inst.d, 1),), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(nalg * max(inst.d, 1), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(nalg, dtype=torch.int32, device="cuda")
        ev = torch.empty(inst.M, dtype=torch.float64, device="cuda")
        tensors.append((X, P, idx, val, cnt, ev))
        probs.append(doa.make_problem(X, inst.d, mask, doa.grid(inst.lo, inst.step, inst.L), P, idx, val, cnt, ev,
                                      prec=prec, eig_prec=eig_prec, polish=polish))
    plan = doa.BatchPlan(probs, scan_group=scan_group)
    ws = doa.workspace(plan)
    status = torch.full((len(insts),), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    return tensors, status.cpu().numpy()


def _check_batch(torch, doa, insts, masks, prec=0, eig_prec=0, polish=False, tie=1e-4):
    """Every requested spectrum within DB_TOL of the oracle at every point, the peak indices equal
    up to ties whose oracle values differ by less than `tie` (relative), the eigenvalues close."""
    tensors, status = _batch_solve(torch, doa, insts, masks, prec, eig_prec, polish=polish)
    assert np.all(status == 0), status
    worst = 0.0
    for inst, mask, t in zip(insts, masks, tensors):
        _, P, idx, _, cnt, ev = t
        P = P.cpu().numpy().reshape(-1, inst.L)
        idx = idx.cpu().numpy().reshape(-1, max(inst.d, 1))
        cnt = cnt.cpu().numpy()
        slot = 0
        for alg in range(4):
            if not (mask >> alg) & 1:
                continue
            ref = oracle.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
            err = db_error(P[slot], ref["P"])
            worst = max(worst, err)
            assert err < DB_TOL, (inst.seed, alg, err)
            ok, ties = compare_peaks(idx[slot][:cnt[slot]], ref["idx"], ref["P"], tie)
            assert ok, (inst.seed, alg, idx[slot][:cnt[slot]], ref["idx"], ties)
            slot += 1
        np.testing.assert_allclose(ev.cpu().numpy(), ref["evals"], rtol=0, atol=1e-5 * ref["evals"][0])
    return worst


def test_batch_c1_all_algorithms(env):
    torch, doa = env
    _check_batch(torch, doa, [synth.single_c1()], [0xF])


def test_batch_paper_density_sample(env):
    """Peak polish on, as in the headline: peak indices equal to the oracle's up to ties below
    float resolution (1e-6 relative)."""
    torch, doa = env
    insts = [synth.paper_density(i) for i in range(8)]
    _check_batch(torch, doa, insts, [0xF] * len(insts), polish=True, tie=1e-6)


def test_batch_paper_density_sample_unpolished(env):
    """Without the polish two neighbouring grid points whose oracle values differ by less than the
    FP32 path's error bound may swap: ties up to 1e-4 relative are accepted there."""
    torch, doa = env
    insts = [synth.paper_density(i) for i in range(8)]
    _check_batch(torch, doa, insts, [0xF] * len(insts))


def test_scan_refinement_queue_overflow(env):
    """More near-null points than the refinement queue holds (1024) before a drain: a 2-element
    array with a strong source at broadside, scanned from -0.1 to 0.1 deg in steps of 1e-5 deg,
    puts about half of the 20001 points below the refinement threshold (den = 1 - cos(pi u) near
    the MUSIC null), so the queue overflows and the overflowing points are re-evaluated in place,
    one thread each. Alone (per-problem scan, runs of several tiles per drain) and as 32 problems
    sharing the grid (grid-shared scan, one tile of all 32 per drain), with all four algorithms and
    with PHD and MN alone (points flagged for those readouts only fill the queue from its back),
    every point stays within DB_TOL of the oracle."""
    torch, doa = env
    base = synth.custom(2, 1, 2048, [0.0], 20.0, 0.01, seed=777)
    inst = dataclasses.replace(base, lo=-0.1, step=1e-5, L=20001)
    refs = [oracle.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)["P"] for alg in range(4)]
    # the MUSIC denominator near the null: far more than 1024 points below 2.05e-6 (sum |f_m|)^2 = 4.1e-6
    assert np.sum(1.0 / refs[MUSIC] < 4.1e-6) > 4 * 1024
    # all four spectra (MUSIC / EV flagged: the whole re-evaluation, front of the queue), and PHD + MN
    # alone (their columns only, back of the queue)
    for mask in (0xF, (1 << PHD) | (1 << MN)):
        algs = [a for a in range(4) if (mask >> a) & 1]
        for group in ([inst], [inst] * 32):
            tensors, status = _batch_solve(torch, doa, group, [mask] * len(group))
            assert np.all(status == 0), status
            for t in tensors:
                P = t[1].cpu().numpy().reshape(len(algs), inst.L)
                for slot, alg in enumerate(algs):
                    err = db_error(P[slot], refs[alg])
                    assert err < DB_TOL, (mask, len(group), alg, err)


def test_batch_paper_density_sample_polished(env):
    """The headline configuration (peak polish on): peak indices equal to the oracle's up to ties
    below float resolution (1e-6 relative), on a sample of the paper-density batch."""
    torch, doa = env
    insts = [synth.paper_density(i) for i in range(8, 24)]
    _check_batch(torch, doa, insts, [0xF] * len(insts), polish=True, tie=1e-6)


def test_batch_uneven_sample(env):
    """Problems drawn from the uneven recipe (every M bucket, every algorithm), fine grids thinned."""
    torch, doa = env
    specs = synth.uneven_specs(4096)
    picked, seen = [], set()
    for s in specs:
        key = (s.M, s.alg)
        if key in seen or s.step < 0.01:
            continue
        seen.add(key)
        picked.append(s)
    insts = [synth.uneven_instance(s) for s in picked]
    _check_batch(torch, doa, insts, [1 << s.alg for s in picked])


@pytest.mark.parametrize("mask", [1 << PHD, 1 << MUSIC])
def test_batch_covariance_entries(env, mask):
    """Every covariance work-item class of the batch (M in 4..17, one and several 1024-snapshot
    chunks, compensated for PHD and plain otherwise): the trace-normalised upper triangle the
    batch writes as the proposal features matches the oracle's R entry by entry, and the
    eigenvalues follow R to FP64 accuracy in the compensated mode."""
    torch, doa = env
    cases = [(4, 700), (5, 1500), (8, 1024), (9, 2500), (12, 333), (13, 4096), (16, 3000), (17, 1100)]
    insts = [synth.custom(M, 1, N, None, 10.0, 1.0, seed=950 + M) for M, N in cases]
    tensors, probs = [], []
    for inst in insts:
        M = inst.M
        X = torch.from_numpy(inst.X).cuda()
        P = torch.empty(inst.L, dtype=torch.float32, device="cuda")
        idx = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(1, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        ev = torch.empty(M, dtype=torch.float64, device="cuda")
        F = torch.empty(M * (M + 1), dtype=torch.float32, device="cuda")
        tensors.append((X, P, idx, val, cnt, ev, F))
        probs.append(doa.make_problem(X, 1, mask, doa.grid(inst.lo, inst.step, inst.L), P, idx, val, cnt, ev,
                                      features=F))
    plan = doa.BatchPlan(probs)
    ws = doa.workspace(plan)
    status = torch.full((len(insts),), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for inst, t in zip(insts, tensors):
        M = inst.M
        R = oracle.covariance(inst.X)
        iu = np.triu_indices(M)
        want = np.stack([R[iu].real, R[iu].imag], axis=1).reshape(-1) / np.trace(R).real
        got = t[6].cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-6 * np.max(np.abs(want)), err_msg=f"M={M}")
        ev_ref, _, _ = oracle.eigh(R)
        tol = (1e-10 if mask == 1 << PHD else 1e-5) * ev_ref[0]
        np.testing.assert_allclose(t[5].cpu().numpy(), ev_ref, rtol=0, atol=tol, err_msg=f"M={M}")


def test_batch_every_algorithm_subset(env):
    """All 15 non-empty algorithm sets, over every M bucket: the shared-contraction scan reads
    each requested spectrum from one factor (E_n with PHD / EV / MUSIC readouts, valph for MN,
    or v_min / valph alone) and every one matches the oracle's Table 3 spectrum."""
    torch, doa = env
    Ms = [8, 12, 16, 33, 6]
    insts, masks = [], []
    for mask in range(1, 16):
        M = Ms[mask % len(Ms)]
        insts.append(synth.custom(M, 1 + mask % 3, 1500 + 37 * mask, None, 5.0 + mask, 0.1, seed=900 + mask))
        masks.append(mask)
    insts.append(synth.custom(5, 0, 64, [], 0.0, 0.5, seed=931))     # d = 0: E_n = all of V, valph = e1
    masks.append(0xF)
    _check_batch(torch, doa, insts, masks)


@pytest.mark.parametrize("prec", [2, 3])   # DOA_BF16X3, DOA_FP16X3
def test_batch_tensor_core_scan(env, prec):
    """Split-operand tcgen05 scan in the batch (shared contraction, four readouts, FP32 then FP64
    re-evaluation of the near-null points): every spectrum within 0.01 dB of the oracle and the
    same peaks, over every algorithm subset and M up to 32."""
    torch, doa = env
    insts = [synth.paper_density(i) for i in range(4)]
    masks = [0xF] * 4
    Ms = [8, 12, 16, 32, 5]
    for mask in range(1, 16):
        M = Ms[mask % len(Ms)]
        insts.append(synth.custom(M, 1 + mask % 3, 1500 + 37 * mask, None, 5.0 + mask, 0.1, seed=700 + mask))
        masks.append(mask)
    insts.append(synth.custom(5, 0, 64, [], 0.0, 0.5, seed=731))     # d = 0: Kf = M + 1
    masks.append(0xF)
    _check_batch(torch, doa, insts, masks, prec)


@pytest.mark.parametrize("prec", [2, 3])   # DOA_BF16X3, DOA_FP16X3
def test_batch_tensor_core_scan_grid_groups(env, prec):
    """The grid-shared tensor-core scan: 40 problems of every M bucket (M = 6 .. 32) and mixed
    algorithm subsets on one grid (groups of stacked factors, chunks of groups sharing a steering
    block, a ragged last tile), against the oracle on every fifth problem (0.01 dB, same peaks),
    and against the per-problem tensor-core scan (scan_group 1) on all of them."""
    torch, doa = env
    Ms = [6, 8, 12, 16, 16, 24, 32]
    insts, masks = [], []
    for i in range(40):
        M = Ms[i % len(Ms)]
        d = 1 + i % min(4, M - 2)
        inst = synth.custom(M, d, 600 + 13 * i, None, 6.0 + (i % 9), 0.1, seed=1300 + i)
        insts.append(inst)
        masks.append([0xF, 0x2, 0x5, 0xA, 0x7][i % 5])
    assert len({(x.lo, x.step, x.L) for x in insts}) == 1      # one grid for all
    grouped, st = _batch_solve(torch, doa, insts, masks, prec)
    assert np.all(st == 0), st
    alone, st1 = _batch_solve(torch, doa, insts, masks, prec, scan_group=[1, 1, 1, 1])
    assert np.all(st1 == 0), st1
    for inst, mask, a, b in zip(insts, masks, grouped, alone):
        assert db_error(a[1].cpu().numpy(), b[1].cpu().numpy().astype(np.float64)) < 2e-3, inst.seed
    _check_batch(torch, doa, insts[::5], masks[::5], prec)


def test_batch_fp64_jacobi(env):
    """The batch's FP64 Jacobi (doa_problem.eig_prec = DOA_EIG_FP64) meets the same bar, and its
    spectra agree with the default double-float Jacobi's to far inside the tolerance."""
    torch, doa = env
    insts = [synth.paper_density(i) for i in range(3)] + [synth.custom(32, 6, 3000, None, 12.0, 0.1, seed=41),
                                                          synth.custom(8, 2, 900, None, 8.0, 0.1, seed=42)]
    masks = [0xF] * len(insts)
    _check_batch(torch, doa, insts, masks, eig_prec=1)
    a, _ = _batch_solve(torch, doa, insts, masks, eig_prec=1)
    b, _ = _batch_solve(torch, doa, insts, masks, eig_prec=0)
    for ta, tb in zip(a, b):
        assert db_error(ta[1].cpu().numpy(), tb[1].cpu().numpy().astype(np.float64)) < 1e-3


def test_batch_cluster_jacobi_bucket(env):
    """The batch's M <= 64 bucket: double-float Jacobi on four-CTA clusters (odd M pads the round-
    robin order with a skipped index; M = 33 leaves the fourth CTA without rows) and the FP64
    Jacobi in one CTA of the same kernel; both meet the oracle bar and agree with each other."""
    torch, doa = env
    insts = [synth.custom(33, 3, 2000, None, 12.0, 0.1, seed=51),
             synth.custom(48, 5, 2500, None, 10.0, 0.1, seed=52),
             synth.custom(64, 8, 4000, None, 12.0, 0.1, seed=53)]
    masks = [0xF, 0b0110, 0xF]
    _check_batch(torch, doa, insts, masks, eig_prec=0)
    _check_batch(torch, doa, insts, masks, eig_prec=1)
    a, _ = _batch_solve(torch, doa, insts, masks, eig_prec=1)
    b, _ = _batch_solve(torch, doa, insts, masks, eig_prec=0)
    for ta, tb in zip(a, b):
        assert db_error(ta[1].cpu().numpy(), tb[1].cpu().numpy().astype(np.float64)) < 1e-3


def test_batch_peak_polish(env):
    """With DOA_FLAG_POLISH_PEAKS every peak whose neighbourhood the FP32 values do not decide is
    re-evaluated in FP64, so the peak indices equal the oracle's up to ties below float resolution
    (1e-6 relative); points left as computed are within the FP32 path's bound."""
    torch, doa = env
    insts = [synth.paper_density(i) for i in range(12)]
    masks = [0xF] * len(insts)
    tensors, status = _batch_solve(torch, doa, insts, masks, polish=True)
    assert np.all(status == 0)
    for inst, t in zip(insts, tensors):
        P = t[1].cpu().numpy().reshape(-1, inst.L)
        idx = t[2].cpu().numpy().reshape(-1, inst.d)
        cnt = t[4].cpu().numpy()
        for alg in range(4):
            ref = oracle.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
            assert db_error(P[alg], ref["P"]) < DB_TOL
            ok, ties = compare_peaks(idx[alg][:cnt[alg]], ref["idx"], ref["P"], 1e-6)
            assert ok, (inst.seed, alg, ties)
            for k in idx[alg][:cnt[alg]]:   # FP64 values rounded once, or FP32 values within the bound
                for q in range(max(k - 2, 0), min(k + 3, inst.L)):
                    assert abs(P[alg][q] / ref["P"][q] - 1.0) < 5e-4


def test_batch_edge_shapes(env):
    torch, doa = env
    insts = [synth.custom(2, 1, 5, [10.0], 20.0, 45.0, seed=1),           # L = 5
             synth.custom(3, 0, 64, [], 0.0, 60.0, seed=2),               # d = 0, L = 4
             synth.custom(9, 8, 700, None, 25.0, 0.25, seed=3),           # d = M - 1
             synth.custom(64, 8, 2500, None, 10.0, 0.05, seed=4),
             synth.custom(17, 3, 1, None, 10.0, 0.5, seed=5)]             # N = 1
    insts[0].angles = np.array([10.0])
    masks = [0xF, 0b0010, 0xF, 0b0110, 0b0010]
    tensors, status = _batch_solve(torch, doa, insts, masks)
    assert np.all(status == 0)
    for inst, mask, t in zip(insts, masks, tensors):
        P = t[1].cpu().numpy().reshape(-1, inst.L)
        slot = 0
        for alg in range(4):
            if (mask >> alg) & 1:
                ref = oracle.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
                if inst.N >= inst.M:   # rank-deficient R (N = 1) has an ill-posed noise basis
                    assert db_error(P[slot], ref["P"]) < DB_TOL
                slot += 1


# ------------------------------------------------------------------------------ Step-5, tensor cores
@pytest.mark.parametrize("M,d,step,L", [(16, 4, 0.01, 18001), (64, 8, 0.01, 18001), (37, 5, 0.05, 3601),
                                        (48, 47, 0.1, 1801), (64, 0, 0.5, 361)])
def test_scan_tensor_core_split(env, M, d, step, L):
    """BF16x3 / FP16x3 tcgen05 scan with near-null re-evaluation: within 0.01 dB of the oracle."""
    torch, doa = env
    inst = synth.custom(M, d, 4 * M + 500, None if d <= 8 else np.linspace(-70, 70, d) + 0.31, 12.0, step,
                        seed=4000 + M + d)
    Ro = oracle.covariance(inst.X)
    ev_o, V_o, _ = oracle.eigh(Ro)
    for alg in (PHD, MUSIC, EV, MN):
        Co, _ = oracle.weighting(ev_o, V_o, d, alg)
        Bf = factor_from_decomposition(ev_o, V_o, d, alg)
        K = Bf.shape[1]
        Po, _ = oracle.scan(Co, -90.0, step, L)
        B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
        for prec in (doa.BF16X3, doa.FP16X3):
            P = torch.empty(L, dtype=torch.float32, device="cuda")
            doa.doa_scan(B, M, K, doa.grid(-90.0, step, L), P, prec=prec)
            torch.cuda.synchronize()
            err = db_error(P.cpu().numpy(), Po)
            assert err < DB_TOL, (alg, prec, err)
        P = torch.empty(L, dtype=torch.float32, device="cuda")
        doa.doa_scan(B, M, K, doa.grid(-90.0, step, L), P, prec=doa.BF16)      # one BF16 product
        torch.cuda.synchronize()
        assert np.all(np.isfinite(P.cpu().numpy()))


def test_scan_tensor_core_large_array_sampled(env):
    """Full large-array grid (M=64, d=8, 360001 points at 0.0005 deg): tensor-core split scan vs the
    oracle at sampled grid points, including every picked peak and its neighbours."""
    torch, doa = env
    inst = synth.large_array(0)
    Ro = oracle.covariance(inst.X)
    ev_o, V_o, _ = oracle.eigh(Ro)
    rng = np.random.default_rng(1)
    for alg in (MUSIC, EV):
        Co, _ = oracle.weighting(ev_o, V_o, inst.d, alg)
        Bf = factor_from_decomposition(ev_o, V_o, inst.d, alg)
        B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
        g = doa.grid(inst.lo, inst.step, inst.L)
        for prec in (doa.FP32, doa.BF16X3, doa.FP16X3):
            P = torch.empty(inst.L, dtype=torch.float32, device="cuda")
            doa.doa_scan(B, inst.M, Bf.shape[1], g, P, prec=prec)
            idx = torch.zeros(inst.d, dtype=torch.int32, device="cuda")
            val = torch.zeros(inst.d, dtype=torch.float32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            doa.doa_peaks(P, inst.d, idx, val, cnt)
            torch.cuda.synchronize()
            Pg = P.cpu().numpy()
            pk = idx.cpu().numpy()[:cnt.item()]
            ks = set(rng.integers(0, inst.L, 1500).tolist())
            for k in pk:
                ks.update(range(max(0, k - 3), min(inst.L, k + 4)))
            ks = sorted(ks)
            Po = np.array([oracle.scan(Co, inst.lo + k * inst.step, inst.step, 1)[0][0] for k in ks])
            err = float(np.max(np.abs(10 * np.log10(Pg[ks].astype(np.float64) / Po))))
            assert err < DB_TOL, (alg, prec, err)
            # the picked peaks are local maxima of the oracle's spectrum too
            for k in pk:
                a = [oracle.scan(Co, inst.lo + j * inst.step, inst.step, 1)[0][0] for j in (k - 1, k, k + 1)]
                assert a[1] >= a[0] and a[1] >= a[2]


# ------------------------------------------------------------------------------ Step-1, tensor cores
def tc_cov_tol(prec, N):
    """Relative error bound (max |R_gpu - R_oracle| / max |R|) of the tcgen05 covariance: the
    operand representation (BF16 2^-8; split BF16 ~2^-16; split FP16 ~2^-21, each doubled for the
    two factors) plus FP32 accumulation over 2N products (4 sqrt(2N) 2^-24)."""
    rep = {1: 2 * 2.0 ** -8, 2: 4 * 2.0 ** -16, 3: 4 * 2.0 ** -21}[prec]
    return rep + 4 * np.sqrt(2 * N) * 2.0 ** -24


@pytest.mark.parametrize("M,N", [(8, 1024), (16, 4096), (37, 1000), (64, 16384), (64, 33), (5, 20000)])
def test_covariance_tensor_core(env, M, N):
    torch, doa = env
    inst = synth.custom(M, min(4, M - 1), N, None, 10.0, 0.1, seed=5000 + M * 11 + N)
    ld = N + (N & 1)                      # TMA needs an even row pitch (16-byte rows)
    Xh = np.zeros((M, ld), np.complex64)
    Xh[:, :N] = inst.X
    X = torch.from_numpy(Xh).cuda()[:, :N]
    Ro = oracle.covariance(inst.X)
    scale = np.max(np.abs(Ro))
    for prec in (doa.BF16, doa.BF16X3, doa.FP16X3):
        tol = tc_cov_tol(prec, N)
        R64 = torch.full((M, M), float("nan"), dtype=torch.complex128, device="cuda")
        doa.doa_covariance(X, R64=R64, prec=prec)
        torch.cuda.synchronize()
        Rg = R64.cpu().numpy()
        err = np.max(np.abs(Rg - Ro)) / scale
        assert err < tol, (prec, err)
        assert np.array_equal(Rg, Rg.conj().T)


def test_covariance_tensor_core_rejects_unaligned(env):
    torch, doa = env
    X = torch.zeros((8, 101), dtype=torch.complex64, device="cuda")
    R = torch.empty((8, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(doa.DoaError):
        doa.doa_covariance(X[:, :100], R64=R, prec=doa.FP16X3)     # row pitch 101 is odd
    doa.doa_covariance(X[:, :100], R64=R, prec=doa.FP32)           # the FP32 path takes any pitch
