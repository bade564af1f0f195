"""GPU parity of the root form of the ULA scan (Aberth-Ehrlich roots in FP64) against the oracle
(numpy.roots on the explicit C): single calls on the same factor and batch solves end to end."""
import numpy as np
import pytest

import oracle
from paper_2007_14135_gb300 import synth
from tests.gpu_common import EV, MN, MUSIC, PHD, factor_from_decomposition, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.mark.parametrize("M,d,snr", [(8, 2, 10.0), (16, 4, 15.0), (12, 3, 0.0), (33, 5, 10.0), (64, 8, 12.0),
                                     (2, 1, 10.0)])
def test_root_music_single_matches_oracle(env, M, d, snr):
    torch, doa = env
    ang = None if d <= 8 else np.linspace(-60, 60, d)
    inst = synth.custom(M, d, 4096, ang, snr, 1.0, seed=900 + M)
    ev, V, _ = oracle.eigh(oracle.covariance(inst.X))
    for alg in (MUSIC, EV, PHD, MN):
        Bf = factor_from_decomposition(ev, V, d, alg)
        B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
        th = torch.full((d,), -99.0, dtype=torch.float64, device="cuda")
        info = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        doa.doa_root_music(B, M, Bf.shape[1], d, th, info)
        torch.cuda.synchronize()
        assert info.item() == 0
        want, _ = oracle.root_music(Bf @ Bf.conj().T, d)
        np.testing.assert_allclose(th.cpu().numpy(), want, rtol=0, atol=1e-6, err_msg=f"alg {alg}")


def test_root_music_batch(env):
    torch, doa = env
    insts = [synth.paper_density(i) for i in range(6)] + [synth.single_c1()]
    keep, probs = [], []
    for inst in insts:
        X = torch.from_numpy(inst.X).cuda()
        P = torch.empty(4 * inst.L, dtype=torch.float32, device="cuda")
        idx = torch.full((4 * inst.d,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(4 * inst.d, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
        ra = torch.full((4 * inst.d,), float("nan"), dtype=torch.float64, device="cuda")
        keep.append((X, P, idx, val, cnt, ra))
        probs.append(doa.make_problem(X, inst.d, 0xF, doa.grid(inst.lo, inst.step, inst.L), P, idx, val, cnt,
                                      root_angle=ra))
    plan = doa.BatchPlan(probs)
    ws = doa.workspace(plan)
    status = torch.full((len(insts),), -1, dtype=torch.int32, device="cuda")
    doa.doa_solve_batch(plan, ws, status)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for inst, t in zip(insts, keep):
        ra = t[5].cpu().numpy().reshape(4, inst.d)
        for alg in range(4):
            ref = oracle.solve(inst.X, inst.d, alg, inst.lo, inst.step, inst.L)
            want, _ = oracle.root_music(ref["C"], inst.d)
            np.testing.assert_allclose(ra[alg], want, rtol=0, atol=1e-6, err_msg=f"seed {inst.seed} alg {alg}")


@pytest.mark.parametrize("M,d", [(3, 2), (5, 4), (8, 7)])
def test_root_music_one_noise_vector(env, M, d):
    """d = M - 1: one noise eigenvector, a degree 2M-2 polynomial with M-1 roots inside."""
    torch, doa = env
    inst = synth.custom(M, d, 2000, np.linspace(-50, 50, d) + 0.3, 20.0, 1.0, seed=950 + M)
    ev, V, _ = oracle.eigh(oracle.covariance(inst.X))
    Bf = factor_from_decomposition(ev, V, d, MUSIC)
    B = torch.from_numpy(np.ascontiguousarray(Bf.T).reshape(-1)).cuda()
    th = torch.full((d,), -99.0, dtype=torch.float64, device="cuda")
    info = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    doa.doa_root_music(B, M, 1, d, th, info)
    torch.cuda.synchronize()
    assert info.item() == 0
    want, _ = oracle.root_music(Bf @ Bf.conj().T, d)
    np.testing.assert_allclose(th.cpu().numpy(), want, rtol=0, atol=1e-6)
