"""Proposal network on the GPU (tcgen05 GEMMs + elementwise kernels) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import mlp as mlp_oracle
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _bf16(torch, x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _rounded_params(torch, net):
    return [(_bf16(torch, W), b) for W, b in net.params_numpy()]


def _cos_rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))
    rel = float(np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300))
    return cos, rel


def _batch(rng, B):
    X = rng.standard_normal((B, 272)).astype(np.float32) * 0.3
    Y = (rng.random((B, 181)) < 0.02).astype(np.float32)
    return X, Y


@pytest.mark.parametrize("B", [8, 200, 1024])
def test_forward_matches_oracle(env, B):
    torch, doa = env
    net = doa.Mlp(seed=11)
    rng = np.random.default_rng(B)
    X, _ = _batch(rng, B)
    ws = net.workspace(B)
    probs = torch.empty((B, 181), dtype=torch.float32, device="cuda")
    logits = torch.empty((B, 181), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(X).cuda(), ws, probs=probs, logits=logits)
    torch.cuda.synchronize()
    z_ref, _ = mlp_oracle.forward(_rounded_params(torch, net), _bf16(torch, X))
    cos, rel = _cos_rel(logits.cpu().numpy(), z_ref)
    assert cos > 0.9999 and rel < 2e-2, (cos, rel)
    np.testing.assert_allclose(probs.cpu().numpy(), 1 / (1 + np.exp(-logits.cpu().numpy())), rtol=1e-5)


def test_gradients_match_oracle(env):
    torch, doa = env
    B = 512
    net = doa.Mlp(seed=12)
    rng = np.random.default_rng(3)
    X, Y = _batch(rng, B)
    ws = net.workspace(B)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.backward(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), ws, loss=loss)
    torch.cuda.synchronize()
    l_ref, g_ref = mlp_oracle.loss_and_grads(_rounded_params(torch, net), _bf16(torch, X), Y.astype(np.float64))
    assert abs(loss.item() - l_ref) < 1e-2 * abs(l_ref)
    for l in range(4):
        gW = net.buf["gW"][l].cpu().numpy()
        gb = net.buf["gb"][l].cpu().numpy()
        for got, ref in ((gW, g_ref[l][0]), (gb, g_ref[l][1])):
            cos, rel = _cos_rel(got, ref)
            assert cos > 0.999 and rel < 5e-2, (l, cos, rel)


def test_adam_update_matches_oracle(env):
    torch, doa = env
    B = 256
    net = doa.Mlp(seed=13)
    rng = np.random.default_rng(4)
    X, Y = _batch(rng, B)
    ws = net.workspace(B)
    before = [t.cpu().numpy().astype(np.float64) for t in net.buf["W"]]
    net.backward(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), ws)
    grads = [t.cpu().numpy().astype(np.float64) for t in net.buf["gW"]]
    net.adam(1e-3)
    torch.cuda.synchronize()
    for l in range(4):
        w_ref, _, _ = mlp_oracle.adam(before[l], 0.0, 0.0, grads[l], 1e-3, 0.9, 0.999, 1e-8, 1)
        np.testing.assert_allclose(net.buf["W"][l].cpu().numpy(), w_ref, rtol=1e-5, atol=1e-7)
        # the BF16 copies follow the masters
        Wh = net.buf["Wh"][l].float().cpu().numpy()
        np.testing.assert_allclose(Wh, _bf16(torch, net.buf["W"][l].cpu().numpy()), rtol=0, atol=0)
        WhT = net.buf["WhT"][l].float().cpu().numpy()[:, :Wh.shape[0]]
        np.testing.assert_array_equal(WhT, Wh.T)


def test_training_reduces_loss_and_checkpoint_roundtrip(env, tmp_path):
    torch, doa = env
    B = 512
    net = doa.Mlp(seed=14)
    rng = np.random.default_rng(5)
    proj = rng.standard_normal((272, 181)).astype(np.float32) * 0.2
    X = rng.standard_normal((4096, 272)).astype(np.float32) * 0.3
    Y = (X @ proj > 0.35).astype(np.float32)               # a learnable multi-label target
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    ws = net.workspace(B)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for step in range(160):
        i = (step * B) % 4096
        net.backward(Xd[i:i + B], Yd[i:i + B], ws, loss=loss)
        net.adam(2e-3)
        hist.append(loss.item())
    assert np.mean(hist[-16:]) < 0.6 * np.mean(hist[:16]), (hist[:4], hist[-4:])
    path = str(tmp_path / "net.bin")
    net.save(path)
    net2 = doa.Mlp(seed=99)
    net2.load(path)
    p1 = torch.empty((B, 181), device="cuda")
    p2 = torch.empty((B, 181), device="cuda")
    net.forward(Xd[:B], ws, probs=p1)
    net2.forward(Xd[:B], net2.workspace(B), probs=p2)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2) and net2.t == net.t
