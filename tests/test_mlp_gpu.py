"""GPU MLP kernels (BF16 tensor-core GEMMs, FP32 accumulation) against the
CPU reference with the same bf16 rounding points: agreement within BF16
tolerance."""
import numpy as np
import pytest
import torch

from oracle import mlp as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mlpmod():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import mlp
    return mlp


def _blocks(v):
    sizes = [om.H * om.IN, om.H, om.H * om.H, om.H, om.H * om.H, om.H, om.OUT * om.H, om.OUT]
    out, o = [], 0
    for n in sizes:
        out.append(v[o:o + n]); o += n
    return out


@pytest.mark.parametrize("B", [1, 37, 256, 1000, 20000])   # 20000: split-K weight gradients
def test_forward_backward_match_reference(mlpmod, B):
    rng = np.random.default_rng(B)
    p = mlpmod.init_params(B)
    x = rng.uniform(-1, 1, size=(B, om.IN)).astype(np.float32)
    gy = rng.normal(size=(B, om.OUT)).astype(np.float32)
    m = mlpmod.MLP(p, max(B, 64))
    y = m.forward(torch.as_tensor(x)).cpu().numpy()
    yr, _ = om.forward(p, x, "bf16")
    assert np.max(np.abs(y - yr)) <= 2e-2 * np.max(np.abs(yr)) + 1e-6
    g = m.backward(torch.as_tensor(x), torch.as_tensor(gy)).cpu().numpy()
    gr = om.backward(p, x, gy, "bf16")
    for a, b in zip(_blocks(g), _blocks(gr)):
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b) + 1e-6


def test_training_reduces_loss(mlpmod):
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, size=(4096, om.IN)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], np.cos(x[:, 2] + x[:, 3])], 1).astype(np.float32)
    m = mlpmod.MLP(mlpmod.init_params(0), 512)
    X = torch.as_tensor(x).cuda(); T = torch.as_tensor(t).cuda()
    first = None
    for s in range(600):
        idx = torch.randint(0, 4096, (512,), device="cuda")
        loss = m.train_step(X[idx].contiguous(), T[idx].contiguous(), lr=2e-3)
        if first is None:
            first = float(loss.item())
    y = m.forward(X[:512]).cpu().numpy()
    final = float(np.mean((y - t[:512]) ** 2))
    assert final < 0.1 * first
    # the loss reported by the device equals the reference loss at the same weights
    params = m.params().cpu().numpy()
    ref = om.loss(params, x[:512], t[:512], "bf16")
    assert abs(final - ref) <= 3e-2 * ref + 1e-6
