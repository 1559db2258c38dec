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


def _rss_tolerance(ref, rss, k=2.0 ** -5, floor=1e-5):
    """Per-entry bound k * rss + floor * max|ref|.  The GPU and the reference
    round to bf16 at the same points; they differ by FP32 against FP64
    accumulation and by the few stored bf16 values that round the other way
    (one bf16 ulp, 2^-8 relative, of single terms of a sum), so an entry's
    error is a small multiple of 2^-8 times the root sum of squares of its
    terms.  A wrong entry (a dropped, swapped or misplaced term or row) is off
    by the size of the entry itself, which for a sum of B random-sign terms is
    of the order of that root sum of squares: far above k = 2^-5."""
    return k * rss + floor * float(np.max(np.abs(ref)))


def _assert_entries(got, ref, rss, what):
    got = np.asarray(got); ref = np.asarray(ref)
    assert got.shape == ref.shape
    tol = _rss_tolerance(ref, rss)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} entries off, worst "
                           f"{np.max(np.abs(got - ref) / tol):.2f} x tolerance")


@pytest.mark.parametrize("B", [1, 37, 256, 1000, 20000])   # 20000: split-K weight gradients
def test_forward_backward_match_reference(mlpmod, B):
    """Every output and every entry of every weight and bias gradient against
    the CPU reference with the same bf16 rounding points."""
    rng = np.random.default_rng(B)
    p = mlpmod.init_params(B)
    x = rng.uniform(-1, 1, size=(B, om.IN)).astype(np.float32)
    gy = rng.normal(size=(B, om.OUT)).astype(np.float32)
    m = mlpmod.MLP(p, max(B, 64))
    y = m.forward(torch.as_tensor(x)).cpu().numpy()
    yr, cache = om.forward(p, x, "bf16")
    a3, W4 = cache[6], cache[10]
    b4 = om.unpack(p)[7]
    _assert_entries(y, yr, np.sqrt((a3 ** 2) @ (W4 ** 2).T + b4 ** 2), "y")
    g = m.backward(torch.as_tensor(x), torch.as_tensor(gy)).cpu().numpy()
    gr, terms = om.backward(p, x, gy, "bf16", return_terms=True)
    gblocks, rblocks = _blocks(g), _blocks(gr)
    # block order: W1, b1, W2, b2, W3, b3, W4, b4; terms are listed from layer 4 down
    for layer, (gl, al) in zip((4, 3, 2, 1), terms):
        iw = 2 * (layer - 1)
        shape = (gl.shape[1], al.shape[1])
        _assert_entries(gblocks[iw].reshape(shape), rblocks[iw].reshape(shape),
                        np.sqrt((gl ** 2).T @ (al ** 2)), f"grad W{layer}")
        _assert_entries(gblocks[iw + 1], rblocks[iw + 1], np.sqrt(np.sum(gl ** 2, axis=0)),
                        f"grad b{layer}")


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
