"""CPU reference of the proposal MLP.  TEST INFRASTRUCTURE ONLY.

The paper defines no learned model (Sec. 1 leaves ansatz, cost and target
outside its scope); this is the plain definition of the one the library
trains: y = W4 s(W3 s(W2 s(W1 x + b1) + b2) + b3) + b4 with s(z) = z
sigmoid(z) (SiLU), and the MSE loss mean over the batch and the two outputs
of (y - t)^2.

Two arithmetic modes:
  * exact: float64 throughout (pinned by central finite differences);
  * bf16: float64 arithmetic with rounding to bfloat16 (round to nearest
    even) at the points where the device stores bf16 -- the input, the
    weights, the hidden activations and the back-propagated gradients --
    so the GPU kernels can be compared element by element within BF16
    tolerance.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 15, 256, 2


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    shapes = [(H, IN), (H,), (H, H), (H,), (H, H), (H,), (OUT, H), (OUT,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    assert o == p.size
    return out


def n_params():
    return H * IN + H + 2 * (H * H + H) + OUT * H + OUT


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, mode="exact"):
    """Returns y and the cache for backward."""
    r = bf16 if mode == "bf16" else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(params)
    W1, W2, W3, W4 = r(W1), r(W2), r(W3), r(W4)
    a0 = r(x)
    z1 = a0 @ W1.T + b1
    a1 = r(silu(z1))
    z2 = a1 @ W2.T + b2
    a2 = r(silu(z2))
    z3 = a2 @ W3.T + b3
    a3 = r(silu(z3))
    y = a3 @ W4.T + b4
    return y, (a0, z1, a1, z2, a2, z3, a3, W1, W2, W3, W4)


def backward(params, x, gy, mode="exact", return_terms=False):
    """Packed gradient of sum(gy * y) with respect to the parameters.

    With ``return_terms`` also the factors of each weight-gradient sum over
    the batch, [(g_l, a_{l-1})] for l = 4, 3, 2, 1 (gW_l = g_l^T a_{l-1},
    gb_l = sum_k g_l[k]), for tests that size tolerances per entry."""
    r = bf16 if mode == "bf16" else (lambda a: np.asarray(a, np.float64))
    _, (a0, z1, a1, z2, a2, z3, a3, W1, W2, W3, W4) = forward(params, x, mode)
    g = r(gy)
    gW4 = g.T @ a3
    gb4 = g.sum(0)
    g3 = r((g @ W4) * dsilu(z3))
    gW3 = g3.T @ a2
    gb3 = g3.sum(0)
    g2 = r((g3 @ W3) * dsilu(z2))
    gW2 = g2.T @ a1
    gb2 = g2.sum(0)
    g1 = r((g2 @ W2) * dsilu(z1))
    gW1 = g1.T @ a0
    gb1 = g1.sum(0)
    packed = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, gW4.ravel(), gb4])
    if return_terms:
        return packed, [(g, a3), (g3, a2), (g2, a1), (g1, a0)]
    return packed


def loss(params, x, t, mode="exact"):
    y, _ = forward(params, x, mode)
    return float(np.mean((y - t) ** 2))
