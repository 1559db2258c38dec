"""Pins of the MLP reference (oracle/mlp.py) on the CPU: its backward is the
gradient of its forward (central differences, float64), and bf16 rounding
is round-to-nearest-even on the float32 bit pattern."""
import numpy as np

from oracle import mlp as om


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-5, 1.0 + 2 ** -9])
    r = om.bf16(x)
    assert r[0] == 1.0 and r[3] == -2.5
    assert r[1] == 1.0                       # tie -> even
    assert r[2] == 1.0 + 4 * 2 ** -8          # tie -> even (up)
    assert r[5] == 1.0                        # below half an ulp
    assert abs(r[4] - 3.0e-5) <= 3.0e-5 * 2 ** -8


def test_backward_is_gradient_of_forward():
    rng = np.random.default_rng(0)
    p = rng.normal(scale=0.2, size=om.n_params())
    x = rng.uniform(-1, 1, size=(5, om.IN))
    gy = rng.normal(size=(5, om.OUT))
    g = om.backward(p, x, gy)
    f = lambda q: float(np.sum(gy * om.forward(q, x)[0]))
    h = 1e-6
    idx = rng.choice(p.size, 40, replace=False)
    for i in idx:
        e = np.zeros_like(p); e[i] = h
        fd = (f(p + e) - f(p - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd))
