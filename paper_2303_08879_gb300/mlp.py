"""Python binding of the proposal MLP (include/fockdiag_mlp.h).

Marshalling only: forward, backward, loss and the Adam step run in the
library's CUDA kernels (BF16 tensor-core GEMMs with FP32 accumulation).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import fockdiag as fd

IN, HIDDEN, OUT = 15, 256, 2


def _lib():
    L = fd.lib()
    if not getattr(L, "_mlp_bound", False):
        P, I, Z, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
        L.fk_mlp_sizes.argtypes = [I, ctypes.POINTER(Z), ctypes.POINTER(Z),
                                   ctypes.POINTER(ctypes.c_int64)]
        L.fk_mlp_load.argtypes = [P, P, P]
        L.fk_mlp_forward.argtypes = [P, I, P, P, P, Z, P]
        L.fk_mlp_backward.argtypes = [P, I, P, P, P, P, Z, P]
        L.fk_mlp_train_step.argtypes = [P, I, P, P, F, F, F, F, I, P, P, Z, P]
        L._mlp_bound = True
    return L


def n_params():
    n = ctypes.c_int64(0)
    fd._check(_lib().fk_mlp_sizes(1, None, None, ctypes.byref(n)), "fk_mlp_sizes")
    return int(n.value)


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (packed FP32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fo, fi in ((HIDDEN, IN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (OUT, HIDDEN)):
        s = 1.0 / np.sqrt(fi)
        parts.append(rng.uniform(-s, s, size=fo * fi))
        parts.append(rng.uniform(-s, s, size=fo))
    return np.concatenate(parts).astype(np.float32)


class MLP:
    """Device-resident model state plus a workspace sized for `batch`."""

    def __init__(self, params, batch, device="cuda"):
        self.device = torch.device(device)
        self.batch = int(batch)
        sb, wb = ctypes.c_size_t(0), ctypes.c_size_t(0)
        n = ctypes.c_int64(0)
        fd._check(_lib().fk_mlp_sizes(self.batch, ctypes.byref(sb), ctypes.byref(wb),
                                      ctypes.byref(n)), "fk_mlp_sizes")
        self.n_params = int(n.value)
        self.state = fd.workspace(sb.value, self.device)
        self.ws = fd.workspace(wb.value, self.device)
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step_count = 0
        self.load(params)

    def load(self, params):
        p = torch.as_tensor(np.asarray(params, np.float32), device=self.device).contiguous()
        assert p.numel() == self.n_params
        fd._check(_lib().fk_mlp_load(fd._ptr(self.state), fd._ptr(p), fd._stream(None)),
                  "fk_mlp_load")
        self.step_count = 0

    def params(self):
        return self.state[: self.n_params * 4].view(torch.float32).clone()

    def forward(self, x):
        x = x.to(self.device, torch.float32).contiguous()
        B = x.shape[0]
        assert B <= self.batch and x.shape[1] == IN
        y = torch.empty((B, OUT), dtype=torch.float32, device=self.device)
        fd._check(_lib().fk_mlp_forward(fd._ptr(self.state), B, fd._ptr(x), fd._ptr(y),
                                        fd._ptr(self.ws), self.ws.numel(), fd._stream(None)),
                  "fk_mlp_forward")
        return y

    def backward(self, x, gy):
        x = x.to(self.device, torch.float32).contiguous()
        gy = gy.to(self.device, torch.float32).contiguous()
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        fd._check(_lib().fk_mlp_backward(fd._ptr(self.state), x.shape[0], fd._ptr(x), fd._ptr(gy),
                                         fd._ptr(g), fd._ptr(self.ws), self.ws.numel(),
                                         fd._stream(None)), "fk_mlp_backward")
        return g

    def train_step(self, x, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam step; returns the loss (a device tensor, no sync)."""
        self.step_count += 1
        fd._check(_lib().fk_mlp_train_step(fd._ptr(self.state), x.shape[0], fd._ptr(x), fd._ptr(t),
                                           lr, beta1, beta2, eps, self.step_count,
                                           fd._ptr(self.loss_buf), fd._ptr(self.ws),
                                           self.ws.numel(), fd._stream(None)),
                  "fk_mlp_train_step")
        return self.loss_buf


def _main(argv):
    """python -m paper_2303_08879_gb300.mlp [batch] [steps]: training steps of
    the model on random data (CUDA-event timed), for profiling the GEMMs."""
    import time
    batch = int(argv[0]) if argv else 65536
    steps = int(argv[1]) if len(argv) > 1 else 10
    dev = torch.device("cuda")
    m = MLP(init_params(0), batch, dev)
    gen = torch.Generator(device=dev).manual_seed(0)
    X = torch.rand((batch, IN), device=dev, generator=gen) * 2 - 1
    Y = torch.rand((batch, OUT), device=dev, generator=gen)
    for _ in range(3):
        m.train_step(X, Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        m.train_step(X, Y)
    e1.record()
    torch.cuda.synchronize()
    print(f"batch {batch}: {e0.elapsed_time(e1) / steps:.4f} ms per training step")


if __name__ == "__main__":
    import sys
    _main(sys.argv[1:])
