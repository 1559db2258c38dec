"""Large batches of small circuits: with at least two circuits per block the
all-detected walk runs circuit by circuit in each block (block barriers
between its phases) instead of level by level over the grid.  Every circuit
must come out as in a small launch (the level-synchronous mode) and as the
oracle says, forward and VJP, on both engines, with b = 0 and b != 0 and
with the early stop."""
import numpy as np
import pytest
import torch

import oracle
from oracle import gradients as ograd
from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu

B = 4096   # more than twice the blocks of any launch on 152 SMs


@pytest.fixture(scope="module")
def fd():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    return fockdiag


def batch(cut, withb, seed):
    rng = np.random.default_rng(seed)
    As, bs = [], []
    for _ in range(B):
        A, b = inputs.random_symmetric(2 * len(cut), rng, scale=0.2, with_b=withb)
        As.append(A); bs.append(b)
    c = 0.8 - 0.1j + 0.05 * rng.normal(size=B)
    w = rng.normal(size=(B,) + cut) + 1j * rng.normal(size=(B,) + cut)
    t = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.complex128).cuda()
    return t(np.stack(As)), t(np.stack(bs)), t(c), t(w)


def run(fd, A, b, c, w, cut, flags):
    p, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags)
    g = fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags)
    fd.check_workspace(ws)
    return p, g


@pytest.mark.parametrize("engine", ["tensor", "fp64"])
@pytest.mark.parametrize("cut,withb", [((4, 3), True), ((5, 4), False), ((3, 2, 3), True)])
def test_many_small_circuits_match_small_launch_and_oracle(fd, engine, cut, withb):
    fl = (fd.FK_FLAG_ENGINE_TENSOR if engine == "tensor" else fd.FK_FLAG_ENGINE_FP64) | \
        (0 if withb else fd.FK_FLAG_B_ZERO)
    A, b, c, w = batch(cut, withb, 11 + sum(cut))
    p, (gA, gb, gc) = run(fd, A, b, c, w, cut, fl)
    # the same circuits in launches of 8 (level by level over the grid)
    for lo in (0, 2000, B - 8):
        sl = slice(lo, lo + 8)
        p8, (gA8, gb8, gc8) = run(fd, A[sl].contiguous(), b[sl].contiguous(), c[sl].contiguous(),
                                 w[sl].contiguous(), cut, fl)
        assert torch.equal(p[sl], p8)   # the same arithmetic per amplitude
        for x, y in ((gA[sl], gA8), (gb[sl], gb8), (gc[sl], gc8)):
            scale = max(float(torch.max(torch.abs(y))), 1e-300)
            assert float(torch.max(torch.abs(x - y))) <= 1e-12 * scale
    # against the oracle
    for i in (0, 1, 2047, B - 1):
        An, bn, cn = A[i].cpu().numpy(), b[i].cpu().numpy(), complex(c[i].item())
        G = oracle.full_lattice(An, bn, cn, oracle.dm_dims(cut))
        gfull = np.zeros_like(G)
        wn = w[i].cpu().numpy()
        ref = np.zeros(cut, np.complex128)
        for n in np.ndindex(*cut):
            k = tuple(v for a in n for v in (a, a))
            ref[n] = G[k]
            gfull[k] = wn[n]
        got = p[i].cpu().numpy()
        big = np.abs(ref) > 1e-12
        assert np.max(np.abs(got - ref)[big] / np.abs(ref[big])) <= 1e-10
        rA, rb, rc = ograd.vjp(G, gfull, cn)
        scale = np.max(np.abs(rA))
        assert np.max(np.abs(gA[i].cpu().numpy() - rA)) <= 1e-8 * scale
        if withb:
            assert np.max(np.abs(gb[i].cpu().numpy() - rb)) <= 1e-8 * max(np.max(np.abs(rb)), 1e-300)
        assert abs(gc[i].item() - rc) <= 1e-8 * abs(rc)


def test_many_small_circuits_early_stop(fd):
    """The probability-sum stop decides per circuit; in the circuit-per-block
    mode the decisions and outputs equal those of small launches."""
    cut = (6, 6)
    A, b, c, w = batch(cut, True, 5)
    p, lev, ws = fd.fock_diag_probs_stop_batched(A, b, c, cut, 1e-3)
    fd.check_workspace(ws)
    g = fd.fock_diag_probs_stop_vjp_batched(A, b, c, cut, 1e-3, w, ws)
    for lo in (0, 3000):
        sl = slice(lo, lo + 8)
        p8, lev8, ws8 = fd.fock_diag_probs_stop_batched(A[sl].contiguous(), b[sl].contiguous(),
                                                        c[sl].contiguous(), cut, 1e-3)
        fd.check_workspace(ws8)
        assert torch.equal(lev[sl], lev8)
        assert torch.equal(p[sl], p8)
        g8 = fd.fock_diag_probs_stop_vjp_batched(A[sl].contiguous(), b[sl].contiguous(),
                                                 c[sl].contiguous(), cut, 1e-3, w[sl].contiguous(), ws8)
        for x, y in zip(g, g8):
            scale = max(float(torch.max(torch.abs(y))), 1e-300)
            assert float(torch.max(torch.abs(x[sl] - y))) <= 1e-12 * scale
