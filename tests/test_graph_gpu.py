"""Both walks are stream-ordered and allocate nothing, so a whole batched
call (control-block reset, plan copy, one cooperative launch) can be captured
into a CUDA graph; replays reproduce the eager result bit for bit."""
import numpy as np
import pytest
import torch

from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    return fockdiag


def _capture(fn, s):
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()                                   # eager run on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn()
    return g


def test_conditional_batch_graph_replay(fd):
    mask = (1, 1, 0)
    circs = inputs.workload("cond_m3_batch64", 8)
    cuts = [cc.cutoffs for cc in circs]
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = torch.tensor(np.stack([t[0] for t in trip])).cuda()
    b = torch.tensor(np.stack([t[1] for t in trip])).cuda()
    c = torch.tensor(np.array([t[2] for t in trip])).cuda()
    rho, offs, ws = fd.fock_conditional_dm_batched(A, b, c, cuts, mask)
    ref = rho.clone()
    s = torch.cuda.Stream()
    g = _capture(lambda: fd.fock_conditional_dm_batched(A, b, c, cuts, mask, rho=rho, ws=ws,
                                                        stream=s), s)
    for _ in range(2):
        rho.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(rho, ref)
    fd.check_workspace(ws)


def test_diag_forward_vjp_graph_replay(fd):
    circs = inputs.workload("gbs_m8_c6_batch16", 4)
    cut = (4, 4, 3, 3, 4, 3, 3, 4)
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = torch.tensor(np.stack([t[0] for t in trip])).cuda()
    b = torch.tensor(np.stack([t[1] for t in trip])).cuda()
    c = torch.tensor(np.array([t[2] for t in trip])).cuda()
    flags = fd.FK_FLAG_B_ZERO
    p, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags)
    w = torch.randn(p.shape, dtype=torch.float64, device="cuda").to(torch.complex128)
    gA, gb, gc = fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags)
    ref = (p.clone(), gA.clone(), gc.clone())
    s = torch.cuda.Stream()

    def step():
        fd.fock_diag_probs_batched(A, b, c, cut, probs=p, flags=flags, ws=ws, stream=s)
        fd.fock_diag_probs_vjp_batched(A, b, c, cut, w, ws, flags=flags, stream=s, out=(gA, gb, gc))

    g = _capture(step, s)
    p.zero_(); gA.zero_(); gc.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(p, ref[0]) and torch.equal(gA, ref[1]) and torch.equal(gc, ref[2])
    fd.check_workspace(ws)
