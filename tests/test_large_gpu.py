"""The 12-mode, cutoff-5 all-detected workload at full size (5^12 = 244 M
probabilities, 4.6 G walk amplitudes): forward and VJP in one go with the
whole walk resident (about 150 GB of workspace).  Sampled probabilities are
computed one by one by the oracle; the VJP is checked by the exact identities
c conj(grad_c) = sum conj(gbar) p and Euler homogeneity
sum conj(gbar) |k| p = sum 2 A conj(grad_A)."""
import time

import numpy as np
import pytest
import torch

import oracle
from oracle import triple as otriple
from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_gbs_m12_c5_forward_and_vjp():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag as fd
    free, total = torch.cuda.mem_get_info()
    circ = inputs.workload("gbs_m12_c5")[0]
    cut = circ.cutoffs
    flags = fd.FK_FLAG_B_ZERO
    need = fd.fk_workspace_size(12, cut, 1, fd.FK_OP_DIAG_VJP, flags)
    if need + 3 * 5 ** 12 * 16 > free:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory")
    A, b, c = fd.fk_gaussian_to_triple(circ.V, circ.mean)
    Ad = torch.tensor(A[None]).cuda(); bd = torch.tensor(b[None]).cuda()
    cd = torch.tensor([c], dtype=torch.complex128).cuda()
    ws = fd.workspace(need)
    t0 = time.perf_counter()
    p, _ = fd.fock_diag_probs_batched(Ad, bd, cd, cut, flags=flags, ws=ws)
    fd.check_workspace(ws)
    t_fwd = time.perf_counter() - t0
    pr = p[0].real
    assert float(pr.min()) > -1e-15
    s = float(pr.sum())
    assert 0.3 < s <= 1 + 1e-12
    assert float(p[0].imag.abs().max()) < 1e-14
    # sampled probabilities against the oracle's naive walk, one by one
    Ao, bo, co = otriple.gaussian_to_triple(circ.V, circ.mean)
    w = oracle.Walk(Ao, bo, co, cut)
    rng = np.random.default_rng(12)
    pats = [(0,) * 12, (4,) + (0,) * 11, (0,) * 11 + (4,)]
    for _ in range(24):
        n = np.zeros(12, int)
        sup = rng.choice(12, size=int(rng.integers(1, 5)), replace=False)
        n[sup] = rng.integers(1, 5, size=sup.size)
        pats.append(tuple(n))
    for _ in range(6):
        n = np.zeros(12, int)
        sup = rng.choice(12, size=6, replace=False)
        n[sup] = rng.integers(1, 3, size=6)
        pats.append(tuple(n))
    pc = p[0].cpu()
    for n in pats:
        ref, _ = w.prob(n)
        got = complex(pc[n])
        assert abs(got - ref) <= 1e-10 * abs(ref) + 1e-12, (n, got, ref)
    del pc
    # VJP of sum_n w_n Re p_n with the walk kept from the forward
    wgt = torch.randn(p.shape, dtype=torch.float64, device="cuda").to(torch.complex128)
    t0 = time.perf_counter()
    gA, gb, gc = fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, wgt, ws, flags=flags)
    fd.check_workspace(ws)
    t_vjp = time.perf_counter() - t0
    lc = complex((wgt.conj() * p).sum())
    assert abs(c * np.conj(gc[0].item()) - lc) <= 1e-10 * float((wgt.abs() * p.abs()).sum())
    # |k| = 2 sum_j n_j for the diagonal index of pattern n
    ksum = torch.zeros(cut, dtype=torch.float64, device="cuda")
    for j in range(12):
        shape = [1] * 12
        shape[j] = 5
        ksum = ksum + 2 * torch.arange(5, dtype=torch.float64, device="cuda").reshape(shape)
    lhs = complex((wgt[0].conj() * ksum * p[0]).sum())
    rhs = complex(np.sum(2 * A * np.conj(gA[0].cpu().numpy())))
    assert abs(lhs - rhs) <= 1e-9 * float((wgt[0].abs() * ksum * p[0].abs()).sum())
    print(f"M=12 C=5: workspace {need / 1e9:.1f} GB, forward {t_fwd:.2f} s, VJP {t_vjp:.2f} s")
