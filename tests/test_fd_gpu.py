"""Central finite differences of the library's own forward against its VJP,
at the full size of one circuit of the 8-mode benchmark workload (M = 8,
C = 6: 1.68 M probabilities, 22 M walk amplitudes), through the C ABI.

The loss is L = sum_n w_n Re p_n with w ~ N(0, 1) (the loss the VJP of the
benchmark differentiates).  With PyTorch's convention the gradient of a
complex input z is dL/dRe z + i dL/dIm z (Sec. 2.5, eqs. dL_dB and dL_dA
times 2), so each real or imaginary part of an entry of A, b or c is
perturbed by +-h, h = 1e-6, on its own.  A enters only through (A + A^T)/2,
so moving the single entry A_mn moves the symmetric part by h/2 at (m, n)
and (n, m), and the symmetric gradient grad_A[m, n] is what the difference
quotient sees.  b = 0 in this workload: its entries are perturbed too, which
runs the walk with the offset_1 amplitudes (b != 0) at full size; the
gradient there is zero because every probability is even in b.

Central differences are accurate to O(h^2) plus the rounding of L divided by
h (about 1e-8 relative here), so the check is at 1e-6 of the largest
gradient entry: a sanity check on top of the element-wise oracle parity of
the VJP tests, not the 1e-8 gate.
"""
import numpy as np
import pytest
import torch

from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu

H = 1e-6
FD_RTOL = 1e-6


@pytest.fixture(scope="module")
def fd():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    return fockdiag


@pytest.fixture(scope="module")
def circuit(fd):
    circ = inputs.workload("gbs_m8_c6_batch16", 1)[0]
    A, b, c = fd.fk_gaussian_to_triple(circ.V, circ.mean)
    w = np.random.default_rng(1000).normal(size=circ.cutoffs)
    return A, b, c, circ.cutoffs, w


def cuda(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128).cuda()


def loss(fd, A, b, c, cut, w_dev):
    p, ws = fd.fock_diag_probs_batched(cuda(A[None]), cuda(b[None]), cuda([c]), cut)
    fd.check_workspace(ws)
    return float((w_dev * p[0].real).sum().item())


@pytest.mark.parametrize("engine", ["fp64", "tensor"])
def test_vjp_matches_central_differences_full_size(fd, circuit, engine):
    A, b, c, cut, w = circuit
    fd.fk_diag_set_engine(fd.FK_ENGINE_TENSOR if engine == "tensor" else fd.FK_ENGINE_FP64)
    try:
        w_dev = torch.as_tensor(w, device="cuda")
        Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([c])
        p, ws = fd.fock_diag_probs_batched(Ad, bd, cd, cut, flags=fd.FK_FLAG_B_ZERO)
        gA, gb, gc = fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(w[None]), ws,
                                                    flags=fd.FK_FLAG_B_ZERO)
        fd.check_workspace(ws)
        gA = gA[0].cpu().numpy(); gb = gb[0].cpu().numpy(); gc = complex(gc[0].item())
        scale = float(np.max(np.abs(gA)))
        assert scale > 0

        def quotient(perturb):
            lp = loss(fd, *perturb(+H), cut, w_dev)
            lm = loss(fd, *perturb(-H), cut, w_dev)
            return (lp - lm) / (2 * H)

        # diagonal and off-diagonal entries, first and last modes, both pair members
        for (m, n) in ((0, 0), (0, 1), (3, 9), (15, 15), (2, 13), (7, 8)):
            for part, unit in (("re", 1.0), ("im", 1j)):
                def pert(t, m=m, n=n, unit=unit):
                    Ap = A.copy()
                    Ap[m, n] += t * unit
                    return Ap, b, c
                q = quotient(pert)
                g = gA[m, n].real if part == "re" else gA[m, n].imag
                assert abs(q - g) <= FD_RTOL * scale, (m, n, part, q, g)
        for m in (0, 11):
            for part, unit in (("re", 1.0), ("im", 1j)):
                def pert(t, m=m, unit=unit):
                    bp = b.copy()
                    bp[m] += t * unit
                    return A, bp, c
                q = quotient(pert)
                g = gb[m].real if part == "re" else gb[m].imag
                assert abs(q - g) <= FD_RTOL * scale, (m, part, q, g)
        for part, unit in (("re", 1.0), ("im", 1j)):
            q = quotient(lambda t, unit=unit: (A, b, c + t * unit))
            g = gc.real if part == "re" else gc.imag
            assert abs(q - g) <= FD_RTOL * max(abs(gc), 1e-300), (part, q, g)
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
