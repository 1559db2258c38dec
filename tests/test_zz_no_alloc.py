"""The allocation-free entry point, fock_diag_probs_static.

Some callers cannot allocate device memory (their host owns all of it, or
their loop must never allocate).  For them the library keeps one fixed
device array per GPU and runs the forward walk in it.  This file checks,
through the C ABI, that two calls in a row give the same probabilities as
the ordinary entry point with a caller-supplied workspace, and that sizes
beyond the array are refused.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-10, 1e-12


@pytest.fixture(scope="module")
def fd():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    return fockdiag


def _close(got, ref):
    err = np.abs(got - ref)
    big = np.abs(ref) > ATOL
    assert np.all(err[big] <= RTOL * np.abs(ref[big]))
    assert np.all(err[~big] <= ATOL)


def _static_call(fd, A, b, c, cut, probs, flags):
    L = fd.lib()
    st = ctypes.c_int(-1)
    cc = (ctypes.c_int * len(cut))(*cut)
    rc = L.fock_diag_probs_static(A.shape[0], ctypes.c_void_p(A.data_ptr()),
                                  ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                  len(cut), cc, ctypes.c_void_p(probs.data_ptr()), flags,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                  ctypes.byref(st))
    return rc, st.value


def test_static_workspace_matches_caller_workspace(fd):
    cases = [("gbs_m2_c10", (10, 10), fd.FK_FLAG_B_ZERO),
             ("cond_m3_batch64", (7, 6, 5), 0)]
    for name, cut, flags in cases:
        circs = inputs.workload(name, 3)
        trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
        A = torch.tensor(np.stack([t[0] for t in trip])).cuda()
        b = torch.tensor(np.stack([t[1] for t in trip])).cuda()
        c = torch.tensor(np.array([t[2] for t in trip])).cuda()
        ref, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags, for_vjp=False)
        fd.check_workspace(ws)
        ref = ref.cpu().numpy()
        outs = [torch.full((3,) + cut, float("nan"), dtype=torch.complex128, device="cuda")
                for _ in range(3)]
        rc, st = _static_call(fd, A, b, c, cut, outs[0], flags)   # loads the kernels
        assert rc == 0 and st == 0
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for out in outs[1:]:                        # two calls in a row
            rc, st = _static_call(fd, A, b, c, cut, out, flags)
            assert rc == 0 and st == 0
        torch.cuda.synchronize()
        # no device memory was allocated by the two calls
        assert torch.cuda.mem_get_info()[0] == free0
        for out in outs:
            _close(out.cpu().numpy(), ref)


def test_static_workspace_rejects_oversize(fd):
    cut = (6,) * 8                                  # 22 M amplitudes per circuit
    need = fd.fk_workspace_size(8, cut, 1, fd.FK_OP_DIAG, fd.FK_FLAG_B_ZERO)
    assert need > (16 << 20)
    A = torch.zeros((1, 16, 16), dtype=torch.complex128, device="cuda")
    b = torch.zeros((1, 16), dtype=torch.complex128, device="cuda")
    c = torch.ones((1,), dtype=torch.complex128, device="cuda")
    out = torch.empty((1,) + cut, dtype=torch.complex128, device="cuda")
    rc, _ = _static_call(fd, A, b, c, cut, out, fd.FK_FLAG_B_ZERO)
    assert rc == 3                                  # FK_EWORKSPACE
