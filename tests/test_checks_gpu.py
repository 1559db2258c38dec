"""Input and memory checks that stand in for a sanitizer, through the C ABI.

* FK_FLAG_CHECK_FINITE: a NaN or Inf planted on the host in A, b or c makes
  the workspace status FK_ENONFINITE, the walk does not run, and the context
  stays usable (the next call is FK_OK).  No GPU fault is involved.
* Poisoned workspace: every byte of the workspace is set to 0xFF (a NaN in
  every double) before the forward walk and its VJP.  An amplitude or
  adjoint read before it is written would carry a NaN into the outputs, so
  outputs that match the oracle show that every read location was written
  first (the claim the walk's storage relies on: each amplitude written once,
  before its readers; Sec. 3.1.4).
* Canaries: guard regions before and after the workspace and the outputs are
  filled with a pattern and must be unchanged afterwards; outputs are
  NaN-poisoned before the call and every slot must be written.
* Per-call engine flags and the default engine (tensor up to 8 kept modes).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import gradients as ograd
from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL, ATOL, VJP_RTOL = 1e-10, 1e-12, 1e-8
GUARD = 4096                       # bytes of canary on each side (keeps 256-byte alignment)
CANARY = 0xA5


@pytest.fixture(scope="module")
def fd():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    return fockdiag


def cuda(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128).cuda()


def assert_amp_close(got, ref):
    got = np.asarray(got); ref = np.asarray(ref)
    assert np.all(np.isfinite(got)), "an output slot was left unwritten (NaN)"
    err = np.abs(got - ref)
    big = np.abs(ref) > ATOL
    assert np.all(err[big] <= RTOL * np.abs(ref[big])), np.max(err[big] / np.abs(ref[big]))
    assert np.all(err[~big] <= ATOL)


def assert_grad_close(got, ref):
    got = np.asarray(got); ref = np.asarray(ref)
    assert np.all(np.isfinite(got))
    floor = 1e-12 * max(1.0, float(np.max(np.abs(ref))))
    big = np.abs(ref) > floor
    assert np.all(np.abs(got - ref)[big] <= VJP_RTOL * np.abs(ref)[big])
    assert np.all(np.abs(got - ref)[~big] <= floor)


class Guarded:
    """A device buffer of `nbytes` with canary regions around it."""

    def __init__(self, nbytes, fill):
        self.n = int(max(nbytes, 256) + 255) // 256 * 256
        self.raw = torch.full((self.n + 2 * GUARD,), CANARY, dtype=torch.uint8, device="cuda")
        self.raw[GUARD:GUARD + self.n] = fill
        self.inner = self.raw[GUARD:GUARD + self.n]

    def view(self, dtype, shape):
        count = int(np.prod(shape))
        return self.inner.view(dtype)[:count].view(shape)

    def check(self):
        torch.cuda.synchronize()
        head = self.raw[:GUARD].cpu().numpy()
        tail = self.raw[GUARD + self.n:].cpu().numpy()
        assert np.all(head == CANARY) and np.all(tail == CANARY), "a canary was overwritten"


def oracle_vjp(A, b, c, cut, gbar):
    G = oracle.full_lattice(A, b, c, oracle.dm_dims(cut))
    gfull = np.zeros_like(G)
    for n in np.ndindex(*cut):
        gfull[tuple(v for a in n for v in (a, a))] = gbar[n]
    return ograd.vjp(G, gfull, c)


@pytest.mark.parametrize("engine", ["fp64", "tensor"])
@pytest.mark.parametrize("cut,withb", [((5, 4, 5), True), ((4, 3, 3, 4), False), ((3, 2, 2, 2, 2, 3), False)])
def test_poisoned_workspace_and_canaries_diag(fd, engine, cut, withb):
    eflag = fd.FK_FLAG_ENGINE_TENSOR if engine == "tensor" else fd.FK_FLAG_ENGINE_FP64
    rng = np.random.default_rng(300 + sum(cut))
    A, b = inputs.random_symmetric(2 * len(cut), rng, scale=0.15, with_b=withb)
    c = 0.7 - 0.2j
    gbar = rng.normal(size=cut) + 1j * rng.normal(size=cut)
    ref = oracle.full_dm_probs(A, b, c, cut)
    rA, rb, rc = oracle_vjp(A, b, c, cut, gbar)
    for flags in ((eflag,) if withb else (eflag, eflag | fd.FK_FLAG_B_ZERO)):
        need = fd.fk_workspace_size(len(cut), cut, 1, fd.FK_OP_DIAG_VJP, flags)
        ws = Guarded(need, 0xFF)
        out = Guarded(16 * int(np.prod(cut)), 0xFF)
        probs = out.view(torch.complex128, (1,) + cut)
        Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([c])
        fd.fock_diag_probs_batched(Ad, bd, cd, cut, probs=probs, flags=flags, ws=ws.inner)
        fd.check_workspace(ws.inner)
        assert_amp_close(probs[0].cpu().numpy(), ref)
        D = 2 * len(cut)
        gout = Guarded(16 * (D * D + D + 1), 0xFF)
        flat = gout.view(torch.complex128, (D * D + D + 1,))
        gA, gb, gc = flat[:D * D].view(1, D, D), flat[D * D:D * D + D].view(1, D), flat[D * D + D:]
        fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(gbar[None]), ws.inner, flags=flags,
                                       out=(gA, gb, gc))
        fd.check_workspace(ws.inner)
        assert_grad_close(gA[0].cpu().numpy(), rA)
        if withb:
            assert_grad_close(gb[0].cpu().numpy(), rb)
        assert abs(gc[0].item() - rc) <= VJP_RTOL * abs(rc)
        for g in (ws, out, gout):
            g.check()


def test_poisoned_workspace_conditional(fd):
    mask = (1, 1, 0)
    cut = (4, 3, 5)
    rng = np.random.default_rng(17)
    A, b = inputs.random_symmetric(6, rng, with_b=True)
    c = 0.6 + 0.1j
    ref = oracle.full_dm_conditional(A, b, c, cut, mask)
    need, offs = fd.fk_conditional_workspace_size([cut], mask, fd.FK_OP_COND_VJP)
    ws = Guarded(need, 0xFF)
    out = Guarded(16 * int(offs[-1]), 0xFF)
    rho = out.view(torch.complex128, (int(offs[-1]),))
    Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([c])
    fd.fock_conditional_dm_batched(Ad, bd, cd, [cut], mask, rho=rho, ws=ws.inner)
    fd.check_workspace(ws.inner)
    got = fd.conditional_blocks(rho, [cut], mask)[0].cpu().numpy()
    assert_amp_close(got, ref)
    gbar = rng.normal(size=ref.shape) + 1j * rng.normal(size=ref.shape)
    fd.fock_conditional_dm_vjp_batched(Ad, bd, cd, [cut], mask, cuda(gbar.reshape(-1)), ws.inner)
    fd.check_workspace(ws.inner)
    ws.check(); out.check()


@pytest.mark.parametrize("where", ["A", "b", "c"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_check_finite_flag(fd, where, bad):
    rng = np.random.default_rng(4)
    cut = (4, 3, 3)
    A, b = inputs.random_symmetric(6, rng, with_b=True)
    c = 0.8 + 0j
    Ab, bb, cb = A.copy(), b.copy(), c
    if where == "A":
        Ab[2, 3] = complex(bad, 0.0)
    elif where == "b":
        bb[4] = complex(0.0, bad)
    else:
        cb = complex(bad, 1.0)
    Ad, bd, cd = cuda(Ab[None]), cuda(bb[None]), cuda([cb])
    fl = fd.FK_FLAG_CHECK_FINITE
    # all-detected forward and VJP
    p, ws = fd.fock_diag_probs_batched(Ad, bd, cd, cut, flags=fl)
    assert fd.fk_workspace_status(ws) == fd.FK_ENONFINITE
    fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(np.ones((1,) + cut)), ws, flags=fl)
    assert fd.fk_workspace_status(ws) == fd.FK_ENONFINITE
    # conditional walk
    _, _, wsc = fd.fock_conditional_dm_batched(Ad, bd, cd, [cut], (1, 1, 0), flags=fl)
    assert fd.fk_workspace_status(wsc) == fd.FK_ENONFINITE
    # finite inputs on the same workspace: the context is usable and the flag passes
    good = (cuda(A[None]), cuda(b[None]), cuda([c]))
    p, ws = fd.fock_diag_probs_batched(*good, cut, flags=fl, ws=ws)
    assert fd.fk_workspace_status(ws) == fd.FK_OK
    assert_amp_close(p[0].cpu().numpy(), oracle.full_dm_probs(A, b, c, cut))


def test_check_finite_flag_pure_walk(fd):
    circ = inputs.make_circuit(2, np.random.default_rng(2), r_range=(0.2, 0.5), eta_range=(1.0, 1.0),
                               alpha_var=0.3, cutoffs=(5, 5))
    A, b, c = fd.fk_gaussian_to_pure_triple(circ.V, circ.mean)
    A = A.copy(); A[0, 1] = complex(float("nan"), 0.0)
    psi, ws = fd.fock_pure_amplitudes_batched(cuda(A[None]), cuda(b[None]), cuda([c]), (5, 5),
                                              flags=fd.FK_FLAG_CHECK_FINITE)
    assert fd.fk_workspace_status(ws) == fd.FK_ENONFINITE


def test_default_engine_is_tensor_up_to_twelve_modes(fd):
    """With nothing set, an 8-mode call runs the tensor engine (its VJP
    workspace is the tensor engine's, and its forward is bit-identical to a
    call that asks for the tensor engine); so do 9 and 12 modes."""
    fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    cut = (3, 2, 2, 2, 2, 2, 2, 3)
    ws_auto = fd.fk_workspace_size(8, cut, 2, fd.FK_OP_DIAG_VJP, 0)
    ws_tc = fd.fk_workspace_size(8, cut, 2, fd.FK_OP_DIAG_VJP, fd.FK_FLAG_ENGINE_TENSOR)
    ws_64 = fd.fk_workspace_size(8, cut, 2, fd.FK_OP_DIAG_VJP, fd.FK_FLAG_ENGINE_FP64)
    assert ws_auto == ws_tc != ws_64
    rng = np.random.default_rng(8)
    A, b = inputs.random_symmetric(16, rng, scale=0.12, with_b=False)
    Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([0.9])
    p0, _ = fd.fock_diag_probs_batched(Ad, bd, cd, cut, flags=fd.FK_FLAG_B_ZERO)
    p1, _ = fd.fock_diag_probs_batched(Ad, bd, cd, cut,
                                       flags=fd.FK_FLAG_B_ZERO | fd.FK_FLAG_ENGINE_TENSOR)
    p2, _ = fd.fock_diag_probs_batched(Ad, bd, cd, cut,
                                       flags=fd.FK_FLAG_B_ZERO | fd.FK_FLAG_ENGINE_FP64)
    assert torch.equal(p0, p1)
    ref = oracle.full_dm_probs(A, b, 0.9, cut)
    assert_amp_close(p2[0].cpu().numpy(), ref)
    assert_amp_close(p0[0].cpu().numpy(), ref)
    for m in (9, 12):
        cutm = (2,) * m
        ws_auto = fd.fk_workspace_size(m, cutm, 1, fd.FK_OP_DIAG_VJP, 0)
        assert ws_auto == fd.fk_workspace_size(m, cutm, 1, fd.FK_OP_DIAG_VJP, fd.FK_FLAG_ENGINE_TENSOR)
        assert ws_auto != fd.fk_workspace_size(m, cutm, 1, fd.FK_OP_DIAG_VJP, fd.FK_FLAG_ENGINE_FP64)


def test_per_call_tile_flags_override_process_default(fd):
    """A call that carries its own tile bits runs with them whatever the
    process default is, and a VJP sized with them needs them again."""
    rng = np.random.default_rng(12)
    cut = (5, 4, 4)
    A, b = inputs.random_symmetric(6, rng, with_b=True)
    ref = oracle.full_dm_probs(A, b, 0.8, cut)
    gbar = rng.normal(size=cut)
    rA, rb, rc = oracle_vjp(A, b, 0.8, cut, gbar)
    tile = fd.fk_diag_tuning_flags(fd.FK_ENGINE_FP64, 64, 4, 2)
    try:
        fd.fk_diag_set_tuning(256, 8, 0)          # a different process default
        fd.fk_diag_set_engine(fd.FK_ENGINE_TENSOR)
        Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([0.8])
        p, ws = fd.fock_diag_probs_batched(Ad, bd, cd, cut, flags=tile)
        assert_amp_close(p[0].cpu().numpy(), ref)
        gA, gb, gc = fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(gbar[None]), ws, flags=tile)
        fd.check_workspace(ws)
        assert_grad_close(gA[0].cpu().numpy(), rA)
        assert_grad_close(gb[0].cpu().numpy(), rb)
        with pytest.raises(fd.FockError) as e:   # sized for the per-call shape, run with the default
            fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(gbar[None]), ws, flags=0)
        assert e.value.status == 3
    finally:
        fd.fk_diag_set_tuning(0, 0, 0)
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
