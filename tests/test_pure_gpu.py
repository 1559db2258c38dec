"""GPU parity of the state-vector walk (Sec. 2.2) and its VJP against the CPU
oracle (O1: eq. recrel over the whole box with the first-nonzero parent rule,
here on the M-mode lattice of a pure triple), through the C ABI.

Tolerances as for the density-matrix walk: 1e-10 relative where |psi| >
1e-12 (1e-12 absolute below), VJPs to 1e-8 of each gradient's largest entry.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import gradients as ograd
from oracle import triple as otriple
from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL, ATOL, VJP_RTOL = 1e-10, 1e-12, 1e-8


@pytest.fixture(scope="module")
def fd():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    return fockdiag


def cuda(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128).cuda()


def assert_close(got, ref):
    err = np.abs(got - ref)
    big = np.abs(ref) > ATOL
    if big.any():
        assert np.max(err[big] / np.abs(ref[big])) <= RTOL
    if (~big).any():
        assert np.max(err[~big]) <= ATOL


def generic(M, rng, withb, scale=0.25):
    X = (rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))) * scale
    A = X + X.T
    b = (rng.normal(size=M) + 1j * rng.normal(size=M)) * 0.3 if withb else np.zeros(M, complex)
    return A, b, 0.7 - 0.2j


CASES = [((12,), True), ((6, 5), True), ((5, 5), False), ((4, 3, 5), True), ((3, 4, 3, 2), False),
         ((1, 6), True), ((2, 2, 2, 2, 2, 2), True), ((4, 4, 4, 4, 4), False), ((3,) * 8, True)]


@pytest.mark.parametrize("cut,withb", CASES)
def test_pure_forward_matches_oracle(fd, cut, withb):
    rng = np.random.default_rng(5 * sum(cut) + len(cut))
    A, b, c = generic(len(cut), rng, withb)
    ref = oracle.full_lattice(A, b, c, cut)
    psi, ws = fd.fock_pure_amplitudes_batched(cuda(A[None]), cuda(b[None]), cuda([c]), cut)
    fd.check_workspace(ws)
    assert_close(psi[0].cpu().numpy(), ref)
    if not withb:
        psi0, ws = fd.fock_pure_amplitudes_batched(cuda(A[None]), cuda(b[None]), cuda([c]), cut,
                                                   flags=fd.FK_FLAG_B_ZERO)
        fd.check_workspace(ws)
        assert_close(psi0[0].cpu().numpy(), ref)


def test_pure_batch_of_physical_states(fd):
    """24 pure 4-mode states (squeezing, displacement, Haar interferometer, no
    loss): state vectors against the oracle, |psi|^2 against the density walk."""
    rng = np.random.default_rng(7)
    cut = (6, 5, 6, 5)
    circs = [inputs.make_circuit(4, rng, r_range=(0.1, 0.8), eta_range=(1.0, 1.0), alpha_var=0.3,
                                 cutoffs=cut) for _ in range(24)]
    trip = [fd.fk_gaussian_to_pure_triple(cc.V, cc.mean) for cc in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    psi, ws = fd.fock_pure_amplitudes_batched(cuda(A), cuda(b), cuda(c), cut)
    fd.check_workspace(ws)
    got = psi.cpu().numpy()
    for i in (0, 11, 23):
        Ao, bo, co = otriple.pure_triple(circs[i].V, circs[i].mean)
        assert_close(got[i], oracle.full_lattice(Ao, bo, co, cut))
    dm = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs[:4]]
    p, ws2 = fd.fock_diag_probs_batched(cuda(np.stack([t[0] for t in dm])), cuda(np.stack([t[1] for t in dm])),
                                        cuda(np.array([t[2] for t in dm])), cut)
    fd.check_workspace(ws2)
    assert np.max(np.abs(np.abs(got[:4]) ** 2 - p.cpu().numpy().real)) < 1e-13
    assert np.all((np.abs(got) ** 2).reshape(24, -1).sum(axis=1) <= 1 + 1e-12)


VJP_CASES = [((7,), True), ((5, 4), True), ((4, 4), False), ((3, 4, 3), True), ((3, 3, 3, 3), False),
             ((2, 3, 2, 3, 2), True)]


@pytest.mark.parametrize("cut,withb", VJP_CASES)
def test_pure_vjp_matches_oracle(fd, cut, withb):
    rng = np.random.default_rng(200 + sum(cut))
    A, b, c = generic(len(cut), rng, withb)
    G = oracle.full_lattice(A, b, c, cut)
    gbar = rng.normal(size=cut) + 1j * rng.normal(size=cut)
    rA, rb, rc = ograd.vjp(G, gbar, c)
    for flags in ((0, fd.FK_FLAG_B_ZERO) if not withb else (0,)):
        Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([c])
        _, ws = fd.fock_pure_amplitudes_batched(Ad, bd, cd, cut, flags=flags)
        gA, gb, gc = fd.fock_pure_amplitudes_vjp_batched(Ad, bd, cd, cut, cuda(gbar[None]), ws, flags=flags)
        fd.check_workspace(ws)
        for got, ref, what in ((gA[0], rA, "A"), (gb[0], rb, "b")):
            got = got.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= VJP_RTOL * np.max(np.abs(ref)), what
        assert abs(gc[0].item() - rc) <= VJP_RTOL * abs(rc)


def test_pure_vjp_recompute(fd):
    rng = np.random.default_rng(3)
    cut = (4, 5, 3)
    A, b, c = generic(3, rng, True)
    G = oracle.full_lattice(A, b, c, cut)
    gbar = rng.normal(size=cut) + 1j * rng.normal(size=cut)
    rA, rb, rc = ograd.vjp(G, gbar, c)
    gA, gb, gc = fd.fock_pure_amplitudes_vjp_batched(cuda(A[None]), cuda(b[None]), cuda([c]), cut,
                                                     cuda(gbar[None]), None)
    assert np.max(np.abs(gA[0].cpu().numpy() - rA)) <= VJP_RTOL * np.max(np.abs(rA))
    assert np.max(np.abs(gb[0].cpu().numpy() - rb)) <= VJP_RTOL * np.max(np.abs(rb))
