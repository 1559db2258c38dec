"""GPU parity of the global-cutoff walk (patterns with n_1 + ... + n_M < n_max,
outputs packed level-major) against the CPU oracle, both product engines.

The oracle runs the plain walk with per-mode cutoffs n_max; amplitudes do not
depend on the cutoffs (Sec. 4.2), so its patterns with fewer than n_max
photons are the reference.  Tolerances as for the per-mode walk.
"""
import itertools

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


def assert_amp_close(got, ref):
    err = np.abs(got - ref)
    big = np.abs(ref) > ATOL
    if big.any():
        assert np.max(err[big] / np.abs(ref[big])) <= RTOL
    if (~big).any():
        assert np.max(err[~big]) <= ATOL


def patterns(M, n):
    return sorted((p for p in itertools.product(range(n), repeat=M) if sum(p) < n),
                  key=lambda p: (sum(p), p))


def reference(A, b, c, M, n):
    full = oracle.Walk(A, b, c, (n,) * M).all_probs()
    return np.array([full[p] for p in patterns(M, n)])


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("M,n,withb", [(1, 9, True), (2, 7, False), (2, 6, True), (3, 6, True),
                                       (4, 5, False), (4, 6, True), (5, 4, True), (8, 3, False)])
def test_global_forward_matches_oracle(fd, engine, M, n, withb):
    try:
        fd.fk_diag_set_engine(engine)
        rng = np.random.default_rng(11 * M + n)
        A, b = inputs.random_symmetric(2 * M, rng, scale=0.2, with_b=withb)
        c = 0.55 + 0.05j
        ref = reference(A, b, c, M, n)
        p, ws = fd.fock_diag_probs_global_batched(cuda(A[None]), cuda(b[None]), cuda([c]), n)
        fd.check_workspace(ws)
        assert p.shape == (1, len(ref))
        assert_amp_close(p[0].cpu().numpy(), ref)
        if not withb:
            p0, ws = fd.fock_diag_probs_global_batched(cuda(A[None]), cuda(b[None]), cuda([c]), n,
                                                       flags=fd.FK_FLAG_B_ZERO)
            fd.check_workspace(ws)
            assert_amp_close(p0[0].cpu().numpy(), ref)
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)


def test_global_gbs_batch_matches_oracle(fd):
    """8 circuits of the 8-mode GBS workload with fewer than 6 photons (1287
    patterns each), tensor engine, against the per-mode oracle walk."""
    circs = inputs.workload("gbs_m8_c6_batch16", 8)
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    try:
        fd.fk_diag_set_engine(1)
        p, ws = fd.fock_diag_probs_global_batched(cuda(A), cuda(b), cuda(c), 6, flags=fd.FK_FLAG_B_ZERO)
        fd.check_workspace(ws)
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    got = p.cpu().numpy()
    pats = patterns(8, 6)
    rng = np.random.default_rng(5)
    for i in (0, 3, 7):
        Ao, bo, co = otriple.gaussian_to_triple(circs[i].V, circs[i].mean)
        w = oracle.Walk(Ao, bo, co, (6,) * 8)
        for k in list(rng.integers(0, len(pats), size=40)) + [0, len(pats) - 1]:
            ref, _ = w.prob(pats[k])
            assert_amp_close(np.array([got[i, k]]), np.array([ref]))
    # probabilities of fewer than 6 photons: real, nonnegative, sum below 1
    assert np.max(np.abs(got.imag)) < 1e-14
    assert np.all(got.real > -1e-15) and np.all(got.real.sum(axis=1) < 1 + 1e-12)


def oracle_vjp_global(A, b, c, M, n, gbar):
    G = oracle.full_lattice(A, b, c, oracle.dm_dims((n,) * M))
    gfull = np.zeros_like(G)
    for k, p in enumerate(patterns(M, n)):
        gfull[tuple(v for a in p for v in (a, a))] = gbar[k]
    return ograd.vjp(G, gfull, c)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("M,n,withb", [(2, 6, True), (3, 5, False), (3, 4, True)])
def test_global_vjp_matches_oracle(fd, engine, M, n, withb):
    try:
        fd.fk_diag_set_engine(engine)
        rng = np.random.default_rng(100 + 7 * M + n)
        A, b = inputs.random_symmetric(2 * M, rng, with_b=withb)
        c = 0.8 - 0.1j
        npat = fd.fk_global_size(M, n)
        gbar = rng.normal(size=npat) + 1j * rng.normal(size=npat)
        rA, rb, rc = oracle_vjp_global(A, b, c, M, n, gbar)
        Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([c])
        _, ws = fd.fock_diag_probs_global_batched(Ad, bd, cd, n)
        gA, gb, gc = fd.fock_diag_probs_global_vjp_batched(Ad, bd, cd, n, cuda(gbar[None]), ws)
        fd.check_workspace(ws)
        for got, ref, what in ((gA[0], rA, "A"), (gb[0], rb, "b")):
            got = got.cpu().numpy()
            scale = max(np.max(np.abs(ref)), 1e-300)
            assert np.max(np.abs(got - ref)) / scale <= VJP_RTOL, what
        assert abs(gc[0].item() - rc) <= VJP_RTOL * abs(rc)
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
