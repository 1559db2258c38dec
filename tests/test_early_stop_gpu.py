"""GPU parity of the probability-sum early stop (Sec. 2.3: after the pivots of
each photon number, stop once the probabilities computed so far sum to
>= 1 - eps) against the CPU oracle, both product engines.

The expected stop comes from the definition: with the oracle's probabilities
summed by total photon number n, the walk completes photon numbers 0..n* where
n* is the first n whose cumulative sum reaches 1 - eps.  Outputs above n* are
zero; the VJP is that of the stopped walk (gradients of the zero outputs do
not propagate).
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


def expected_levels(ref, eps):
    """Photon numbers completed: 0..n* with n* the first n whose cumulative
    probability is >= 1 - eps (all if none)."""
    tot = np.zeros(sum(ref.shape))
    for n in np.ndindex(*ref.shape):
        tot[sum(n)] += ref[n].real
    cum = np.cumsum(tot)
    L = sum(s - 1 for s in ref.shape)
    for n in range(L):
        if cum[n] >= 1 - eps:
            return n + 1
    return L + 1


def stopped(ref, levels):
    out = ref.copy()
    for n in np.ndindex(*ref.shape):
        if sum(n) >= levels:
            out[n] = 0
    return out


def circuit(M, cut, seed, r=(0.2, 0.6)):
    circ = inputs.make_circuit(M, np.random.default_rng(seed), r_range=r, eta_range=(0.7, 1.0),
                               cutoffs=cut)
    return otriple.gaussian_to_triple(circ.V, circ.mean)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("eps", [1e-2, 1e-4, 0.5, 0.0])
def test_stop_matches_definition(fd, engine, eps):
    cut = (6, 6, 6, 6)
    A, b, c = circuit(4, cut, 3)
    ref = oracle.Walk(A, b, c, cut).all_probs()
    lv = expected_levels(ref, eps)
    try:
        fd.fk_diag_set_engine(engine)
        p, levels, ws = fd.fock_diag_probs_stop_batched(cuda(A[None]), cuda(b[None]), cuda([c]), cut, eps)
        fd.check_workspace(ws)
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    assert int(levels[0]) == lv
    got = p[0].cpu().numpy()
    want = stopped(ref, lv)
    big = np.abs(want) > ATOL
    assert np.max(np.abs(got - want)[big] / np.abs(want[big])) <= RTOL
    if (~big).any():
        assert np.max(np.abs(got - want)[~big]) <= ATOL
    if eps == 0.0:
        assert lv == sum(s - 1 for s in cut) + 1


def test_stop_per_circuit_batch(fd):
    """Circuits of different brightness stop at different photon numbers in one launch."""
    cut = (5, 5, 5)
    trips = [circuit(3, cut, s, r=(0.1 + 0.2 * k, 0.2 + 0.25 * k)) for k, s in enumerate((1, 2, 3, 4))]
    A = np.stack([t[0] for t in trips]); b = np.stack([t[1] for t in trips])
    c = np.array([t[2] for t in trips])
    eps = 3e-3
    p, levels, ws = fd.fock_diag_probs_stop_batched(cuda(A), cuda(b), cuda(c), cut, eps)
    fd.check_workspace(ws)
    got = p.cpu().numpy()
    seen = set()
    for i in range(4):
        ref = oracle.Walk(A[i], b[i], c[i], cut).all_probs()
        lv = expected_levels(ref, eps)
        seen.add(lv)
        assert int(levels[i]) == lv
        want = stopped(ref, lv)
        assert np.max(np.abs(got[i] - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))
    assert len(seen) > 1


@pytest.mark.parametrize("engine", [0, 1])
def test_stop_vjp_matches_oracle(fd, engine):
    cut = (4, 4, 3)
    A, b, c = circuit(3, cut, 9, r=(0.3, 0.7))
    ref = oracle.Walk(A, b, c, cut).all_probs()
    eps = 0.1          # cumulative 0.657, 0.667, 0.895, 0.900, 0.948: stops after 4 photons
    lv = expected_levels(ref, eps)
    assert 1 < lv < sum(s - 1 for s in cut) + 1
    rng = np.random.default_rng(2)
    gbar = rng.normal(size=cut) + 1j * rng.normal(size=cut)
    gstop = stopped(gbar, lv)
    G = oracle.full_lattice(A, b, c, oracle.dm_dims(cut))
    gfull = np.zeros_like(G)
    for n in np.ndindex(*cut):
        gfull[tuple(v for a in n for v in (a, a))] = gstop[n]
    rA, rb, rc = ograd.vjp(G, gfull, c)
    try:
        fd.fk_diag_set_engine(engine)
        Ad, bd, cd = cuda(A[None]), cuda(b[None]), cuda([c])
        _, levels, ws = fd.fock_diag_probs_stop_batched(Ad, bd, cd, cut, eps)
        gA, gb, gc = fd.fock_diag_probs_stop_vjp_batched(Ad, bd, cd, cut, eps, cuda(gbar[None]), ws)
        fd.check_workspace(ws)
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_AUTO)
    assert int(levels[0]) == lv
    for got, want, what in ((gA[0], rA, "A"), (gb[0], rb, "b")):
        got = got.cpu().numpy()
        assert np.max(np.abs(got - want)) <= VJP_RTOL * np.max(np.abs(want)), what
    assert abs(gc[0].item() - rc) <= VJP_RTOL * abs(rc)
