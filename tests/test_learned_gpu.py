"""The learned proposal loop: herald scores against the oracle, exact
parameter gradients against finite differences, and what the trained
network gains over the same number of random starts."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import triple as otriple
from paper_2303_08879_gb300.inputs import propagate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prop():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import proposal
    return proposal


def circuit_state(theta, eta):
    """Gaussian state of the 15-parameter circuit, built independently."""
    M = 3
    r, x, ang = theta[:3], theta[3:6], theta[6:]
    U = np.eye(M, dtype=complex)
    bs = 0
    for i in range(M - 1):
        for k in range(M - 1 - i):
            t, ph = ang[2 * bs], ang[2 * bs + 1]
            T = np.eye(M, dtype=complex)
            T[k, k] = T[k + 1, k + 1] = np.cos(t)
            T[k, k + 1] = -np.exp(-1j * ph) * np.sin(t)
            T[k + 1, k] = np.exp(1j * ph) * np.sin(t)
            U = T @ U
            bs += 1
    U = np.diag(np.exp(1j * ang[2 * bs:])) @ U
    return propagate(M, r, x.astype(complex), U, np.full(M, eta))


def test_herald_scores_match_oracle(prop):
    task = prop.HeraldTask()
    ev = prop.Evaluator(task)
    rng = np.random.default_rng(0)
    theta = task.sample(3, rng)
    P, F, J = ev.scores(theta)
    for i in range(3):
        V, mean = circuit_state(theta[i], task.eta)
        A, b, c = otriple.gaussian_to_triple(V, mean)
        rho = oracle.Walk(A, b, c, task.cutoffs, task.mask).all_conditional()[task.pattern]
        Pr = np.trace(rho).real
        Fr = np.real(np.conj(task.target) @ rho @ task.target) / Pr
        assert abs(P[i] - Pr) <= 1e-10 * Pr
        assert abs(F[i] - Fr) <= 1e-9
        assert abs(J[i] - (Fr + task.lam * math.log(Pr))) <= 1e-9


def test_exact_parameter_gradient(prop):
    task = prop.HeraldTask()
    ev = prop.Evaluator(task)
    theta = task.sample(2, np.random.default_rng(1))
    _, _, J, G = ev.scores(theta, grad=True)
    h = 1e-5
    for p in range(15):
        e = np.zeros(15); e[p] = h
        Jp = ev.scores(theta + e)[2]
        Jm = ev.scores(theta - e)[2]
        fd = (Jp - Jm) / (2 * h)
        assert np.all(np.abs(fd - G[:, p]) <= 1e-6 * np.maximum(1.0, np.abs(fd))), (p, fd, G[:, p])


def test_trained_network_beats_random_starts(prop):
    task = prop.HeraldTask()
    ev = prop.Evaluator(task)
    _, X, Y = prop.make_dataset(task, ev, 16384, seed=5)
    mlp, losses = prop.train_mlp(X, Y, 1500, batch=1024, lr=2e-3, seed=5, log_every=100)
    assert losses[-1][1] < 0.5 * losses[0][1]
    k = 32
    th_mlp, _ = prop.propose(mlp, task, 1 << 16, k, seed=6)
    th_rnd = task.sample(k, np.random.Generator(np.random.PCG64(7)))
    J_mlp = ev.scores(th_mlp)[2]
    J_rnd = ev.scores(th_rnd)[2]
    # the network's picks, verified by the exact walk, beat random picks
    assert np.median(J_mlp) > np.median(J_rnd)
    assert J_mlp.max() > J_rnd.max()


def test_heralded_block_does_not_depend_on_detected_cutoffs(prop):
    """The learned workload's stated detected cutoffs are C = 15, 15 (with the
    undetected mode at C = 40); the proposal loop walks with C = n* + 1 =
    (4, 4).  An amplitude is a coefficient of the generating function
    c exp(z^T A z / 2 + b^T z) (Sec. 2.1), which no cutoff enters, and each is
    computed from the same parent and reads whatever the box, so the heralded
    block rho(n* = (3, 3)) and every pattern below (4, 4) agree between the
    two walks up to rounding order.  Checked on 8 random circuits of the
    15-parameter family in one batched launch each."""
    from paper_2303_08879_gb300 import fockdiag as fd
    task = prop.HeraldTask()
    theta = task.sample(8, np.random.default_rng(44))
    A, b, c = task.triples(theta)[:3]
    Ad = torch.as_tensor(A).cuda(); bd = torch.as_tensor(b).cuda(); cd = torch.as_tensor(c).cuda()
    blocks = {}
    for cut in ((4, 4, 40), (15, 15, 40)):
        rho, _, ws = fd.fock_conditional_dm_batched(Ad, bd, cd, [cut] * 8, task.mask, for_vjp=False)
        fd.check_workspace(ws)
        blocks[cut] = [x.cpu().numpy() for x in fd.conditional_blocks(rho, [cut] * 8, task.mask)]
    for i in range(8):
        small, big = blocks[(4, 4, 40)][i], blocks[(15, 15, 40)][i]
        for n0 in range(4):
            for n1 in range(4):
                s = small[n0 * 4 + n1]
                g = big[n0 * 15 + n1]
                scale = max(float(np.max(np.abs(s))), 1e-300)
                assert np.max(np.abs(s - g)) <= 1e-13 * scale, (i, n0, n1)
        # the heralded block itself, entry by entry
        s, g = small[3 * 4 + 3], big[3 * 15 + 3]
        big_entries = np.abs(s) > 1e-12 * np.max(np.abs(s))
        assert np.all(np.abs(s - g)[big_entries] <= 1e-12 * np.abs(s)[big_entries])
