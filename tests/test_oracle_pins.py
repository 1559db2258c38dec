"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check is a closed form,
an independent definition (loop hafnian), an exact count printed in App. B,
a brute-force restatement, or an exact identity.  Sizes are small enough for
the whole file to run in well under a minute on one core.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import gradients, hafnian, triple
from paper_2303_08879_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b, floor=1e-300):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), floor))


# ---------------------------------------------------------------------------
# Gaussian -> (A, b, c)  (Sec. 2.1 eqs. A_rho, b_rho; Sec. 2.2 vacuum amplitude)
# ---------------------------------------------------------------------------

def test_vacuum_triple():
    A, b, c = triple.gaussian_to_triple(np.eye(4) / 2, np.zeros(4))
    assert np.allclose(A, 0) and np.allclose(b, 0) and abs(c - 1) < 1e-15


def test_thermal_geometric_distribution():
    # thermal state, mean photon number nbar: p_n = nbar^n / (1+nbar)^(n+1)
    for nb in (0.1, 0.7, 2.5):
        A, b, c = triple.gaussian_to_triple(np.eye(2) * (nb + 0.5), np.zeros(2))
        assert abs(c - 1 / (1 + nb)) < 1e-15
        P = oracle.full_dm_probs(A, b, c, (14,))
        exact = np.array([nb ** n / (1 + nb) ** (n + 1) for n in range(14)])
        assert np.max(np.abs(P - exact)) < 1e-15
        assert np.max(np.abs(P.imag)) < 1e-17


def test_squeezed_vacuum_distribution():
    # p_{2n} = (2n)! / (4^n (n!)^2) tanh^{2n} r / cosh r, odd photon numbers vanish
    for r in (0.3, 0.9):
        V = np.diag([math.exp(-2 * r), math.exp(2 * r)]) / 2
        A, b, c = triple.gaussian_to_triple(V, np.zeros(2))
        assert abs(c - 1 / math.cosh(r)) < 1e-15
        P = oracle.full_dm_probs(A, b, c, (16,))
        for n in range(16):
            ex = (math.factorial(n) / (2 ** n * math.factorial(n // 2) ** 2)
                  * math.tanh(r) ** n / math.cosh(r)) if n % 2 == 0 else 0.0
            assert abs(P[n] - ex) < 1e-15


def test_pure_state_block_structure():
    # pure state: A_rho = A_psi* (+) A_psi (Sec. 2.1) -> no coupling between
    # row and column indices, and the two blocks are complex conjugates.
    rng = inputs.rng_for(99, 0)
    c = inputs.make_circuit(3, rng, r_range=(0.2, 1.0), eta_range=(1.0, 1.0), cutoffs=(2, 2, 2))
    A, b, _ = triple.gaussian_to_triple(c.V, c.mean)
    row = A[0::2, 0::2]; col = A[1::2, 1::2]
    assert np.max(np.abs(A[0::2, 1::2])) < 1e-14
    assert np.max(np.abs(row - col.conj())) < 1e-14
    assert np.max(np.abs(A - A.T)) < 1e-14


def test_coherent_state_matrix_and_pair_order():
    # <m|rho|n> = e^{-|a|^2} a^m conj(a)^n / sqrt(m! n!); lattice index 2j = m.
    al = 0.7 - 0.4j
    A, b, c = triple.gaussian_to_triple(np.eye(2) / 2, math.sqrt(2) * np.array([al.real, al.imag]))
    G = oracle.full_lattice(A, b, c, (8, 8))
    for m in range(8):
        for n in range(8):
            ex = math.exp(-abs(al) ** 2) * al ** m * np.conj(al) ** n / math.sqrt(
                math.factorial(m) * math.factorial(n))
            assert abs(G[m, n] - ex) < 1e-15
    assert abs(G[0, 1] - math.exp(-abs(al) ** 2) * np.conj(al)) < 1e-15


def test_product_state_factorises():
    # identity interferometer: p(n1, n2, n3) = prod_j p_j(n_j)
    rng = inputs.rng_for(98, 0)
    circ = inputs.make_circuit(3, rng, r_range=(0.2, 0.9), eta_range=(0.5, 1.0), alpha_var=0.5,
                               cutoffs=(5, 4, 6), identity_interferometer=True)
    A, b, c = triple.gaussian_to_triple(circ.V, circ.mean)
    P = oracle.full_dm_probs(A, b, c, circ.cutoffs)
    singles = []
    for j in range(3):
        idx = [j, 3 + j]
        Aj, bj, cj = triple.gaussian_to_triple(circ.V[np.ix_(idx, idx)], circ.mean[idx])
        singles.append(oracle.full_dm_probs(Aj, bj, cj, (circ.cutoffs[j],)))
    ex = np.einsum("i,j,k->ijk", *singles)
    assert rel(P, ex) < 1e-13


# ---------------------------------------------------------------------------
# O1 (full lattice) against the loop hafnian definition
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,seed", [((4, 4, 3, 3), 0), ((3, 2, 3, 2, 2, 3), 1), ((6, 5), 2)])
def test_full_lattice_vs_loop_hafnian(dims, seed):
    rng = np.random.default_rng(seed)
    D = len(dims)
    A, b = inputs.random_symmetric(D, rng)
    A = A + 0.05 * (rng.normal(size=(D, D)))      # non-symmetric input: only As matters
    c = 0.6 - 0.2j
    G = oracle.full_lattice(A, b, c, dims)
    for k in np.ndindex(*dims):
        if sum(k) > 9:
            continue
        h = hafnian.amplitude(A, b, c, k)
        assert abs(G[k] - h) <= 1e-13 * max(1.0, abs(h)), k


def test_b_zero_parity():
    # eq. (recrel_noB): with b = 0 every odd-weight amplitude vanishes exactly
    rng = np.random.default_rng(5)
    A, b = inputs.random_symmetric(4, rng, with_b=False)
    G = oracle.full_lattice(A, b, 0.8, (5, 5, 4, 4))
    for k in np.ndindex(*G.shape):
        if sum(k) % 2:
            assert G[k] == 0


# ---------------------------------------------------------------------------
# O2 (naive Algorithm 1 / 2) against O1 and against App. B
# ---------------------------------------------------------------------------

CASES_ALG1 = [((5, 4), True), ((3, 4, 3), True), ((4, 4, 4), False), ((2, 5, 1), True),
              ((1, 3), False), ((6,), True), ((3, 3, 2, 3), False), ((2, 2, 2, 2), True)]


@pytest.mark.parametrize("cut,withb", CASES_ALG1)
def test_alg1_matches_full_density_matrix(cut, withb):
    rng = np.random.default_rng(hash(cut) % 1000)
    D = 2 * len(cut)
    A, b = inputs.random_symmetric(D, rng, with_b=withb)
    c = 0.6 + 0.1j
    P1 = oracle.full_dm_probs(A, b, c, cut)
    P2 = oracle.Walk(A, b, c, cut).all_probs()
    assert rel(P2, P1) < 1e-13


def _appb():
    rows = []
    with open(os.path.join(GOLDEN, "appb_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _appb())
def test_alg1_counts_match_appendix_b(row):
    M, C, off1, off0, off2, o1010, o1001, piv = row
    rng = np.random.default_rng(M * 100 + C)
    A, b = inputs.random_symmetric(2 * M, rng)
    w = oracle.Walk(A, b, 0.5, (C,) * M)
    w.all_probs()
    s = w.stats()
    assert s["off1_ket"] + s["off1_bra"] == off1
    assert s["diag"] == off0
    assert s["off2"] == off2
    assert s["off1010"] == o1010 and s["off1001"] == o1001
    assert s["pivots"] == piv
    # "fully dense": every stored amplitude is one of the App. B.2 types
    assert s["stored"] == off1 + off0 + off2 + o1010 + o1001


CASES_ALG2 = [((4, 3), (0, 1)), ((3, 4, 3), (0, 1, 1)), ((3, 2, 3, 3), (0, 0, 1, 1)),
              ((3, 4, 3), (1, 0, 1)), ((5, 4, 2), (1, 1, 0))]


@pytest.mark.parametrize("cut,det", CASES_ALG2)
def test_alg2_matches_full_density_matrix(cut, det):
    rng = np.random.default_rng(sum(cut) * 7 + sum(det))
    D = 2 * len(cut)
    A, b = inputs.random_symmetric(D, rng)
    R1 = oracle.full_dm_conditional(A, b, 0.6, cut, det)
    w = oracle.Walk(A, b, 0.6, cut, det)
    R2 = w.all_conditional()
    assert rel(R2, R1) < 1e-12
    # Sec. 4 (complexity of Algorithm 2): the block walk stores prod_U C^2 x |Algorithm-1 closure over D|
    dcut = tuple(c for c, d in zip(cut, det) if d)
    ucut = tuple(c for c, d in zip(cut, det) if not d)
    A1, b1 = inputs.random_symmetric(2 * len(dcut), rng)
    w1 = oracle.Walk(A1, b1, 0.5, dcut)
    w1.all_probs()
    assert w.stats()["stored"] == int(np.prod([c * c for c in ucut])) * w1.stats()["stored"]


def test_conditional_physical_properties():
    # each conditional block is Hermitian and PSD; traces sum to <= 1
    circ = inputs.workload("cond_m3_batch64", 1)[0]
    cut = (6, 5, 9)
    A, b, c = triple.gaussian_to_triple(circ.V, circ.mean)
    R = oracle.Walk(A, b, c, cut, (1, 1, 0)).all_conditional()
    tot = 0.0
    for blk in R:
        assert np.max(np.abs(blk - blk.conj().T)) < 1e-14
        ev = np.linalg.eigvalsh(0.5 * (blk + blk.conj().T))
        assert ev.min() > -1e-13
        tot += np.trace(blk).real
    assert 0.5 < tot <= 1 + 1e-12


def test_probabilities_sum_and_monotone_in_cutoff():
    circ = inputs.workload("gbs_m2_c10", 1)[0]
    A, b, c = triple.gaussian_to_triple(circ.V, circ.mean)
    prev = 0.0
    for C in (2, 4, 6, 10, 16):
        P = oracle.Walk(A, b, c, (C, C)).all_probs()
        assert np.all(P.real > -1e-16)
        s = P.real.sum()
        assert prev - 1e-15 <= s <= 1 + 1e-12
        prev = s
    assert prev > 0.99


def test_marginal_against_reduced_state():
    # 0 <= p_j^red(n) - sum_{n_-j} P(n) <= 1 - sum P   (reduced single-mode state)
    circ = inputs.workload("gbs_m8_c6_batch16", 1)[0]
    cut = (4, 5, 3, 4)
    idx = [0, 1, 2, 3, 8, 9, 10, 11]
    V4 = circ.V[np.ix_(idx, idx)]
    A, b, c = triple.gaussian_to_triple(V4, np.zeros(8))
    P = oracle.Walk(A, b, c, cut).all_probs().real
    missing = 1 - P.sum()
    for j in range(4):
        Aj, bj, cj = triple.gaussian_to_triple(V4[np.ix_([j, 4 + j], [j, 4 + j])], np.zeros(2))
        pj = oracle.full_dm_probs(Aj, bj, cj, (cut[j],)).real
        marg = P.sum(axis=tuple(a for a in range(4) if a != j))
        d = pj - marg
        assert d.min() > -1e-14 and d.max() <= missing + 1e-14


# ---------------------------------------------------------------------------
# Gradients (Sec. 2.5)
# ---------------------------------------------------------------------------

def _rand_dir(D, rng):
    dA = rng.normal(size=(D, D)) + 1j * rng.normal(size=(D, D))
    db = rng.normal(size=D) + 1j * rng.normal(size=D)
    dc = rng.normal() + 1j * rng.normal()
    return dA, db, dc


def test_tangent_recurrence_matches_central_differences():
    rng = np.random.default_rng(11)
    dims = (4, 4, 3, 3)
    A, b = inputs.random_symmetric(4, rng)
    c = 0.7 + 0.1j
    dA, db, dc = _rand_dir(4, rng)
    G, Gd = oracle.full_lattice(A, b, c, dims, tangent=(dA, db, dc))
    h = 1e-6
    Gp = oracle.full_lattice(A + h * dA, b + h * db, c + h * dc, dims)
    Gm = oracle.full_lattice(A - h * dA, b - h * db, c - h * dc, dims)
    fd = (Gp - Gm) / (2 * h)
    assert np.max(np.abs(Gd - fd)) < 1e-8


def test_tangent_recurrence_matches_closed_form():
    # eqs. (recrel_dB), (recrel_dA) carried through the walk == derivatives of
    # the generating function (shift identities)
    rng = np.random.default_rng(12)
    dims = (5, 5, 4, 4)
    A, b = inputs.random_symmetric(4, rng)
    c = 0.9 - 0.3j
    dA, db, dc = _rand_dir(4, rng)
    G, Gd = oracle.full_lattice(A, b, c, dims, tangent=(dA, db, dc))
    assert np.max(np.abs(Gd - gradients.jvp(G, c, dA, db, dc))) < 1e-13


def test_walk_tangent_matches_full_lattice_tangent():
    rng = np.random.default_rng(13)
    for cut, det in [((4, 3, 3), None), ((3, 4, 3), (1, 1, 0))]:
        D = 2 * len(cut)
        A, b = inputs.random_symmetric(D, rng)
        dA, db, dc = _rand_dir(D, rng)
        G, Gd = oracle.full_lattice(A, b, 0.5, oracle.dm_dims(cut), tangent=(dA, db, dc))
        w = oracle.Walk(A, b, 0.5, cut, det, tangent=(dA, db, dc))
        for k in list(np.ndindex(*[c for c in cut]))[::3]:
            x = [v for a in k for v in (a, a)]
            g, t = w.amplitude(x)
            assert abs(g - G[tuple(x)]) < 1e-13 and abs(t - Gd[tuple(x)]) < 1e-12


def test_vjp_is_adjoint_of_jvp_and_homogeneous():
    rng = np.random.default_rng(14)
    dims = (4, 4, 3, 3)
    A, b = inputs.random_symmetric(4, rng)
    c = 0.7 + 0.2j
    G = oracle.full_lattice(A, b, c, dims)
    gbar = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    gA, gb, gc = gradients.vjp(G, gbar, c)
    assert np.max(np.abs(gA - gA.T)) < 1e-14
    # dot-product test: Re<gbar, J d> == Re<vjp, d>
    dA, db, dc = _rand_dir(4, rng)
    Jd = gradients.jvp(G, c, dA, db, dc)
    lhs = np.real(np.vdot(gbar, Jd))
    rhs = np.real(np.vdot(gA, dA) + np.vdot(gb, db) + np.conj(gc) * dc)
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))
    # Euler homogeneity: G_k(t^2 A, t b, c) = t^{|k|} G_k
    w = np.zeros(dims)
    for k in np.ndindex(*dims):
        w[k] = sum(k)
    lhs = np.sum(np.conj(gbar) * w * G)
    rhs = np.sum(2 * A * np.conj(gA)) + np.sum(b * np.conj(gb))
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))
    assert abs(c * np.conj(gc) - np.sum(np.conj(gbar) * G)) < 1e-13


def test_vjp_closed_form_matches_finite_differences():
    rng = np.random.default_rng(15)
    dims = (3, 3, 3, 3)
    A, b = inputs.random_symmetric(4, rng)
    c = 0.8
    G = oracle.full_lattice(A, b, c, dims)
    gbar = rng.normal(size=dims) + 1j * rng.normal(size=dims)
    gA, gb, gc = gradients.vjp(G, gbar, c)
    L = lambda A_, b_: np.real(np.vdot(gbar, oracle.full_lattice(A_, b_, c, dims)))
    h = 1e-6
    for (m, n) in [(0, 0), (0, 3), (2, 1)]:
        E = np.zeros((4, 4), complex); E[m, n] = h
        d_re = (L(A + E, b) - L(A - E, b)) / (2 * h)
        d_im = (L(A + 1j * E, b) - L(A - 1j * E, b)) / (2 * h)
        assert abs(complex(d_re, d_im) - gA[m, n]) < 1e-7
    for m in range(4):
        e = np.zeros(4, complex); e[m] = h
        d_re = (L(A, b + e) - L(A, b - e)) / (2 * h)
        d_im = (L(A, b + 1j * e) - L(A, b - 1j * e)) / (2 * h)
        assert abs(complex(d_re, d_im) - gb[m]) < 1e-7


# ------------------------------------------------------------- pure states
def test_pure_state_vector_squares_to_density_diagonal():
    # |psi_n|^2 from the M-mode recurrence on the pure triple equals the
    # diagonal of the density matrix from the 2M-mode recurrence (Sec. 2.2)
    rng = inputs.rng_for(98, 1)
    circ = inputs.make_circuit(3, rng, r_range=(0.2, 0.9), eta_range=(1.0, 1.0), alpha_var=0.4,
                               cutoffs=(4, 3, 4))
    Ap, bp, cp = triple.pure_triple(circ.V, circ.mean)
    psi = oracle.full_lattice(Ap, bp, cp, (4, 3, 4))
    A, b, c = triple.gaussian_to_triple(circ.V, circ.mean)
    P = oracle.full_dm_probs(A, b, c, (4, 3, 4))
    assert np.max(np.abs(np.abs(psi) ** 2 - P.real)) < 1e-14
    with pytest.raises(ValueError):
        lossy = inputs.make_circuit(2, rng, r_range=(0.5, 0.6), eta_range=(0.5, 0.6), cutoffs=(2, 2))
        triple.pure_triple(lossy.V, lossy.mean)


def test_pure_coherent_and_squeezed_closed_forms():
    # coherent: psi_n = e^{-|a|^2/2} a^n / sqrt(n!)
    al = 0.6 + 0.3j
    Ap, bp, cp = triple.pure_triple(np.eye(2) / 2, math.sqrt(2) * np.array([al.real, al.imag]))
    psi = oracle.full_lattice(Ap, bp, cp, (10,))
    for n in range(10):
        ex = math.exp(-abs(al) ** 2 / 2) * al ** n / math.sqrt(math.factorial(n))
        assert abs(psi[n] - ex) < 1e-15
    # x-squeezed vacuum: psi_2k = (-tanh r / 2)^k sqrt((2k)!) / (k! sqrt(cosh r)), odd = 0
    r = 0.7
    V = np.diag([math.exp(-2 * r), math.exp(2 * r)]) / 2
    Ap, bp, cp = triple.pure_triple(V, np.zeros(2))
    psi = oracle.full_lattice(Ap, bp, cp, (12,))
    for n in range(12):
        k = n // 2
        ex = ((-math.tanh(r) / 2) ** k * math.sqrt(math.factorial(n)) / math.factorial(k)
              / math.sqrt(math.cosh(r))) if n % 2 == 0 else 0.0
        assert abs(psi[n] - ex) < 1e-15
