"""GPU parity of the tensor-core product engine of the all-detected walk
(FK_ENGINE_TENSOR: exact base-256 digit products on the bf16 tensor cores)
against the CPU oracle, through the C ABI.

The engine must meet the same bar as the FP64 engine: amplitudes to 1e-10
relative where |G| > 1e-12 (1e-12 absolute below), gradients of a VJP that
follows a tensor-engine forward to 1e-8 relative.  Inputs with amplitudes
far from 1 check the per-pivot and per-row power-of-two scaling.
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
    fockdiag.fk_diag_set_engine(fockdiag.FK_ENGINE_TENSOR)
    yield fockdiag
    fockdiag.fk_diag_set_engine(fockdiag.FK_ENGINE_AUTO)


def cuda(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128).cuda()


def assert_amp_close(got, ref, rtol=RTOL, atol=ATOL):
    got = np.asarray(got); ref = np.asarray(ref)
    assert got.shape == ref.shape
    err = np.abs(got - ref)
    big = np.abs(ref) > atol
    if big.any():
        worst = np.max(err[big] / np.abs(ref[big]))
        assert worst <= rtol, f"max relative error {worst:.3e}"
    if (~big).any():
        assert np.max(err[~big]) <= atol, f"max absolute error {np.max(err[~big]):.3e}"


def assert_grad_close(got, ref, what):
    """Every entry within 1e-8 of itself where |ref| > 1e-12 max(1, max|ref|);
    the structural zeros below that floor within the floor."""
    got = np.asarray(got); ref = np.asarray(ref)
    floor = 1e-12 * max(1.0, float(np.max(np.abs(ref))))
    err = np.abs(got - ref)
    big = np.abs(ref) > floor
    if big.any():
        worst = np.max(err[big] / np.abs(ref[big]))
        assert worst <= VJP_RTOL, f"{what}: per-entry relative error {worst:.3e}"
    if (~big).any():
        assert np.max(err[~big]) <= floor, f"{what}: absolute error {np.max(err[~big]):.3e}"


def gpu_probs(fd, A, b, c, cut, flags=0):
    A = cuda(np.asarray(A)[None] if np.ndim(A) == 2 else A)
    b = cuda(np.asarray(b)[None] if np.ndim(b) == 1 else b)
    c = cuda(np.atleast_1d(c))
    p, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags)
    fd.check_workspace(ws)
    return p.cpu().numpy(), (A, b, c, ws)


CASES = [((5, 4), True), ((3, 4, 3), True), ((4, 4, 4), False), ((2, 5, 1), True),
         ((1, 3), False), ((6,), True), ((3, 3, 2, 3), False), ((2, 2, 2, 2), True),
         ((1, 1), True), ((7, 2, 5), True), ((4, 1, 3, 2), True), ((2,), False),
         ((3, 2, 3, 2, 2), True), ((2, 3, 2, 2, 3, 2), False), ((2, 2, 3, 2, 2, 2, 2), True),
         ((3, 2, 2, 2, 2, 2, 2, 3), False)]


@pytest.mark.parametrize("cut,withb", CASES)
def test_tensor_forward_matches_oracle(fd, cut, withb):
    """M = 1..8 (one and two 16-row K steps), b != 0 (DP tiles) and b = 0."""
    rng = np.random.default_rng(7 * sum(cut) + len(cut))
    A, b = inputs.random_symmetric(2 * len(cut), rng, scale=0.15, with_b=withb)
    c = 0.6 + 0.1j
    ref = oracle.Walk(A, b, c, cut).all_probs()
    got, _ = gpu_probs(fd, A, b, c, cut)
    assert_amp_close(got[0], ref)
    if not withb:
        got0, _ = gpu_probs(fd, A, b, c, cut, flags=fd.FK_FLAG_B_ZERO)
        assert_amp_close(got0[0], ref)


def test_tensor_many_tiles_ragged(fd):
    """Several 128-pivot tiles per level with ragged tails, b = 0 and b != 0."""
    rng = np.random.default_rng(3)
    for cut, withb in (((6, 6, 6, 6, 6), False), ((7, 5, 6, 4, 6), True)):
        A, b = inputs.random_symmetric(2 * len(cut), rng, scale=0.15, with_b=withb)
        ref = oracle.Walk(A, b, 0.7, cut).all_probs()
        got, _ = gpu_probs(fd, A, b, 0.7, cut)
        assert_amp_close(got[0], ref)


@pytest.mark.parametrize("cscale", [1e-200, 1e150])
def test_tensor_scaling_far_from_one(fd, cscale):
    """Amplitudes of order 1e-200 and 1e150 (c scales every amplitude) and a
    fast-decaying state: the power-of-two scales must follow the values."""
    rng = np.random.default_rng(21)
    cut = (5, 4, 5)
    A, b = inputs.random_symmetric(6, rng, scale=0.03, with_b=True)
    c = cscale * (0.9 - 0.2j)
    ref = oracle.Walk(A, b, c, cut).all_probs()
    got, _ = gpu_probs(fd, A, b, c, cut)
    assert_amp_close(got[0] / cscale, ref / cscale, atol=1e-12 * np.max(np.abs(ref / cscale)))


def test_tensor_large_entries(fd):
    """Strong squeezing (entries of A near 1): slow decay, large sums."""
    circ = inputs.make_circuit(3, np.random.default_rng(5), r_range=(1.2, 1.5), eta_range=(0.95, 1.0),
                               alpha_var=0.5, cutoffs=(8, 7, 6))
    A, b, c = otriple.gaussian_to_triple(circ.V, circ.mean)
    ref = oracle.Walk(A, b, c, circ.cutoffs).all_probs()
    got, _ = gpu_probs(fd, A, b, c, circ.cutoffs)
    assert_amp_close(got[0], ref)


def test_tensor_gbs_m8_c6_batch16_matches_fp64_engine(fd):
    """The benchmark workload at full size (16 circuits, M = 8, C = 6, b = 0):
    sampled outputs against the oracle one by one, and every output against
    the FP64 engine."""
    circs = inputs.workload("gbs_m8_c6_batch16")
    cut = circs[0].cutoffs
    trip = [fd.fk_gaussian_to_triple(c.V, c.mean) for c in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    got, _ = gpu_probs(fd, A, b, c, cut, flags=fd.FK_FLAG_B_ZERO)
    try:
        fd.fk_diag_set_engine(fd.FK_ENGINE_FP64)
        ref64, _ = gpu_probs(fd, A, b, c, cut, flags=fd.FK_FLAG_B_ZERO)
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_TENSOR)
    assert_amp_close(got, ref64)
    rng = np.random.default_rng(11)
    for ci in (0, 7, 15):
        Ao, bo, co = otriple.gaussian_to_triple(circs[ci].V, circs[ci].mean)
        w = oracle.Walk(Ao, bo, co, cut)
        pats = [tuple(rng.integers(0, 6, size=8)) for _ in range(30)]
        pats += [(0,) * 8, (5,) * 8, (5, 0, 0, 0, 0, 0, 0, 0), (0,) * 7 + (5,)]
        for n in pats:
            ref, _ = w.prob(n)
            assert_amp_close(got[ci][n], ref)


WIDE_CASES = [((2,) * 9, True), ((3, 2, 2, 2, 2, 2, 2, 2, 2), False), ((2, 2, 3, 2, 2, 2, 2, 2, 2, 2), True),
              ((2,) * 11, False), ((2,) * 12, True), ((2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 3), False)]


@pytest.mark.parametrize("cut,withb", WIDE_CASES)
def test_tensor_nine_to_twelve_modes_match_oracle(fd, cut, withb):
    """9 to 12 kept modes: three 16-row K steps (KS = 3), outputs from more
    than 16 rows of A per pivot."""
    rng = np.random.default_rng(5 * sum(cut) + len(cut))
    A, b = inputs.random_symmetric(2 * len(cut), rng, scale=0.1, with_b=withb)
    ref = oracle.Walk(A, b, 0.5, cut).all_probs()
    got, _ = gpu_probs(fd, A, b, 0.5, cut)
    assert_amp_close(got[0], ref)
    if not withb:
        got0, _ = gpu_probs(fd, A, b, 0.5, cut, flags=fd.FK_FLAG_B_ZERO)
        assert_amp_close(got0[0], ref)


def test_tensor_nine_modes_many_tiles_ragged(fd):
    """KS = 3 with several tiles per level and ragged tails."""
    rng = np.random.default_rng(19)
    cut = (4, 3, 3, 3, 2, 3, 2, 2, 3)
    A, b = inputs.random_symmetric(18, rng, scale=0.1, with_b=True)
    ref = oracle.Walk(A, b, 0.7, cut).all_probs()
    got, _ = gpu_probs(fd, A, b, 0.7, cut)
    assert_amp_close(got[0], ref)


def oracle_vjp(A, b, c, cut, gbar_probs):
    G = oracle.full_lattice(A, b, c, oracle.dm_dims(cut))
    gfull = np.zeros_like(G)
    for n in np.ndindex(*cut):
        gfull[tuple(v for a in n for v in (a, a))] = gbar_probs[n]
    return ograd.vjp(G, gfull, c)


VJP_CASES = [((4, 3), True), ((3, 3, 3), False), ((3, 4, 2), True), ((2, 1, 3), True),
             ((5,), True), ((2, 2, 2, 2), False), ((4, 4), False), ((2, 2, 2, 2), True),
             ((4, 4, 4, 3), True), ((3, 3, 3, 3), False),
             # five to eight kept modes: two 16-row K steps (the shape of the
             # 8-mode benchmark: reverse walk and partial pass with KS = 2)
             ((2, 3, 2, 2, 3), False), ((2, 3, 2, 2, 3), True), ((3, 2, 2, 2, 2, 3), True),
             ((3, 2, 2, 2, 2, 3), False), ((2, 2, 2, 2, 2, 2, 2), True),
             ((2, 2, 2, 2, 2, 2, 2, 3), False), ((2, 2, 2, 2, 2, 2, 2, 3), True),
             ((3, 3, 2, 2, 2, 2, 2, 2), False), ((2, 2, 1, 3, 2, 2, 2, 2, 2), False),
             # nine and ten kept modes: three K steps; the partial dL/dA of the
             # K = 0 family has 18 or 20 rows (two m16 tiles)
             ((2,) * 9, False), ((2,) * 9, True), ((3, 2, 2, 2, 2, 2, 2, 2, 2), True),
             ((2, 2, 2, 2, 2, 2, 2, 2, 2, 2), False), ((2, 3, 2, 2, 2, 2, 2, 2, 2, 2), True)]


@pytest.mark.parametrize("cut,withb", VJP_CASES)
def test_tensor_vjp_matches_oracle_gradient(fd, cut, withb):
    """Forward and VJP both on the tensor engine (b != 0: DP tiles and dL/db),
    every gradient entry against the oracle's closed-form VJP of the full
    density matrix (Sec. 2.5)."""
    rng = np.random.default_rng(100 + sum(cut) + 31 * len(cut))
    scale = 0.2 if len(cut) <= 4 else 0.12
    A, b = inputs.random_symmetric(2 * len(cut), rng, scale=scale, with_b=withb)
    c = 0.8 - 0.1j
    gbar = rng.normal(size=cut) + 1j * rng.normal(size=cut)
    rA, rb, rc = oracle_vjp(A, b, c, cut, gbar)
    for flags in ((0, fd.FK_FLAG_B_ZERO) if not withb else (0,)):
        _, (Ad, bd, cd, ws) = gpu_probs(fd, A, b, c, cut, flags)
        gA, gb, gc = fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(gbar[None]), ws, flags=flags)
        fd.check_workspace(ws)
        assert_grad_close(gA[0].cpu().numpy(), rA, "grad_A")
        if withb:
            assert_grad_close(gb[0].cpu().numpy(), rb, "grad_b")
        else:
            assert np.max(np.abs(gb[0].cpu().numpy())) < 1e-12 * max(1, np.max(np.abs(rA)))
        assert abs(gc[0].item() - rc) <= VJP_RTOL * max(abs(rc), 1e-300)


def test_tensor_vjp_scaled_adjoints(fd):
    """Upstream gradients spanning 1e-150..1e150 across outputs: the partial
    dL/dA rows take their power of two from the largest product."""
    rng = np.random.default_rng(8)
    cut = (4, 3, 4)
    A, b = inputs.random_symmetric(6, rng, with_b=True)
    c = 0.7 + 0.2j
    gbar = (rng.normal(size=cut) + 1j * rng.normal(size=cut)) * 10.0 ** rng.uniform(-150, 150, size=cut)
    rA, rb, rc = oracle_vjp(A, b, c, cut, gbar)
    _, (Ad, bd, cd, ws) = gpu_probs(fd, A, b, c, cut)
    gA, gb, gc = fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(gbar[None]), ws)
    fd.check_workspace(ws)
    assert_grad_close(gA[0].cpu().numpy(), rA, "grad_A")
    assert_grad_close(gb[0].cpu().numpy(), rb, "grad_b")


def test_tensor_vjp_gbs_m8_c6_batch16_matches_fp64_engine(fd):
    """Full-size benchmark workload: forward + VJP on the tensor engine against
    the FP64 engine for every circuit (1e-10 of each gradient's largest entry)."""
    circs = inputs.workload("gbs_m8_c6_batch16")
    cut = circs[0].cutoffs
    trip = [fd.fk_gaussian_to_triple(c.V, c.mean) for c in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    w = np.random.default_rng(1000).normal(size=(16,) + cut).astype(np.complex128)

    def run():
        _, (Ad, bd, cd, ws) = gpu_probs(fd, A, b, c, cut, flags=fd.FK_FLAG_B_ZERO)
        g = fd.fock_diag_probs_vjp_batched(Ad, bd, cd, cut, cuda(w), ws, flags=fd.FK_FLAG_B_ZERO)
        fd.check_workspace(ws)
        return [x.cpu().numpy() for x in g]

    gA, gb, gc = run()
    try:
        fd.fk_diag_set_engine(fd.FK_ENGINE_FP64)
        rA, rb, rc = run()
    finally:
        fd.fk_diag_set_engine(fd.FK_ENGINE_TENSOR)
    for i in range(16):
        scale = np.max(np.abs(rA[i]))
        assert np.max(np.abs(gA[i] - rA[i])) <= 1e-10 * scale, i
        assert np.allclose(gA[i], gA[i].T, rtol=0, atol=1e-14 * scale)
    assert np.max(np.abs(gc - rc)) <= 1e-10 * np.max(np.abs(rc))


def test_vjp_geometry_table_reused_or_rebuilt_alike(fd):
    """The reverse walk takes the pivot-geometry table its forward built when
    the workspace's control block holds the table's key (shape and address),
    and rebuilds it otherwise.  A copy of the workspace lives at another
    address, so its VJP rebuilds the table: both gradients must agree bit for
    bit, and with the oracle's closed-form VJP."""
    rng = np.random.default_rng(31)
    cut = (3, 2, 2, 2, 2, 3)
    A1, b1 = inputs.random_symmetric(2 * len(cut), rng, scale=0.12, with_b=False)
    A, b, c = cuda(A1[None]), cuda(b1[None]), cuda(np.array([0.7 - 0.2j]))
    w = rng.normal(size=(1,) + cut) + 1j * rng.normal(size=(1,) + cut)
    flags = fd.FK_FLAG_B_ZERO
    _, ws = fd.fock_diag_probs_batched(A, b, c, cut, flags=flags)
    ws2 = ws.clone()
    g_reuse = fd.fock_diag_probs_vjp_batched(A, b, c, cut, cuda(w), ws, flags=flags)
    g_build = fd.fock_diag_probs_vjp_batched(A, b, c, cut, cuda(w), ws2, flags=flags)
    for x, y in zip(g_reuse, g_build):
        assert torch.equal(x, y)
    G = oracle.full_lattice(A1, b1, 0.7 - 0.2j, oracle.dm_dims(cut))
    gfull = np.zeros_like(G)
    for n in np.ndindex(*cut):
        gfull[tuple(v for a in n for v in (a, a))] = w[0][n]
    rA, _, _ = ograd.vjp(G, gfull, 0.7 - 0.2j)
    got = g_reuse[0][0].cpu().numpy()
    big = np.abs(rA) > 1e-12 * max(1.0, float(np.max(np.abs(rA))))
    assert np.max(np.abs(got - rA)[big] / np.abs(rA[big])) <= VJP_RTOL
