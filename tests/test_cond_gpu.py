"""GPU parity of the conditional-state walk (Algorithm 2) and its VJP against
the CPU oracle, through the C ABI, on both product engines (the tensor-core
digits, the default, and FP64).  Tolerances as in test_diag_gpu.py."""
import numpy as np
import pytest
import torch

import oracle
from oracle import gradients as ograd
from oracle import triple as otriple
from paper_2303_08879_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL, ATOL, VJP_RTOL = 1e-10, 1e-12, 1e-8


FLAGS = 0   # product engine of the current module pass (set by the fd fixture)


@pytest.fixture(scope="module", params=["tensor", "fp64"])
def fd(request):
    global FLAGS
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    FLAGS = fockdiag.FK_FLAG_ENGINE_TENSOR if request.param == "tensor" else fockdiag.FK_FLAG_ENGINE_FP64
    yield fockdiag
    FLAGS = 0


def cuda(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128).cuda()


def assert_amp_close(got, ref):
    got = np.asarray(got); ref = np.asarray(ref)
    assert got.shape == ref.shape
    err = np.abs(got - ref)
    big = np.abs(ref) > ATOL
    if big.any():
        worst = np.max(err[big] / np.abs(ref[big]))
        assert worst <= RTOL, f"max relative error {worst:.3e}"
    if (~big).any():
        assert np.max(err[~big]) <= ATOL


def assert_grad_close(got, ref, what):
    scale = max(np.max(np.abs(ref)), 1e-300)
    err = np.max(np.abs(np.asarray(got) - ref)) / scale
    assert err <= VJP_RTOL, f"{what}: relative error {err:.3e}"


def gpu_cond(fd, A, b, c, cuts, mask):
    A = cuda(A); b = cuda(b); c = cuda(np.atleast_1d(c))
    rho, offs, ws = fd.fock_conditional_dm_batched(A, b, c, cuts, mask, flags=FLAGS)
    fd.check_workspace(ws)
    blocks = [x.cpu().numpy() for x in fd.conditional_blocks(rho, cuts, mask)]
    return blocks, (A, b, c, ws)


CASES = [((4, 3), (0, 1)), ((3, 4, 3), (0, 1, 1)), ((3, 2, 3, 3), (0, 0, 1, 1)),
         ((3, 4, 3), (1, 0, 1)), ((5, 4, 2), (1, 1, 0)), ((4, 1, 3), (1, 1, 0)),
         ((3, 3), (0, 0)), ((1, 4, 3), (0, 1, 1)), ((4, 3, 1), (1, 1, 0)), ((6, 5), (1, 0)),
         # the tensor engine's two and three 16-row K steps (2 (2M + 1) real rows)
         ((2, 3, 2, 2, 3), (1, 1, 0, 1, 0)), ((2, 2, 2, 2, 2, 2, 2, 3), (1, 1, 1, 1, 1, 1, 1, 0))]


@pytest.mark.parametrize("cut,mask", CASES)
@pytest.mark.parametrize("withb", [True, False])
def test_forward_matches_full_density_matrix(fd, cut, mask, withb):
    rng = np.random.default_rng(17 * sum(cut) + 3 * sum(mask) + withb)
    D = 2 * len(cut)
    A, b = inputs.random_symmetric(D, rng, with_b=withb)
    ref = oracle.full_dm_conditional(A, b, 0.6, cut, mask)
    got, _ = gpu_cond(fd, A[None], b[None], 0.6, [cut], mask)
    assert_amp_close(got[0], ref)


def test_heterogeneous_batch_many_tiles(fd):
    """Circuits with different cutoffs in one launch; u-blocks of several
    128-thread chunks with ragged tails."""
    mask = (1, 1, 0)
    cuts = [(5, 4, 13), (3, 6, 12), (4, 4, 11), (2, 3, 17)]
    circs = inputs.workload("cond_m3_batch64", len(cuts))
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    got, _ = gpu_cond(fd, A, b, c, cuts, mask)
    for i, cc in enumerate(circs):
        Ao, bo, co = otriple.gaussian_to_triple(cc.V, cc.mean)
        ref = oracle.Walk(Ao, bo, co, cuts[i], mask).all_conditional()
        assert_amp_close(got[i], ref)


def test_cond_m3_batch64_full_size(fd):
    """The 64-circuit conditional workload at full size in one launch: three
    circuits compared with the oracle block by block, every block checked for
    Hermiticity and the traces for sum <= 1."""
    mask = (1, 1, 0)
    circs = inputs.workload("cond_m3_batch64")
    cuts = [cc.cutoffs for cc in circs]
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    got, _ = gpu_cond(fd, A, b, c, cuts, mask)
    for i in range(64):
        blk = got[i]
        # each entry within 1e-10 relative (1e-12 absolute) of the exact
        # Hermitian block bounds the mismatch of an entry and its transpose
        herm = np.conj(np.swapaxes(blk, 1, 2))
        bound = RTOL * (np.abs(blk) + np.abs(herm)) + 2 * ATOL
        assert np.all(np.abs(blk - herm) <= bound)
        tr = np.einsum("pkk->p", blk).real
        assert tr.min() > -1e-14 and 0.3 < tr.sum() <= 1 + 1e-12
    rng = np.random.default_rng(4)
    for i in (0, 31, 63):
        Ao, bo, co = otriple.gaussian_to_triple(circs[i].V, circs[i].mean)
        w = oracle.Walk(Ao, bo, co, cuts[i], mask)
        C0, C1, CU = cuts[i]
        for _ in range(12):
            n0, n1 = int(rng.integers(0, C0)), int(rng.integers(0, C1))
            kk, bb = int(rng.integers(0, CU)), int(rng.integers(0, CU))
            ref, _ = w.amplitude([n0, n0, n1, n1, kk, bb])
            assert_amp_close(got[i][n0 * C1 + n1, kk, bb], ref)
        for (n0, n1) in ((0, 0), (C0 - 1, C1 - 1), (2, 3)):
            for kk in range(0, CU, 7):
                ref, _ = w.amplitude([n0, n0, n1, n1, kk, CU - 1 - kk])
                assert_amp_close(got[i][n0 * C1 + n1, kk, CU - 1 - kk], ref)


def oracle_cond_vjp(A, b, c, cut, mask, gbar):
    G = oracle.full_lattice(A, b, c, oracle.dm_dims(cut))
    M = len(cut)
    det = [j for j in range(M) if mask[j]]
    und = [j for j in range(M) if not mask[j]]
    gfull = np.zeros_like(G)
    for p, n in enumerate(np.ndindex(*[cut[j] for j in det])):
        for kk, ket in enumerate(np.ndindex(*[cut[j] for j in und])):
            for bb, bra in enumerate(np.ndindex(*[cut[j] for j in und])):
                x = [0] * (2 * M)
                for a, j in enumerate(det):
                    x[2 * j] = x[2 * j + 1] = n[a]
                for a, j in enumerate(und):
                    x[2 * j] = ket[a]
                    x[2 * j + 1] = bra[a]
                gfull[tuple(x)] = gbar[p, kk, bb]
    return ograd.vjp(G, gfull, c)


VJP_CASES = [((4, 3), (0, 1), True), ((3, 4, 3), (1, 1, 0), True), ((3, 4, 3), (1, 1, 0), False),
             ((3, 2, 3, 3), (0, 0, 1, 1), True), ((4, 1, 3), (1, 1, 0), True), ((3, 3), (0, 0), True),
             ((5, 4), (1, 0), False), ((2, 3, 2, 2, 3), (1, 1, 0, 1, 0), True),
             ((2, 2, 2, 2, 2, 2, 2, 3), (1, 1, 1, 1, 1, 1, 1, 0), True)]


@pytest.mark.parametrize("cut,mask,withb", VJP_CASES)
def test_vjp_matches_oracle_gradient(fd, cut, mask, withb):
    rng = np.random.default_rng(200 + sum(cut) + withb)
    D = 2 * len(cut)
    A, b = inputs.random_symmetric(D, rng, with_b=withb)
    c = 0.7 + 0.1j
    ref_rho = oracle.full_dm_conditional(A, b, c, cut, mask)
    gbar = rng.normal(size=ref_rho.shape) + 1j * rng.normal(size=ref_rho.shape)
    rA, rb, rc = oracle_cond_vjp(A, b, c, cut, mask, gbar)
    got, (Ad, bd, cd, ws) = gpu_cond(fd, A[None], b[None], c, [cut], mask)
    gA, gb, gc = fd.fock_conditional_dm_vjp_batched(Ad, bd, cd, [cut], mask,
                                                    cuda(gbar.reshape(-1)), ws, flags=FLAGS)
    fd.check_workspace(ws)
    assert_grad_close(gA[0].cpu().numpy(), rA, "grad_A")
    if withb:
        assert_grad_close(gb[0].cpu().numpy(), rb, "grad_b")
    assert abs(gc[0].item() - rc) <= VJP_RTOL * max(abs(rc), 1e-300)
    # recompute path
    gA2, gb2, gc2 = fd.fock_conditional_dm_vjp_batched(Ad, bd, cd, [cut], mask,
                                                       cuda(gbar.reshape(-1)), None, flags=FLAGS)
    assert_grad_close(gA2[0].cpu().numpy(), rA, "grad_A (recompute)")


# Large undetected blocks: step 1 keeps its u-block in the block's shared
# staging area only when the values and levels fit (17 bytes a point).  With
# U2 = 34^2 the forward reads F directly and the VJP stages; with U2 = 50^2
# both read global memory (for either engine's buffer sizes).
LARGE_U_CASES = [((3, 34), (1, 0)), ((2, 50), (1, 0))]


@pytest.mark.parametrize("cut,mask", LARGE_U_CASES)
def test_large_undetected_block_forward_and_vjp(fd, cut, mask):
    rng = np.random.default_rng(300 + sum(cut))
    A, b = inputs.random_symmetric(2 * len(cut), rng, scale=0.12, with_b=True)
    c = 0.5 - 0.2j
    ref_rho = oracle.full_dm_conditional(A, b, c, cut, mask)
    got, (Ad, bd, cd, ws) = gpu_cond(fd, A[None], b[None], c, [cut], mask)
    assert_amp_close(got[0], ref_rho)
    gbar = rng.normal(size=ref_rho.shape) + 1j * rng.normal(size=ref_rho.shape)
    rA, rb, rc = oracle_cond_vjp(A, b, c, cut, mask, gbar)
    gA, gb, gc = fd.fock_conditional_dm_vjp_batched(Ad, bd, cd, [cut], mask,
                                                    cuda(gbar.reshape(-1)), ws, flags=FLAGS)
    fd.check_workspace(ws)
    assert_grad_close(gA[0].cpu().numpy(), rA, "grad_A")
    assert_grad_close(gb[0].cpu().numpy(), rb, "grad_b")
    assert abs(gc[0].item() - rc) <= VJP_RTOL * max(abs(rc), 1e-300)


def test_vjp_batch_adjoint_and_homogeneity(fd):
    """Heterogeneous batch: every circuit's VJP satisfies the Euler identity
    sum conj(gbar)|k| G = sum 2 A conj(gA) + sum b conj(gb); one circuit is
    checked against the oracle's forward-mode tangent (dot-product test)."""
    mask = (1, 1, 0)
    cuts = [(6, 5, 9), (4, 7, 8), (5, 5, 10)]
    circs = inputs.workload("cond_m3_batch64", 3)
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    got, (Ad, bd, cd, ws) = gpu_cond(fd, A, b, c, cuts, mask)
    rng = np.random.default_rng(9)
    gbars = [rng.normal(size=g.shape) + 1j * rng.normal(size=g.shape) for g in got]
    flat = np.concatenate([g.reshape(-1) for g in gbars])
    gA, gb, gc = fd.fock_conditional_dm_vjp_batched(Ad, bd, cd, cuts, mask, cuda(flat), ws, flags=FLAGS)
    fd.check_workspace(ws)
    gA = gA.cpu().numpy(); gb = gb.cpu().numpy(); gc = gc.cpu().numpy()
    for i in range(3):
        C0, C1, CU = cuts[i]
        wgt = np.zeros(got[i].shape)
        for p in range(C0 * C1):
            n0, n1 = divmod(p, C1)
            wgt[p] = 2 * (n0 + n1) + np.add.outer(np.arange(CU), np.arange(CU))
        lhs = np.sum(np.conj(gbars[i]) * wgt * got[i])
        rhs = np.sum(2 * A[i] * np.conj(gA[i])) + np.sum(b[i] * np.conj(gb[i]))
        assert abs(lhs - rhs) <= 1e-9 * np.sum(np.abs(gbars[i] * wgt * got[i]))
        assert abs(c[i] * np.conj(gc[i]) - np.sum(np.conj(gbars[i]) * got[i])) <= \
            1e-10 * np.sum(np.abs(gbars[i] * got[i]))
    i = 1
    Ao, bo, co = otriple.gaussian_to_triple(circs[i].V, circs[i].mean)
    dA = rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))
    db = rng.normal(size=6) + 1j * rng.normal(size=6)
    dc = rng.normal() + 1j * rng.normal()
    _, tan = oracle.Walk(Ao, bo, co, cuts[i], mask, tangent=(dA, db, dc)).all_conditional(True)
    lhs = np.real(np.vdot(gbars[i], tan))
    rhs = np.real(np.vdot(gA[i], dA) + np.vdot(gb[i], db) + np.conj(gc[i]) * dc)
    assert abs(lhs - rhs) <= 1e-8 * max(abs(lhs), 1e-12)
