"""Circuits with different cutoffs (and so different kept modes) in one launch
of the all-detected walk (Algorithm 1, Sec. 3.1.3), through the C ABI:
element by element against the CPU oracle (forward and VJP, both engines,
b = 0 and b != 0), against the one-shape launch of each circuit, and
replayed from a captured CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from oracle import gradients as ograd
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
    got = np.asarray(got); ref = np.asarray(ref)
    floor = 1e-12 * max(1.0, float(np.max(np.abs(ref))))
    err = np.abs(got - ref)
    big = np.abs(ref) > floor
    if big.any():
        worst = np.max(err[big] / np.abs(ref[big]))
        assert worst <= VJP_RTOL, f"{what}: per-entry relative error {worst:.3e}"
    if (~big).any():
        assert np.max(err[~big]) <= floor, f"{what}: absolute error {np.max(err[~big]):.3e}"


def oracle_vjp(A, b, c, cut, gbar):
    G = oracle.full_lattice(A, b, c, oracle.dm_dims(cut))
    gfull = np.zeros_like(G)
    for n in np.ndindex(*cut):
        gfull[tuple(v for a in n for v in (a, a))] = gbar[n]
    return ograd.vjp(G, gfull, c)


# four modes: circuits of different cutoffs, some sharing a shape, one with
# two modes cut at 1 (two kept modes, in other positions than the others),
# one vacuum-only circuit, one large enough for several tiles per level
MIXED = [(3, 4, 2, 3), (5, 3, 3, 2), (3, 4, 2, 3), (1, 4, 1, 5), (2, 2, 2, 2), (1, 1, 1, 1),
         (4, 1, 3, 3), (3, 4, 2, 3), (6, 6, 5, 6)]


def mixed_inputs(withb, seed):
    rng = np.random.default_rng(seed)
    A = np.zeros((len(MIXED), 8, 8), complex); b = np.zeros((len(MIXED), 8), complex)
    for i in range(len(MIXED)):
        A[i], b[i] = inputs.random_symmetric(8, rng, scale=0.12, with_b=withb)
    c = 0.5 + 0.3 * rng.random(len(MIXED)) + 0.1j
    return A, b, c


@pytest.mark.parametrize("engine", ["fp64", "tensor"])
@pytest.mark.parametrize("withb", [False, True])
def test_mixed_cutoffs_forward_and_vjp_match_oracle(fd, engine, withb):
    eng = fd.FK_FLAG_ENGINE_TENSOR if engine == "tensor" else fd.FK_FLAG_ENGINE_FP64
    A, b, c = mixed_inputs(withb, 11 + withb)
    rng = np.random.default_rng(5)
    for flags in ((eng,) if withb else (eng, eng | fd.FK_FLAG_B_ZERO)):
        p, offs, ws = fd.fock_diag_probs_multi_batched(cuda(A), cuda(b), cuda(c), MIXED, flags=flags)
        fd.check_workspace(ws)
        blocks = [x.cpu().numpy() for x in fd.multi_blocks(p, MIXED)]
        assert offs[-1] == sum(int(np.prod(cu)) for cu in MIXED)
        gbar = [rng.normal(size=cu) + 1j * rng.normal(size=cu) for cu in MIXED]
        flat = np.concatenate([g.reshape(-1) for g in gbar])
        gA, gb, gc = fd.fock_diag_probs_multi_vjp_batched(cuda(A), cuda(b), cuda(c), MIXED, cuda(flat), ws,
                                                         flags=flags)
        fd.check_workspace(ws)
        gA, gb, gc = gA.cpu().numpy(), gb.cpu().numpy(), gc.cpu().numpy()
        for i, cu in enumerate(MIXED):
            assert_amp_close(blocks[i], oracle.full_dm_probs(A[i], b[i], c[i], cu))
            if int(np.prod(cu)) > 2000:
                continue                       # the full-lattice VJP oracle is too large
            rA, rb, rc = oracle_vjp(A[i], b[i], c[i], cu, gbar[i])
            assert_grad_close(gA[i], rA, f"grad_A[{i}] {cu}")
            if withb:
                assert_grad_close(gb[i], rb, f"grad_b[{i}] {cu}")
            else:
                assert np.max(np.abs(gb[i])) <= 1e-12 * max(1.0, np.max(np.abs(rA)))
            assert abs(gc[i] - rc) <= VJP_RTOL * max(abs(rc), 1e-300)


@pytest.mark.parametrize("engine", ["fp64", "tensor"])
def test_mixed_launch_equals_one_shape_launches(fd, engine):
    """A GBS sweep: 24 six-mode circuits, each mode cut at 3..6 photons at
    random.  Every circuit's probabilities equal, bit for bit, those of the
    one-shape launch of that circuit alone (the same arithmetic per
    amplitude), and its gradients agree to 1e-10 of their largest entry (the
    partial sums are added over another number of slots)."""
    eng = fd.FK_FLAG_ENGINE_TENSOR if engine == "tensor" else fd.FK_FLAG_ENGINE_FP64
    rng = np.random.default_rng(21)
    cuts = [tuple(int(x) for x in rng.integers(3, 7, size=6)) for _ in range(24)]
    circs = [inputs.make_circuit(6, np.random.default_rng(100 + i), r_range=(0.3, 1.0),
                                 eta_range=(0.6, 1.0), cutoffs=cuts[i]) for i in range(24)]
    trip = [fd.fk_gaussian_to_triple(cc.V, cc.mean) for cc in circs]
    A = np.stack([t[0] for t in trip]); b = np.stack([t[1] for t in trip])
    c = np.array([t[2] for t in trip])
    flags = eng | fd.FK_FLAG_B_ZERO
    p, offs, ws = fd.fock_diag_probs_multi_batched(cuda(A), cuda(b), cuda(c), cuts, flags=flags)
    fd.check_workspace(ws)
    blocks = fd.multi_blocks(p, cuts)
    w = torch.randn(int(offs[-1]), dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(3)).to(torch.complex128)
    gA, gb, gc = fd.fock_diag_probs_multi_vjp_batched(cuda(A), cuda(b), cuda(c), cuts, w, ws, flags=flags)
    fd.check_workspace(ws)
    for i in range(24):
        sl = slice(i, i + 1)
        p1, ws1 = fd.fock_diag_probs_batched(cuda(A[sl]), cuda(b[sl]), cuda(c[sl]), cuts[i], flags=flags)
        assert torch.equal(blocks[i], p1[0]), i
        g1 = fd.fock_diag_probs_vjp_batched(cuda(A[sl]), cuda(b[sl]), cuda(c[sl]), cuts[i],
                                            w[offs[i]:offs[i + 1]].view(1, *cuts[i]), ws1, flags=flags)
        for x, y in zip((gA[i], gb[i], gc[i]), (g1[0][0], g1[1][0], g1[2][0])):
            scale = max(float(torch.max(torch.abs(y))), 1e-300)
            assert float(torch.max(torch.abs(x - y))) <= 1e-10 * scale, i
    # sampled outputs against the oracle walk
    for i in (0, 7, 23):
        wk = oracle.Walk(*trip[i], cuts[i])
        for _ in range(12):
            n = tuple(int(rng.integers(0, C)) for C in cuts[i])
            ref, _ = wk.prob(n)
            assert_amp_close(blocks[i][n].item(), ref)


def test_mixed_launch_graph_replay(fd):
    """Forward + VJP of a mixed batch captured in a CUDA graph: replays give
    the probabilities of a direct call bit for bit."""
    A, b, c = mixed_inputs(True, 4)
    Ad, bd, cd = cuda(A), cuda(b), cuda(c)
    p, offs, ws = fd.fock_diag_probs_multi_batched(Ad, bd, cd, MIXED)
    ref = p.clone()
    g = torch.ones_like(p)
    out = tuple(torch.empty_like(x) for x in (Ad, bd, cd))
    fd.fock_diag_probs_multi_vjp_batched(Ad, bd, cd, MIXED, g, ws, out=out)
    ref_g = [x.clone() for x in out]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            fd.fock_diag_probs_multi_batched(Ad, bd, cd, MIXED, probs=p, ws=ws, stream=s)
            fd.fock_diag_probs_multi_vjp_batched(Ad, bd, cd, MIXED, g, ws, stream=s, out=out)
    for _ in range(3):
        p.zero_()
        graph.replay()
        torch.cuda.synchronize()
        fd.check_workspace(ws)
        assert torch.equal(p, ref)
        for x, y in zip(out, ref_g):
            scale = max(float(torch.max(torch.abs(y))), 1e-300)
            assert float(torch.max(torch.abs(x - y))) <= 1e-12 * scale
