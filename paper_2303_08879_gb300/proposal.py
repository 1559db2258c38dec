"""Learned proposals for heralded non-Gaussian state preparation.

The paper optimises circuits with PNR detectors by gradient descent on the
Fock amplitudes (Sec. 2.5) and leaves the ansatz, cost and target open
(Sec. 1).  This module fixes them:

* circuit: 3 modes, squeezings r_j, real displacements x_j, a 3-beam-splitter
  triangle plus 3 output phases (9 angles), loss eta on every mode
  (``fk_circuit_triple``, 15 parameters);
* heralding: modes 0 and 1 detected with pattern n* = (3, 3); mode 2 keeps
  its density matrix, cutoff 40 (Algorithm 2).  The walk runs with detected
  cutoffs n* + 1: Sec. 4.2 notes that p(n) needs cutoffs n_i + 1 only, and
  the amplitudes do not depend on the cutoffs;
* target: the even cat |alpha> + |-alpha>, alpha = 2, truncated at 40;
* scores: P = Tr rho(n*), F = <cat|rho(n*)|cat>/P, objective J = F + lambda ln P.

A BF16 MLP (``mlp.MLP``) is trained on circuits the batched conditional
walk evaluates; it scores many random parameter vectors, the best are
verified by the exact walk and refined by exact gradients
(``fock_conditional_dm_vjp`` chained through the analytic Jacobian of the
circuit map).  The exact recurrence decides every reported number.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import fockdiag as fd
from .mlp import MLP, init_params


class HeraldTask:
    M = 3
    mask = (1, 1, 0)

    def __init__(self, n_star=(3, 3), cu=40, alpha=2.0, eta=0.95, lam=0.05):
        self.n_star = tuple(n_star)
        self.cu = int(cu)
        self.cutoffs = (n_star[0] + 1, n_star[1] + 1, cu)
        self.pattern = n_star[0] * (n_star[1] + 1) + n_star[1]
        self.alpha, self.eta, self.lam = float(alpha), float(eta), float(lam)
        k = np.arange(cu)
        logamp = k * math.log(alpha) - 0.5 * np.array([math.lgamma(v + 1) for v in k])
        t = np.exp(logamp) * (1 + (-1.0) ** k)
        self.target = (t / np.linalg.norm(t)).astype(np.complex128)
        two_pi = 2 * math.pi
        self.lo = np.array([0.0] * 3 + [-1.0] * 3 + [0.0, 0.0] * 3 + [0.0] * 3)
        self.hi = np.array([1.0] * 3 + [1.0] * 3 + [math.pi / 2, two_pi] * 3 + [two_pi] * 3)

    def sample(self, n, rng):
        return self.lo + (self.hi - self.lo) * rng.random((n, 15))

    def normalize(self, theta):
        return (2.0 * (theta - self.lo) / (self.hi - self.lo) - 1.0).astype(np.float32)

    def clip(self, theta):
        th = theta.copy()
        th[:, :6] = np.clip(th[:, :6], self.lo[:6], self.hi[:6])
        return th

    def triples(self, theta, jacobian=False):
        """Host (A, b, c[, dA, db, dc]) for every parameter row (C++ threads)."""
        return fd.fk_circuit_triple_batched(theta, self.eta, M=3, jacobian=jacobian)


class Evaluator:
    """Exact scores (and gradients) of parameter vectors on the GPU."""

    def __init__(self, task, max_batch=1024, device="cuda"):
        self.task = task
        self.max_batch = int(max_batch)
        self.device = torch.device(device)
        self.target = torch.as_tensor(task.target, device=self.device)
        self._ws = {}

    def _workspace(self, B):
        if B not in self._ws:
            need, offs = fd.fk_conditional_workspace_size([self.task.cutoffs] * B, self.task.mask)
            self._ws[B] = (fd.workspace(need, self.device), offs)
        return self._ws[B]

    def _chunk(self, theta, grad):
        t = self.task
        B = theta.shape[0]
        trip = t.triples(theta, jacobian=grad)
        A = torch.as_tensor(trip[0], device=self.device)
        b = torch.as_tensor(trip[1], device=self.device)
        c = torch.as_tensor(trip[2], device=self.device)
        ws, offs = self._workspace(B)
        cuts = [t.cutoffs] * B
        rho, _, _ = fd.fock_conditional_dm_batched(A, b, c, cuts, t.mask, ws=ws)
        nu2 = t.cu * t.cu
        boff = torch.as_tensor(offs[:-1] + t.pattern * nu2, dtype=torch.int64, device=self.device)
        P = torch.empty(B, dtype=torch.float64, device=self.device)
        F = torch.empty_like(P)
        g = torch.zeros_like(rho) if grad else None
        st = fd.lib().fk_herald_scores(B, fd._ptr(rho), fd._ptr(boff), t.cu, fd._ptr(self.target),
                                       t.lam, fd._ptr(P), fd._ptr(F), fd._ptr(g),
                                       fd._stream(None))
        fd._check(st, "fk_herald_scores")
        if not grad:
            fd.check_workspace(ws)
            return P.cpu().numpy(), F.cpu().numpy(), None
        gA, gb, gc = fd.fock_conditional_dm_vjp_batched(A, b, c, cuts, t.mask, g, ws)
        fd.check_workspace(ws)
        gA, gb, gc = gA.cpu().numpy(), gb.cpu().numpy(), gc.cpu().numpy()
        dA, db, dc = trip[3], trip[4], trip[5]
        # dJ/dtheta_p = Re( sum conj(gbar) dz_p )
        dth = (np.einsum("bij,bpij->bp", np.conj(gA), dA).real
               + np.einsum("bi,bpi->bp", np.conj(gb), db).real
               + (np.conj(gc)[:, None] * dc).real)
        return P.cpu().numpy(), F.cpu().numpy(), dth

    def scores(self, theta, grad=False):
        """(P, F, J[, dJ/dtheta]) for parameter rows theta [n, 15]."""
        Ps, Fs, Gs = [], [], []
        for s in range(0, theta.shape[0], self.max_batch):
            P, F, G = self._chunk(theta[s:s + self.max_batch], grad)
            Ps.append(P); Fs.append(F)
            if grad:
                Gs.append(G)
        P = np.concatenate(Ps); F = np.concatenate(Fs)
        J = F + self.task.lam * np.log(np.maximum(P, 1e-300))
        return (P, F, J, np.concatenate(Gs)) if grad else (P, F, J)


# ------------------------------------------------------------------ model
LOGP_SCALE = 10.0


def labels(P, F):
    return np.stack([np.log(np.maximum(P, 1e-300)) / LOGP_SCALE, F], axis=1).astype(np.float32)


def make_dataset(task, ev, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = task.sample(n, rng)
    P, F, _ = ev.scores(theta)
    return theta, task.normalize(theta), labels(P, F)


def train_mlp(X, Y, steps, batch=2048, lr=1e-3, seed=0, device="cuda", log_every=0):
    dev = torch.device(device)
    Xd = torch.as_tensor(X, device=dev)
    Yd = torch.as_tensor(Y, device=dev)
    mlp = MLP(init_params(seed), batch, dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, Xd.shape[0], (batch,), device=dev, generator=gen)
        lr_s = lr * 0.5 * (1 + math.cos(math.pi * s / steps))
        loss = mlp.train_step(Xd[idx].contiguous(), Yd[idx].contiguous(), lr=lr_s)
        if log_every and (s % log_every == 0 or s == steps - 1):
            losses.append((s, float(loss.item())))
    return mlp, losses


def predicted_objective(mlp, task, theta, chunk=None):
    X = torch.as_tensor(task.normalize(theta), device=mlp.device)
    out = []
    chunk = chunk or mlp.batch
    for s in range(0, X.shape[0], chunk):
        out.append(mlp.forward(X[s:s + chunk]))
    y = torch.cat(out).double().cpu().numpy()
    return y[:, 1] + task.lam * LOGP_SCALE * y[:, 0]


def propose(mlp, task, n_candidates, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = task.sample(n_candidates, rng)
    score = predicted_objective(mlp, task, theta)
    top = np.argsort(-score)[:k]
    return theta[top], score[top]


def refine(ev, theta, steps, lr=0.02, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam ascent of the exact objective J from every start (rows)."""
    th = theta.copy()
    m = np.zeros_like(th); v = np.zeros_like(th)
    hist = []
    for s in range(1, steps + 1):
        P, F, J, G = ev.scores(th, grad=True)
        hist.append(J.copy())
        m = beta1 * m + (1 - beta1) * G
        v = beta2 * v + (1 - beta2) * G * G
        th = th + lr * (m / (1 - beta1 ** s)) / (np.sqrt(v / (1 - beta2 ** s)) + eps)
        th = ev.task.clip(th)
    P, F, J = ev.scores(th)
    hist.append(J.copy())
    return th, np.array(hist), (P, F, J)


def compare(n_train=1 << 20, train_steps=6000, n_candidates=1 << 16, starts=32,
            refine_steps=40, targets=(0.3, 0.4, 0.45), seed=0, device="cuda", log=print):
    """MLP-proposed optimisation against plain exact optimisation from random
    starts: the same number of starts and exact-gradient steps, wall times
    measured; reports the best exact J after every step and the steps and
    seconds each method needs to reach each target J."""
    task = HeraldTask()
    ev = Evaluator(task, device=device)
    timings = {}
    t0 = time.perf_counter()
    _, X, Y = make_dataset(task, ev, n_train, seed)
    torch.cuda.synchronize()
    timings["dataset_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    mlp, losses = train_mlp(X, Y, train_steps, seed=seed, device=device, log_every=500)
    torch.cuda.synchronize()
    timings["train_s"] = time.perf_counter() - t0
    log(f"dataset {n_train} circuits in {timings['dataset_s']:.1f} s; "
        f"training {train_steps} steps in {timings['train_s']:.1f} s; loss {losses[0][1]:.4f} -> "
        f"{losses[-1][1]:.4f}")
    res = {"losses": losses}
    for name in ("mlp", "plain"):
        t0 = time.perf_counter()
        if name == "mlp":
            th0, _ = propose(mlp, task, n_candidates, starts, seed + 1)
        else:
            th0 = task.sample(starts, np.random.Generator(np.random.PCG64(seed + 2)))
        t_start = time.perf_counter() - t0
        th, hist, (P, F, J) = refine(ev, th0, refine_steps)
        wall = time.perf_counter() - t0
        per_step = (wall - t_start) / (refine_steps + 1)
        best_curve = np.maximum.accumulate(hist.max(axis=1))
        reach = {}
        for tg in targets:
            ok = np.nonzero(best_curve >= tg)[0]
            reach[str(tg)] = None if ok.size == 0 else {
                "steps": int(ok[0]), "seconds": t_start + per_step * (int(ok[0]) + 1)}
        i = int(np.argmax(J))
        res[name] = {"wall_s": wall, "start_s": t_start, "J_start_best": float(best_curve[0]),
                     "J_start_median": float(np.median(hist[0])), "J_best": float(best_curve[-1]),
                     "F_best": float(F[i]), "P_best": float(P[i]), "reach": reach,
                     "curve": best_curve.tolist()}
        log(f"{name}: start best J {best_curve[0]:.4f} (median {np.median(hist[0]):.4f}) -> "
            f"{best_curve[-1]:.4f} (F {F[i]:.4f}, P {P[i]:.3e}) in {wall:.2f} s; reach {reach}")
    res["timings"] = timings
    return res


if __name__ == "__main__":
    import json
    import sys
    n = int(sys.argv[1]) if len(sys.argv) > 1 else (1 << 20)
    out = compare(n_train=n, log=lambda m: print(m, file=sys.stderr))
    print(json.dumps(out))
