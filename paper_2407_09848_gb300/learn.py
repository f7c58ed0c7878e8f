"""Learned smoother weights: level features, the weight-predicting MLP and its
training loop (no counterpart in the paper; the optimal 4th-kind weights of
Eq. polsmootheropt are both the starting point and the fallback).

The MLP's forward, backward and Adam step are library kernels
(amgps_mlp_*); the loss -- the mean A-norm error reduction of one V-cycle over
random error vectors -- and its gradient in every level's weights come from
amgps_vcycle_loss_grad.  This module only moves the few numbers in between.

CLI:  python -m paper_2407_09848_gb300.learn --problems 512 --grid 64 --steps 200
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import amgps
from . import problems as pr

DEGREE = 4
NPARAM = 4996


def p_weights(beta, x):
    """p(x) = sum_j (beta_j - beta_{j+1})/(2j+1) W_j(1-2x), beta_0 = 1,
    beta_{k+1} = 0, with W by the 4th-kind recurrence (Eq. polsmootheropt)."""
    t = 1.0 - 2.0 * x
    b = np.concatenate([[1.0], np.asarray(beta, dtype=np.float64), [0.0]])
    w_prev, w = np.ones_like(t), 2.0 * t + 1.0
    p = (b[0] - b[1]) * w_prev + (b[1] - b[2]) / 3.0 * w
    for j in range(2, len(beta) + 1):
        w_prev, w = w, 2.0 * t * w - w_prev
        p = p + (b[j] - b[j + 1]) / (2 * j + 1) * w
    return p


_GRID = np.linspace(1e-4, 1.0, 4001)


def is_safe(beta):
    """The polynomial must stay in Pi_k (|p| < 1 on (0, 1]) for the V-cycle
    bound of Proposition 1 to hold."""
    return bool(np.all(np.abs(p_weights(beta, _GRID)) < 1.0))


SAFE_BACKOFF = 0.95


def make_safe(beta, ref):
    """(weights, t): the prediction itself (t = 1) when its polynomial stays in
    Pi_k, else the point beta_ref + t (beta - beta_ref) of the segment towards
    the optimal weights, t = 0.95 t_max with t_max the largest t (bisection)
    whose polynomial stays in Pi_k on the check grid (t = 0, the optimal
    weights, is inside by Proposition 1's bound)."""
    beta = np.asarray(beta, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if is_safe(beta):
        return beta, 1.0
    lo, hi = 0.0, 1.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if is_safe(ref + mid * (beta - ref)):
            lo = mid
        else:
            hi = mid
    t = SAFE_BACKOFF * lo
    return ref + t * (beta - ref), t


def level_features(solver, H, degree=DEGREE):
    """8 features per non-coarsest level: degree, level size, mean stored
    entries per row, the l1-Jacobi spectral estimate (10 power steps on the
    GPU), and coefficient statistics of the level matrix (contrast of the
    diagonal, diagonal share of the l1 row sum, spread of the log-diagonal,
    strongest-coupling share of the off-diagonal row sum).  No feature counts
    levels: a level of a large grid then looks like the level of a smaller
    training grid that has its size and coefficients."""
    import scipy.sparse as sp
    import torch
    rows = []
    for l, lv in enumerate(H.levels[:-1]):
        A = sp.csr_matrix(lv.A)
        n = A.shape[0]
        d = A.diagonal()
        absA = abs(A).tocsr()
        M = np.asarray(absA.sum(axis=1)).ravel()
        offsum = M - np.abs(d)
        offmax = np.asarray((absA - sp.diags(np.abs(d))).max(axis=1).todense()).ravel()
        v0 = torch.from_numpy(pr.vec_uniform(n, seed=0)).cuda()
        lam = solver.estimate_lambda(l, v0, iters=10)
        rows.append([degree / 8.0, np.log2(n) / 24.0, A.nnz / n / 8.0, lam,
                     np.log10(d.max() / d.min()) / 4.0, float(np.mean(d / M)),
                     float(np.std(np.log(d))) / 2.0,
                     float(np.mean(offmax / np.maximum(offsum, 1e-300)))])
    return np.asarray(rows, dtype=np.float64)


class WeightMLP:
    """Parameters, Adam moments and step counter of the MLP, on the GPU."""

    def __init__(self, seed=0, device="cuda"):
        import torch
        g = np.random.default_rng(seed)
        th = np.zeros(NPARAM, dtype=np.float32)
        th[0:512] = g.standard_normal(512) * np.sqrt(2.0 / 8)            # W1
        th[576:576 + 4096] = g.standard_normal(4096) * np.sqrt(2.0 / 64)  # W2
        # W3 = b3 = 0: the untrained network returns the optimal weights
        self.params = torch.from_numpy(th).to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.step_count = 0
        self.beta_ref = torch.from_numpy(amgps.opt4_weights(DEGREE).astype(np.float32)).to(device)

    def forward(self, feats):
        import torch
        F = torch.from_numpy(np.ascontiguousarray(feats, dtype=np.float32)).cuda()
        B = F.shape[0]
        beta = torch.empty(B * 4, dtype=torch.float32, device="cuda")
        acts = torch.empty(B * 132, dtype=torch.float32, device="cuda")
        amgps.mlp_forward(self.params, F, self.beta_ref, beta, acts)
        return F, beta, acts

    def predict(self, feats):
        _, beta, _ = self.forward(feats)
        return beta.view(-1, 4).double().cpu().numpy()

    def backward_and_step(self, F, beta, acts, gbeta, lr):
        import torch
        B = F.shape[0]
        gb = torch.from_numpy(np.ascontiguousarray(gbeta, dtype=np.float32).ravel()).cuda()
        work = torch.empty(B * 132, dtype=torch.float32, device="cuda")
        amgps.mlp_backward(self.params, F, acts, beta, gb, work, self.grads)
        self.step_count += 1
        amgps.mlp_adam(self.params, self.grads, self.m, self.v, self.step_count, lr)

    def state(self):
        return {"params": self.params.cpu().numpy(), "m": self.m.cpu().numpy(),
                "v": self.v.cpu().numpy(), "step": np.array(self.step_count)}

    def save(self, path):
        np.savez(path, **self.state())

    def load(self, path):
        import torch
        z = np.load(path)
        self.params = torch.from_numpy(z["params"]).cuda()
        self.m = torch.from_numpy(z["m"]).cuda()
        self.v = torch.from_numpy(z["v"]).cuda()
        self.step_count = int(z["step"])
        return self


PRE_CYCLES = 6


class Problem:
    """One training problem: hierarchy, library context, features and the
    seeded error vectors of its loss.

    The loss is the one-cycle A-norm error reduction of vectors that first ran
    through `pre_cycles` V-cycles with the weights being evaluated: those
    vectors concentrate on the slowest modes of E = I - B A, so the loss
    estimates the squared convergence factor rho(E)^2 -- the quantity that
    decides PCG iterations -- and, E being A-self-adjoint, the one-cycle
    gradient with the pre-cycled vectors held fixed is its gradient.  With
    pre_cycles = 0 it is the plain mean reduction of random vectors."""

    def __init__(self, H, nvec=32, seed=0, solver=None, pre_cycles=PRE_CYCLES):
        import torch
        from .amgps import Solver
        self.H = H
        self.S = solver or Solver().load(H.A, H.P)
        self.feats = level_features(self.S, H)
        n = H.levels[0].A.shape[0]
        self.E0 = torch.from_numpy(pr.vec_normal(n, seed=seed, count=nvec)).cuda()
        self.pre_cycles = pre_cycles

    def set_weights(self, betas):
        """Installs make_safe of each level's prediction; returns the t's."""
        ts = []
        ref = amgps.opt4_weights(DEGREE)
        for l, b in enumerate(betas):
            w, t = make_safe(b, ref)
            self.S.set_smoother(l, "weights", DEGREE, weights=w)
            ts.append(t)
        return ts

    def loss_grad(self, betas):
        ts = self.set_weights(betas)
        E = self.E0.clone()
        if self.pre_cycles:
            self.S.error_cycles(E, self.pre_cycles)
        loss, gw = self.S.loss_grad(E)
        # the installed weights are ref + t (beta - ref): d/dbeta = t, with t
        # held at its value (t = 0: the level does not depend on the network)
        g = gw[:, :DEGREE] * np.asarray(ts)[:, None]
        return loss, g


def convergence_estimate(solver, weights, E0, cycles=PRE_CYCLES):
    """Squared-convergence-factor estimate of the V-cycle with `weights` per
    level (degree 4): the one-cycle A-norm error reduction of the vectors E0
    (m x n_0, on the GPU, left unchanged) after `cycles` V-cycles."""
    for l, w in enumerate(weights):
        solver.set_smoother(l, "weights", DEGREE, weights=w)
    E = E0.clone()
    if cycles:
        solver.error_cycles(E, cycles)
    return solver.loss_grad(E)[0]


JUDGE_ITERS = 12


def pcg_factor(solver, weights, b, iters=JUDGE_ITERS):
    """Mean residual reduction per iteration of `iters` PCG iterations
    (||r_m|| / ||b||)^(1/m) on the FP64 hierarchy with `weights` per level."""
    import torch
    for l, w in enumerate(weights):
        solver.set_smoother(l, "weights", DEGREE, weights=w)
    x = torch.empty_like(b)
    it, rel = solver.pcg(b, x, rtol=1e-300, maxit=iters, raise_on_noconv=False)
    return rel ** (1.0 / max(it, 1))


def judge(solver, betas, seed=7, iters=JUDGE_ITERS):
    """The optimal 4th-kind weights as judge of the network (set-up, FP64
    hierarchy): the predicted weights (made safe level by level) are kept only
    when PCG preconditioned by their V-cycle reduces the residual of a seeded
    U[-1,1] right-hand side faster, over the same `iters` iterations, than
    with the optimal weights.  PCG convergence follows the spread of the
    preconditioned spectrum, which the one-cycle error reduction (the
    training loss) does not measure: a smoother that over-corrects some modes
    can have the larger error-propagation norm and still give PCG the smaller
    condition number.  Returns (weights per level, learned factor, optimal
    factor, learned kept)."""
    import torch
    ref = amgps.opt4_weights(DEGREE)
    learned = [make_safe(b, ref)[0] for b in betas]
    n = solver.level_info(0)[0]
    b = torch.from_numpy(pr.vec_uniform(n, seed=seed)).cuda()
    f_l = pcg_factor(solver, learned, b, iters)
    f_o = pcg_factor(solver, [ref] * len(betas), b, iters)
    keep = f_l < f_o
    return (learned if keep else [ref] * len(betas)), f_l, f_o, keep


def make_training_set(count, grid, seed0=0, nvec=32):
    """Log-normal coefficient problems: sigma ~ U[0.5, 2], ell ~ U[2, 16]."""
    rng = np.random.default_rng(12345 + seed0)
    out = []
    for i in range(count):
        sigma = rng.uniform(0.5, 2.0)
        ell = rng.uniform(2.0, 16.0)
        H = pr.build_hierarchy(pr.varcoef(grid, sigma, ell, seed=seed0 + i), coarse_max=512)
        out.append(Problem(H, nvec=nvec, seed=seed0 + i))
    return out


def evaluate(mlp, probs):
    """Mean loss with the network's weights and with the optimal weights."""
    learned, ref = [], []
    rb = amgps.opt4_weights(DEGREE)
    for p in probs:
        betas = mlp.predict(p.feats)
        learned.append(p.loss_grad(betas)[0])
        ref.append(p.loss_grad([rb] * len(betas))[0])
    return float(np.mean(learned)), float(np.mean(ref))


def train(mlp, probs, steps, batch=16, lr=1e-3, seed=0, log=None):
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(steps):
        idx = rng.choice(len(probs), size=min(batch, len(probs)), replace=False)
        feats = np.concatenate([probs[i].feats for i in idx])
        F, beta, acts = mlp.forward(feats)
        betas = beta.view(-1, 4).double().cpu().numpy()
        gb, losses, off = [], [], 0
        for i in idx:
            nl = probs[i].feats.shape[0]
            loss, g = probs[i].loss_grad(betas[off:off + nl])
            losses.append(loss)
            gb.append(g / len(idx))
            off += nl
        mlp.backward_and_step(F, beta, acts, np.concatenate(gb), lr)
        hist.append(float(np.mean(losses)))
        if log:
            log(it, hist[-1])
    return hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=512)
    ap.add_argument("--heldout", type=int, default=32)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default="learned_weights.npz")
    ap.add_argument("--resume", default=None)
    a = ap.parse_args()
    t0 = time.time()
    train_set = make_training_set(a.problems, a.grid, seed0=0)
    test_set = make_training_set(a.heldout, a.grid, seed0=100000)
    t_setup = time.time() - t0
    mlp = WeightMLP(seed=0)
    if a.resume:
        mlp.load(a.resume)
    before = evaluate(mlp, test_set)
    t1 = time.time()
    hist = train(mlp, train_set, a.steps, batch=a.batch, lr=a.lr,
                 log=lambda i, l: print(f"step {i} loss {l:.6f}", flush=True) if i % 20 == 0 else None)
    t_train = time.time() - t1
    after = evaluate(mlp, test_set)
    mlp.save(a.out)
    print(json.dumps({"setup_s": t_setup, "train_s": t_train, "steps": a.steps,
                      "heldout_loss_learned_before": before[0], "heldout_loss_opt": before[1],
                      "heldout_loss_learned_after": after[0],
                      "train_loss_first": hist[0], "train_loss_last": hist[-1]}))


if __name__ == "__main__":
    main()
