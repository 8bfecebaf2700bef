"""Surrogate-screened scans of the pair probability (the learned part of the workload).

The solver (``solve_swf``) produces training targets y = ln P, P = sum_r |C((s,p),(r,q=-p))|^2,
for sampled (E, omega, lambda, p_x, p_y, s); the network of ``swf_mlp_*`` (BF16 tensor-core
kernels) learns y with an error estimate sigma; a scan accepts the network where sigma is below
a threshold calibrated on held-out solver data and falls back to the solver elsewhere.  All
arithmetic runs in the CUDA library; this module only arranges calls and data.
"""
from __future__ import annotations

import time

import numpy as np

from . import swf


def instances(E, om, lam, px, py, s, n=256, L=40.0, n_steps=1000, t_window=20.0):
    """Schwinger instances of the surrogate's sample table (one per sample)."""
    out = []
    for i in range(len(E)):
        out.append(swf.make_instance(swf.FIELD_SAUTER_GAUSS, (E[i], om[i], lam[i]), (n, n, 1), (L, L, 1.0),
                                     -t_window, t_window, n_steps, p=(px[i], py[i], 0.0), s=int(s[i]),
                                     q=(-px[i], -py[i], 0.0), r=1))
    return out


def features(table):
    return np.stack([table["E"], table["omega"], table["lam"], table["px"], table["py"],
                     np.asarray(table["s"], float)], axis=1).astype(np.float32)


def solve_targets(ctx, table, batch=128, prec=swf.C64, **grid):
    """ln P from the solver for every row of a sample table (batches of instances per call)."""
    insts = instances(table["E"], table["omega"], table["lam"], table["px"], table["py"], table["s"], **grid)
    y = np.zeros(len(insts))
    for b0 in range(0, len(insts), batch):
        res, _ = ctx.solve(insts[b0:b0 + batch], swf.SCHWINGER, prec)
        for j, r in enumerate(res):
            y[b0 + j] = np.log(r.prob[0] + r.prob[1])
    return y


def normalisation(X, y):
    """Feature and target standardisation (14 floats, the layout of swf_mlp_create)."""
    shift = X.mean(axis=0)
    scale = 1.0 / np.maximum(X.std(axis=0), 1e-6)
    return np.concatenate([shift, scale, [y.mean(), 1.0 / max(y.std(), 1e-6)]]).astype(np.float32)


def init_params(seed=0):
    """He-style initial weights (drawn here and passed in, so that tests can reproduce them)."""
    from .swf import Surrogate
    rng = np.random.default_rng(seed)
    dims = [(6, 256), (256, 256), (256, 256), (256, 256), (256, 2)]
    p = []
    for i, o in dims:
        p.append(rng.normal(scale=np.sqrt(2.0 / i), size=i * o))
        p.append(np.zeros(o))
    p = np.concatenate(p).astype(np.float32)
    assert p.size == Surrogate.param_count()
    return p


def train(sur, X, y, epochs=200, batch=256, lr=1e-3, seed=0):
    """Mini-batch Adam over the training set; returns the loss of every epoch's last batch."""
    import torch
    rng = np.random.default_rng(seed)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(len(X))).cuda()
        for b0 in range(0, len(X) - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            sur.train_step(Xd[idx].contiguous(), yd[idx].contiguous(), lr, loss)
        hist.append(float(loss.item()))
    return hist


def predict(sur, X):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    out = torch.zeros(len(X), 2, dtype=torch.float32, device="cuda")
    sur.forward(Xd, out)
    o = out.cpu().numpy()
    return o[:, 0].astype(float), np.exp(0.5 * o[:, 1].astype(float))


def calibrate(sur, X, y, tol, coverage=0.99):
    """Largest sigma threshold such that at least `coverage` of the accepted held-out points are
    within `tol` of the solver (absolute in ln P, i.e. relative in P)."""
    mu, sig = predict(sur, X)
    err = np.abs(mu - y)
    order = np.argsort(sig)
    ok = err[order] <= tol
    best = 0.0
    for k in range(1, len(order) + 1):
        if ok[:k].mean() >= coverage:
            best = sig[order[k - 1]]
    return best


def screened_scan(sur, ctx, table, threshold, batch=128, **grid):
    """ln P over a scan: the network where its sigma <= threshold, the solver elsewhere.
    Returns (values, accepted mask, seconds in the network, seconds in the solver)."""
    X = features(table)
    t0 = time.perf_counter()
    mu, sig = predict(sur, X)
    t_net = time.perf_counter() - t0
    acc = sig <= threshold
    vals = mu.copy()
    t1 = time.perf_counter()
    rest = np.nonzero(~acc)[0]
    if len(rest):
        sub = {k: np.asarray(v)[rest] for k, v in table.items()}
        vals[rest] = solve_targets(ctx, sub, batch=batch, **grid)
    t_sol = time.perf_counter() - t1
    return vals, acc, t_net, t_sol
