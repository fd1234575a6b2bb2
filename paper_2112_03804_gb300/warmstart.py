"""Learned warm start of the batched RM+ solver (not in the paper).

Every computation runs in libkps.so: the solver (kps_solver_*), the feature,
target and scatter gathers (kps_warm_*) and the network's forward, backward
and Adam kernels (kps_mlp_*).  This module only sequences the calls:

  solve   -- run a solver on a batch until every game's exploitability of the
             average is below a target (checked every `block` iterations)
  sample  -- pick (game, player, node, hand) queries of a solved batch and
             gather their features, action counts, equilibrium targets and
             weights (reach of the node times the hand's belief)
  train   -- minibatch Adam on the weighted cross-entropy
  predict -- the network's strategy at every query of a batch, scattered
             into behavioural strategies in the batch layout
  compare -- iterations and wall time to the target from a cold start and
             from the network's prediction (kps_solver_warm_start)
"""
from __future__ import annotations

import time

import numpy as np

from . import kps


def _torch():
    import torch
    return torch


def solve(batch: "kps.Batch", dtype: int, target: float, block: int = 25, max_iters: int = 2000,
          solver: "kps.Solver" = None, start=None, stream=None, method: int = 0):
    """Runs RM+ (method 0) or Discounted CFR (method 1) until max over games
    of the FP64 exploitability < target (an FP32 estimate every `block`
    iterations decides when to evaluate it).  `start` = (beh1, beh2, kappa, t0) for a
    warm start.  Returns (solver, iterations run, exploitability per game
    [numpy], wall seconds)."""
    torch = _torch()
    ng = len(batch.games)
    s = solver or kps.Solver(batch, dtype)
    s.set_method(method)
    e = torch.zeros(ng, dtype=torch.float64, device="cuda")
    s.step(block, stream)            # capture the iteration graph outside the timed run
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if start is None:
        s.reset(stream=stream)
    else:
        s.warm_start(start[0], start[1], start[2], start[3], stream)
    it = 0
    ex = None
    while True:
        # cheap FP32 estimate every block; a stop is confirmed in FP64 (the
        # estimate's rounding, ~1e-6 of the pot, is covered by the margin)
        s.exploitability_estimate(e, stream=stream)
        if e.max().item() < target * 1.001 or it >= max_iters:
            s.exploitability(e, stream=stream)
            ex = e.cpu().numpy()
            if ex.max() < target or it >= max_iters:
                break
        s.step(block, stream)
        it += block
    return s, it, ex, time.perf_counter() - t0


def sample(batch: "kps.Batch", solver: "kps.Solver", per_game: int, seed: int):
    """Features, action counts, targets and weights of `per_game` random
    queries of every game (uniform over the game's nodes and hands)."""
    torch = _torch()
    off = [batch.offsets(p) for p in (0, 1)]
    x = [torch.zeros(int(off[p][-1]), dtype=torch.float64, device="cuda") for p in (0, 1)]
    b = [torch.zeros(int(off[p][-1]), dtype=torch.float64, device="cuda") for p in (0, 1)]
    solver.average(x[0], x[1], behavioural=False)
    solver.average(b[0], b[1], behavioural=True)
    r = np.random.default_rng(seed)
    # query ranges per game
    starts = [0]
    for g in batch.games:
        inf = g.info()
        starts.append(starts[-1] + (inf["nodes1"] + inf["nodes2"]) * inf["H"])
    idx = np.concatenate([r.integers(starts[i], starts[i + 1], size=per_game) for i in range(len(batch.games))])
    qidx = torch.from_numpy(idx.astype(np.int64)).cuda()
    n = len(idx)
    X = torch.empty(n, kps.WARM_DIN, device="cuda")
    nact = torch.empty(n, dtype=torch.int32, device="cuda")
    T = torch.empty(n, kps.WARM_DOUT, device="cuda")
    w = torch.empty(n, device="cuda")
    kps.warm_features(batch, X, nact, qidx=qidx)
    kps.warm_targets(batch, b[0], b[1], x[0], x[1], T, w, qidx=qidx)
    return {"X": X, "nact": nact, "T": T, "w": w}


def concat(datasets):
    torch = _torch()
    return {k: torch.cat([d[k] for d in datasets]) for k in datasets[0]}


def train(mlp: "kps.MLP", data, epochs: int, rows: int = 4096, lr: float = 1e-3, seed: int = 0,
          lr_decay: float = 1.0):
    """Minibatch Adam; returns the mean loss of every epoch."""
    torch = _torch()
    n = data["X"].shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.zeros(1, device="cuda")
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot = torch.zeros(1, device="cuda")
        nb = 0
        for s in range(0, n - rows + 1, rows):
            sel = perm[s:s + rows]
            X, na, T, w = (data[k][sel].contiguous() for k in ("X", "nact", "T", "w"))
            wsum = float(w.sum().item())
            if not wsum > 0:
                continue
            mlp.gradients(X, rows, na, T, w, wsum, loss)
            mlp.adam(lr)
            tot += loss
            nb += 1
        lr *= lr_decay
        hist.append(float(tot.item()) / max(nb, 1))
    return hist


def predict(mlp: "kps.MLP", batch: "kps.Batch"):
    """Behavioural strategies (device FP32, batch layouts) predicted at every
    query of the batch (the fused predictor)."""
    torch = _torch()
    off = [batch.offsets(p) for p in (0, 1)]
    beh = [torch.zeros(int(off[p][-1]), device="cuda") for p in (0, 1)]
    kps.warm_predict(batch, mlp, beh[0], beh[1])
    return beh


def predict_unfused(mlp: "kps.MLP", batch: "kps.Batch", chunk: int = 1 << 16):
    """The same through materialised feature rows and the training forward
    (FP32 activations); for checks."""
    torch = _torch()
    nq = kps.warm_num_queries(batch)
    off = [batch.offsets(p) for p in (0, 1)]
    beh = [torch.zeros(int(off[p][-1]), device="cuda") for p in (0, 1)]
    X = torch.empty(chunk, kps.WARM_DIN, device="cuda")
    nact = torch.empty(chunk, dtype=torch.int32, device="cuda")
    P = torch.empty(chunk, kps.WARM_DOUT, device="cuda")
    for q0 in range(0, nq, chunk):
        n = min(chunk, nq - q0)
        kps.warm_features(batch, X, nact, q0=q0, nq=n)
        mlp.forward(X, n, nact, P)
        kps.warm_scatter(batch, P, beh[0], beh[1], q0=q0, nq=n)
    return beh


def compare(mlp: "kps.MLP", batch: "kps.Batch", dtype: int, target: float, kappa: float, t0: int,
            block: int = 25, max_iters: int = 2000, method: int = 0):
    """Cold start vs warm start from the network on one batch."""
    torch = _torch()
    s_cold, it_cold, e_cold, sec_cold = solve(batch, dtype, target, block, max_iters, method=method)
    torch.cuda.synchronize()
    t_inf = time.perf_counter()
    beh = predict(mlp, batch)
    torch.cuda.synchronize()
    sec_inf = time.perf_counter() - t_inf
    _, it_warm, e_warm, sec_warm = solve(batch, dtype, target, block, max_iters, solver=s_cold,
                                         start=(beh[0], beh[1], kappa, t0), method=method)
    return {"games": len(batch.games), "target": target, "check_every": block,
            "cold": {"iterations": it_cold, "seconds": sec_cold, "max_expl": float(e_cold.max())},
            "warm": {"iterations": it_warm, "seconds": sec_warm + sec_inf, "solve_seconds": sec_warm,
                     "inference_seconds": sec_inf, "max_expl": float(e_warm.max())},
            "kappa": kappa, "t0": t0, "method": "dcfr" if method else "rm+"}
