"""Learned inner-solve controller: trajectory generation, training on the GPU
with the library's own MLP kernels, and evaluation against the paper's rules.

The network (16 -> 64 -> 64 -> 2, GELU) maps the per-outer-iteration features
of the solver trace (see pdnqp_get_trace in include/pdnqp.h) to a correction
of the rules' action (logit of the rho_in fraction, log ratio of the next
primal weight); with a zero last layer it reproduces the rules.  It is
trained by reward-weighted regression on trajectories the method generates
itself: the solver runs the paper's rules with Gaussian exploration noise on
the actions, each action is scored by the progress it bought (decrease of
log10 of the relative KKT residual per log10 of the inner iterations the next
inner solve needed), and the network regresses onto the deviations from the
rules that were taken, with weights exp(beta * standardised score).  Feature
standardisation is folded into the first layer, so the solver feeds raw
features.  In the solver the paper's rules stay the fallback and decide when
a proposal is overruled (pdnqp_set_controller).

    python -m paper_2609_19557_gb300.controller --train 200 --eval 8 --out weights.npy
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import instances as I
from . import mlp_data as D
from . import pdnqp as P

F0, NF = 3, 16          # feature columns in the trace
A_RULE, A_TAKEN = 19, 21  # the rules' action (19, 20) and the action taken (21, 22)


def make_instance(seed: int, n: int, shift: float = None) -> dict:
    """The mid-size generator (power-law rows, free variables, equality rows) at n variables, m = n / 2."""
    return I.mid_qp(seed, n=n, m=n // 2, replica_n=min(3000, n), shift=shift)


def _make_args(a):
    return make_instance(*a)


def make_instances(specs, procs=0, pool=None):
    """Instances for (seed, n, shift) specs, in `pool` or in a pool of `procs`
    processes (spawned: no copy of a CUDA context) when procs > 1."""
    if pool is not None:
        return pool.map(_make_args, specs, chunksize=1)
    if procs <= 1 or len(specs) < 2:
        return [make_instance(*sp) for sp in specs]
    with spawn_pool(procs) as pl:
        return pl.map(_make_args, specs, chunksize=1)


def spawn_pool(procs):
    """A pool of `procs` spawned processes (no copy of a CUDA context) whose
    numeric libraries run one thread each: the variables are read when a
    child imports them, and one BLAS thread pool per child would oversubscribe
    the cores."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        return mp.get_context("spawn").Pool(procs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def create_all(insts, setup, threads=16):
    """Handles for `insts` (FP32-bulk), created by `threads` host threads at
    once (each creation runs on its own stream; the C calls release the GIL),
    then set up by setup(k, handle)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(k):
        h = P.create_from_instance(insts[k], precision=32)
        setup(k, h)
        return h

    with ThreadPoolExecutor(max(1, threads)) as ex:
        return list(ex.map(one, range(len(insts))))


def generate_batched(count, rng, n_min, n_max, *, eps, explore, time_limit, threads, chunk=64, procs=0,
                     progress=None, budget_s=float("inf")):
    """Training trajectories solved together (pdnqp_solve_batch), `chunk`
    problems at a time; the instances share the diagonal shift of the first
    (same density), which saves the replica eigen-decomposition per instance,
    and are built in `procs` processes."""
    ns = [int(rng.integers(n_min, n_max + 1)) for _ in range(count)]
    shift = make_instance(10_000, ns[0])["shift"] if count else None
    data = []
    pool = spawn_pool(procs) if procs > 1 else None
    t_start = time.perf_counter()
    for c0 in range(0, count, chunk):
        if time.perf_counter() - t_start > budget_s:
            break  # the generation budget is spent: train on the trajectories so far
        idx = list(range(c0, min(count, c0 + chunk)))
        insts = make_instances([(10_000 + i, ns[i], shift) for i in idx], procs, pool)

        def setup(k, h):
            P.pdnqp_set_param(h, "time_limit", time_limit)
            P.pdnqp_set_param(h, "ctrl_explore", explore)
            P.pdnqp_set_param(h, "ctrl_seed", idx[k])

        hs = create_all(insts, setup, max(1, threads))
        P.pdnqp_solve_batch(hs, eps, eps, threads=threads)
        for h in hs:
            data += transitions(P.pdnqp_get_trace(h))
            h.close()
        if progress:
            progress(idx[-1] + 1, data)
    if pool is not None:
        pool.close()
        pool.join()
    return data


def evaluate_batched(insts, theta, *, eps, time_limit, chunk=64):
    """The rules and the network on the same instances (paired), each side
    solved as fused batches; per instance the status, outer and inner
    iterations and the relative KKT residual of both sides."""
    out = []
    for c0 in range(0, len(insts), chunk):
        sub = insts[c0:c0 + chunk]
        res = {}
        for side in ("rule", "mlp"):
            def setup(k, h, side=side):
                P.pdnqp_set_param(h, "time_limit", time_limit)
                if side == "mlp":
                    P.pdnqp_set_controller(h, theta)
                    P.pdnqp_set_param(h, "controller", 1)

            hs = create_all(sub, setup)
            sts = P.pdnqp_solve_batch(hs, eps, eps)
            rows = []
            for h, st in zip(hs, sts):
                x, y, r = P.pdnqp_get(h)
                rows.append({"status": P.STATUS_NAMES[st], "outer": r["outer_iters"], "inner": r["inner_iters"],
                             "rel_kkt": r["rel_kkt"], "ctrl_used": r["ctrl_used"], "x": x, "y": y})
                h.close()
            res[side] = rows
        for inst, a, b in zip(sub, res["rule"], res["mlp"]):
            out.append({"n": inst["Q"].shape[0], "rule": a, "mlp": b})
    return out


def sign_test(d):
    """Two-sided exact sign test of the paired differences d (zeros dropped):
    (count of negatives, count of nonzero, p-value)."""
    from math import comb
    d = np.asarray(d)
    d = d[d != 0]
    k, nn = int((d < 0).sum()), int(d.size)
    if nn == 0:
        return 0, 0, 1.0
    lo = min(k, nn - k)
    p = min(1.0, 2.0 * sum(comb(nn, i) for i in range(lo + 1)) / 2.0 ** nn)
    return k, nn, p


def run(inst: dict, *, precision=32, eps=1e-4, controller=None, explore=0.0, seed=0, time_limit=60.0, stream=None):
    h = P.create_from_instance(inst, precision=precision, stream=stream)
    P.pdnqp_set_param(h, "time_limit", time_limit)
    if controller is not None:
        P.pdnqp_set_controller(h, controller)
        P.pdnqp_set_param(h, "controller", 1)
    if explore > 0:
        P.pdnqp_set_param(h, "ctrl_explore", explore)
        P.pdnqp_set_param(h, "ctrl_seed", seed)
    t = time.perf_counter()
    st = P.pdnqp_solve(h, eps, eps)
    wall = time.perf_counter() - t
    x, y, r = P.pdnqp_get(h)
    tr = P.pdnqp_get_trace(h)
    h.close()
    return {"status": P.STATUS_NAMES[st], "outer": r["outer_iters"], "inner": r["inner_iters"],
            "rel_kkt": r["rel_kkt"], "seconds": wall, "ctrl_used": r["ctrl_used"],
            "ctrl_fallbacks": r["ctrl_fallbacks"], "x": x, "y": y}, tr


def transitions(trace: np.ndarray):
    """(features, action, score) of every action whose outcome the trace shows."""
    out = []
    for k in range(len(trace) - 1):
        a, b = trace[k], trace[k + 1]
        gain = np.log10(max(a[1], 1e-300)) - np.log10(max(b[1], 1e-300))
        cost = np.log10(10.0 + b[2])
        out.append((a[F0:F0 + NF], a[A_TAKEN:A_TAKEN + 2] - a[A_RULE:A_RULE + 2], gain / cost))
    return out


def train(feats, acts, scores, *, beta=1.0, epochs=3000, lr=3e-3, seed=0):
    """Reward-weighted regression with the library's forward / backward / Adam
    kernels; returns FP32 weights with the feature standardisation folded in."""
    import torch
    X = np.asarray(feats, dtype=np.float64)
    A = np.asarray(acts, dtype=np.float32)
    S = np.asarray(scores, dtype=np.float64)
    mu, sd = X.mean(axis=0), X.std(axis=0)
    sd[sd < 1e-6] = 1.0
    Xn = ((X - mu) / sd).astype(np.float32)
    z = (S - S.mean()) / (S.std() + 1e-12)
    wt = np.exp(np.clip(beta * z, -3.0, 3.0)).astype(np.float32)
    B = len(Xn)
    w32 = D.init_weights(seed)
    w32[D.N_PARAMS - D.N_OUT * D.N_HID - D.N_OUT:] = 0.0  # zero last layer: starts as the rules
    w = torch.tensor(w32, device="cuda")
    wb = torch.zeros(w32.size, dtype=torch.int16, device="cuda")
    P.mlp_to_bf16(w, wb)
    x, t, ww = (torch.tensor(v, device="cuda") for v in (Xn, A, wt))
    y = torch.zeros((B, 2), device="cuda")
    cache = torch.zeros((B, 128), device="cuda")
    dy, loss = torch.zeros_like(y), torch.zeros(1, device="cuda")
    m, v, grad = torch.zeros_like(w), torch.zeros_like(w), torch.zeros_like(w)
    scratch = torch.zeros(((B + 15) // 16) * w.numel(), device="cuda")
    hist = []
    for step in range(1, epochs + 1):
        P.mlp_forward(wb, x, y, cache)
        P.mlp_wmse(y, t, ww, dy, loss)
        P.mlp_backward(wb, x, cache, dy, grad, scratch)
        P.mlp_adam(w, wb, grad, m, v, step, lr=lr)
        if step == 1 or step % 500 == 0:
            hist.append((step, loss.item()))
    theta = w.cpu().numpy().astype(np.float64)
    # Fold x_n = (x - mu) / sd into the first layer: W1' = W1 / sd, b1' = b1 - W1' mu.
    n1 = D.N_HID * D.N_IN
    W1 = theta[:n1].reshape(D.N_HID, D.N_IN) / sd
    theta[:n1] = W1.ravel()
    theta[n1:n1 + D.N_HID] -= W1 @ mu
    return theta.astype(np.float32), hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200, help="training trajectories")
    ap.add_argument("--eval", type=int, default=8, help="fresh evaluation instances")
    ap.add_argument("--n-min", type=int, default=10_000)
    ap.add_argument("--n-max", type=int, default=50_000)
    ap.add_argument("--explore", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--time-limit", type=float, default=60.0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--data", default=None, help="transitions file (.npz): loaded if present, else written")
    ap.add_argument("--threads", type=int, default=0, help="solve the training trajectories concurrently")
    ap.add_argument("--eval-n-min", type=int, default=None)
    ap.add_argument("--eval-n-max", type=int, default=None)
    ap.add_argument("--compare", default=None, help="weights (.npy) evaluated on the same instances too")
    ap.add_argument("--procs", type=int, default=0, help="processes that build the instances")
    ap.add_argument("--eval-batched", action="store_true",
                    help="paired evaluation with fused batches (iteration counts; no per-problem wall time)")
    ap.add_argument("--weights", default=None, help="evaluate these weights (.npy) instead of training")
    ap.add_argument("--eval-time-limit", type=float, default=None,
                    help="time limit of the evaluation solves (default: --time-limit)")
    ap.add_argument("--gen-budget", type=float, default=float("inf"),
                    help="seconds after which no new chunk of training trajectories starts")
    a = ap.parse_args()
    P.load()
    rng = np.random.default_rng(np.random.SeedSequence([2024, 7]))
    gen_done = [a.train]  # training trajectories actually generated (a generation budget may cut them)
    t0 = time.perf_counter()
    if a.weights:
        feats = acts = scores = []
        for _ in range(a.train):  # the evaluation sizes of a run that trained on a.train trajectories
            rng.integers(a.n_min, a.n_max + 1)
    elif a.data and os.path.exists(a.data):
        z = np.load(a.data)
        feats, acts, scores = z["feats"], z["acts"], z["scores"]
        for _ in range(a.train):  # keep the evaluation sizes of a fresh run
            rng.integers(a.n_min, a.n_max + 1)
    elif a.threads > 0:
        def progress(done, data):
            gen_done[0] = done
            print(json.dumps({"trajectories_done": done, "transitions": len(data),
                              "seconds": time.perf_counter() - t0}), file=sys.stderr, flush=True)
            if a.data:
                f, ac, sc = (np.array(v) for v in zip(*data))
                np.savez(a.data, feats=f, acts=ac, scores=sc)

        data = generate_batched(a.train, rng, a.n_min, a.n_max, eps=a.eps, explore=a.explore,
                                time_limit=a.time_limit, threads=a.threads, procs=a.procs, progress=progress,
                                budget_s=a.gen_budget)
        feats, acts, scores = (np.array(v) for v in zip(*data))
        if a.data:
            np.savez(a.data, feats=feats, acts=acts, scores=scores)
    else:
        data = []
        for i in range(a.train):
            n = int(rng.integers(a.n_min, a.n_max + 1))
            _, tr = run(make_instance(10_000 + i, n), eps=a.eps, explore=a.explore, seed=i, time_limit=a.time_limit)
            data += transitions(tr)
        feats, acts, scores = (np.array(v) for v in zip(*data))
        if a.data:
            np.savez(a.data, feats=feats, acts=acts, scores=scores)
    gen_s = time.perf_counter() - t0
    if a.weights:
        theta, hist = np.load(a.weights).astype(np.float32), []
    else:
        theta, hist = train(feats, acts, scores)
    if a.out:
        np.save(a.out, theta)
    rows = []
    e_lo = a.eval_n_min if a.eval_n_min else a.n_min
    e_hi = a.eval_n_max if a.eval_n_max else a.n_max
    if a.eval_batched:
        ns = [int(rng.integers(e_lo, e_hi + 1)) for _ in range(a.eval)]
        shift = make_instance(90_000, ns[0])["shift"] if a.eval else None
        insts = make_instances([(90_000 + j, ns[j], shift) for j in range(a.eval)], a.procs)
        ev = evaluate_batched(insts, theta, eps=a.eps,
                              time_limit=a.eval_time_limit if a.eval_time_limit else a.time_limit)
        both = [e for e in ev if e["rule"]["status"] == e["mlp"]["status"] == "SOLVED"]
        summary = {}
        for key in ("outer", "inner"):
            d = [e["mlp"][key] - e["rule"][key] for e in both]
            k, nn, p = sign_test(d)
            summary[key] = {"rule_total": int(sum(e["rule"][key] for e in both)),
                            "mlp_total": int(sum(e["mlp"][key] for e in both)),
                            "mlp_fewer": k, "nonzero": nn, "sign_test_p": p,
                            "median_ratio": float(np.median([e["mlp"][key] / max(1, e["rule"][key]) for e in both]))
                            if both else None}
        print(json.dumps({"trajectories": gen_done[0], "transitions": len(scores), "generation_s": gen_s, "loss": hist,
                          "eval_instances": a.eval, "both_solved": len(both),
                          "statuses": [[e["rule"]["status"], e["mlp"]["status"]] for e in ev],
                          "paired": summary,
                          "rows": [{"n": e["n"], **{f"{s}_{k}": e[s][k] for s in ("rule", "mlp")
                                                    for k in ("outer", "inner", "rel_kkt", "ctrl_used")}}
                                   for e in ev]}, default=float))
        return
    for j in range(a.eval):
        n = int(rng.integers(e_lo, e_hi + 1))
        inst = make_instance(90_000 + j, n)
        base, _ = run(inst, eps=a.eps, time_limit=a.time_limit)
        ctrl, _ = run(inst, eps=a.eps, controller=theta, time_limit=a.time_limit)
        if a.compare:
            old, _ = run(inst, eps=a.eps, controller=np.load(a.compare).astype(np.float32), time_limit=a.time_limit)
        rows.append({"n": n, **{f"rule_{k}": base[k] for k in ("status", "outer", "inner", "seconds", "rel_kkt")},
                     **{f"mlp_{k}": ctrl[k] for k in ("status", "outer", "inner", "seconds", "rel_kkt",
                                                      "ctrl_used", "ctrl_fallbacks")},
                     **({f"old_{k}": old[k] for k in ("status", "outer", "inner", "seconds", "rel_kkt")}
                        if a.compare else {})})
    print(json.dumps({"trajectories": a.train, "transitions": len(scores), "generation_s": gen_s,
                      "loss": hist, "eval": rows}, default=float))


if __name__ == "__main__":
    main()
