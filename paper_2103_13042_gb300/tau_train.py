"""Learned tau: training data generated by the method itself, GPU training and evaluation.

Every step runs in the library's kernels (norm maps, plans, band products,
Frobenius reductions, histogram, network forward / backward / Adam); torch
only holds device memory.

Achieved error without forming AB.  For a pair (A, B) a reference threshold
tau_ref is certified by bisection on the plan's skipped-product bound:
||AB - SpAMM(tau_ref)||_F <= bound2(tau_ref) <= 1e-11 ||A||_F ||B||_F.  The
pruning error at tau > tau_ref is then the band product over
tau_ref <= p < tau (spamm_plan_band), up to that certified 1e-11:

    e(tau) = ||SpAMM_band(tau_ref, tau)||_F / (||A||_F ||B||_F).

Data: for each seeded decay pair (N in {1024, 2048, 4096, 8192}, exponential
or algebraic decay, random rate) and each tau of a jittered log grid, one
tuple (histogram of relative norm products, log10 e(tau)) -> log10(tau /
(||A|| ||B||)).  Training: Adam on the pinball loss at quantile q < 0.5
(the network errs on the small-tau side, where the target error still holds).
Evaluation on held-out pairs: hit rate of e(tau_pred) <= target, and the
time to an admissible tau (prediction + one check, bisection on a miss)
against plain bisection on e.

Usage (on a GPU):
    python -m paper_2103_13042_gb300.tau_train --out paper_2103_13042_gb300/data
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

LEAF = 64
REF_REL = 1e-11           # certified reference bound (relative to ||A|| ||B||)
TARGETS = (1e-3, 1e-4, 1e-5, 1e-6, 1e-7)
WEIGHTS_NAME = "tau_mlp_leaf64.f32"
REPORT_NAME = "tau_mlp_leaf64.json"


def _lib():
    import paper_2103_13042_gb300 as P
    return P


class ErrorMeter:
    """Achieved relative pruning error of one (A, B) pair at any tau, through the library's
    spamm_tau_certify (tau_ref) and spamm_tau_error (band products)."""

    def __init__(self, n: int, device):
        import torch
        P = _lib()
        self.n = n
        self.plan = P.Plan(n, LEAF, P.FP32)
        bd = P.num_blocks(n, LEAF)
        self.nA = torch.empty((bd, bd), dtype=torch.float64, device=device)
        self.nB = torch.empty_like(self.nA)
        self.T = torch.empty((n, n), dtype=torch.float32, device=device)
        self.evals = 0

    def setup(self, A, B):
        P = _lib()
        self.A, self.B = A, B
        P.spamm_normmap(A, LEAF, self.nA)
        P.spamm_normmap(B, LEAF, self.nB)
        self.tau_ref, self.ab = self.plan.tau_certify(self.nA, self.nB, REF_REL)
        return self

    def error(self, tau: float) -> float:
        """e(tau) = ||AB - SpAMM(tau)||_F / (||A|| ||B||) up to the certified REF_REL."""
        self.evals += 1
        return self.plan.tau_error(self.nA, self.nB, self.A, self.B, tau, self.tau_ref, self.T)

    def select(self, eps: float, weights=None):
        """(tau, evaluations, e(tau)) of spamm_tau_select: the network's tau checked once with
        bisection on a miss, or plain bisection without weights."""
        return self.plan.tau_select(self.nA, self.nB, self.A, self.B, eps, weights, self.T)

    def histogram(self):
        h = self.plan.histogram(self.nA, self.nB).astype(np.float64)
        return h / h.sum()


def make_dataset(specs, device, sweep: int, seed: int, log=print):
    """Tuples (features[65], log10 tau_rel) from the given pair specs."""
    import synth
    rng = np.random.default_rng(seed)
    meters = {}
    X, Y = [], []
    t0 = time.time()
    for t, sp in enumerate(specs):
        A, B = synth.spec_matrices_device(sp, device)
        m = meters.get(sp["n"]) or meters.setdefault(sp["n"], ErrorMeter(sp["n"], device))
        m.setup(A, B)
        h = m.histogram()
        grid = np.linspace(-13.0, -1.0, sweep) + rng.uniform(-0.3, 0.3, size=sweep)
        for lg in grid:
            e = m.error(m.ab * 10.0 ** lg)
            if not (1e-13 < e <= 1e-1):
                continue
            X.append(np.concatenate([h, [math.log10(e)]]))
            Y.append(lg)
        if (t + 1) % 100 == 0:
            log(f"  data: {t + 1}/{len(specs)} pairs, {len(X)} tuples, {time.time() - t0:.1f} s")
    return np.asarray(X, dtype=np.float32), np.asarray(Y, dtype=np.float32)


def train(X, Y, device, epochs: int, batch: int, lr: float, q: float, seed: int, log=print):
    import torch
    import synth
    P = _lib()
    theta = synth.mlp_init(seed)
    theta[-1] = float(np.mean(Y))              # output bias at the mean target
    W = torch.from_numpy(theta).to(device)
    m = torch.zeros_like(W)
    v = torch.zeros_like(W)
    Xd = torch.from_numpy(X).to(device)
    Yd = torch.from_numpy(Y).to(device)
    rng = np.random.default_rng(seed)
    per_epoch = len(Y) // batch
    t = 0
    losses = []
    for ep in range(epochs):
        idx = rng.permutation(len(Y))[:per_epoch * batch].astype(np.int32)
        rate = lr if ep < int(0.7 * epochs) else lr * 0.2
        hist = P.spamm_mlp_train(W, m, v, t, Xd, Yd, torch.from_numpy(idx).to(device), per_epoch,
                                 batch, rate, q)
        t += per_epoch
        losses.append(float(hist.mean().item()))
        if (ep + 1) % max(1, epochs // 10) == 0:
            log(f"  train: epoch {ep + 1}/{epochs}, pinball loss {losses[-1]:.4f}")
    return W, losses


def evaluate(W, specs, device, targets=TARGETS, log=print):
    """Hit rate and time to an admissible tau, network vs plain bisection."""
    import torch
    import synth
    P = _lib()
    meters = {}
    rows = []
    for t, sp in enumerate(specs):
        A, B = synth.spec_matrices_device(sp, device)
        m = meters.get(sp["n"]) or meters.setdefault(sp["n"], ErrorMeter(sp["n"], device))
        m.setup(A, B)
        for eps in targets:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tau_p = m.plan.tau_predict(m.nA, m.nB, eps, W)
            t_pred = time.perf_counter() - t0
            e_p = m.error(tau_p)
            t_check = time.perf_counter() - t0
            hit = e_p <= eps
            t1 = time.perf_counter()
            tau_b, n_b, _ = m.select(eps)            # plain bisection (no network)
            t_bis = time.perf_counter() - t1
            rows.append({"n": sp["n"], "kind": sp["kind"], "eps": eps, "tau_pred": tau_p,
                         "err_pred": e_p, "hit": bool(hit), "tau_bisect": tau_b,
                         "bisect_evals": n_b, "t_predict_s": t_pred, "t_predict_check_s": t_check,
                         "t_bisect_s": t_bis})
        if (t + 1) % 100 == 0:
            log(f"  eval: {t + 1}/{len(specs)} pairs")
    out = {"pairs": len(specs), "per_target": {}}
    for eps in targets:
        r = [x for x in rows if x["eps"] == eps]
        hits = [x for x in r if x["hit"]]
        # time to an admissible tau: prediction + check, plus bisection after a miss
        t_net = [x["t_predict_check_s"] + (0.0 if x["hit"] else x["t_bisect_s"]) for x in r]
        t_bis = [x["t_bisect_s"] for x in r]
        ratio = [x["tau_pred"] / x["tau_bisect"] for x in hits if x["tau_bisect"] > 0]
        out["per_target"][f"{eps:g}"] = {
            "hit_rate": len(hits) / len(r),
            "median_tau_pred_over_bisect_hits": float(np.median(ratio)) if ratio else None,
            "mean_bisect_evals": float(np.mean([x["bisect_evals"] for x in r])),
            "mean_time_network_s": float(np.mean(t_net)),
            "mean_time_bisect_s": float(np.mean(t_bis)),
            "speedup": float(np.mean(t_bis) / np.mean(t_net)),
        }
    allr = rows
    out["overall"] = {
        "hit_rate": sum(x["hit"] for x in allr) / len(allr),
        "mean_time_network_s": float(np.mean([x["t_predict_check_s"] + (0 if x["hit"] else x["t_bisect_s"]) for x in allr])),
        "mean_time_bisect_s": float(np.mean([x["t_bisect_s"] for x in allr])),
    }
    out["overall"]["speedup"] = out["overall"]["mean_time_bisect_s"] / out["overall"]["mean_time_network_s"]
    return out, rows


def main(argv=None):
    import torch
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--pairs", type=int, default=1000)
    ap.add_argument("--test", type=int, default=500)
    ap.add_argument("--sweep", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--quantile", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=synth.config_seed(4))
    args = ap.parse_args(argv)
    device = torch.device("cuda", 0)
    os.makedirs(args.out, exist_ok=True)
    log = lambda s: print(s, flush=True)
    t0 = time.time()
    train_specs = synth.training_specs(args.pairs, args.seed)
    X, Y = make_dataset(train_specs, device, args.sweep, args.seed + 1, log)
    t_data = time.time() - t0
    log(f"dataset: {len(Y)} tuples from {args.pairs} pairs in {t_data:.1f} s")
    t1 = time.time()
    W, losses = train(X, Y, device, args.epochs, args.batch, args.lr, args.quantile, args.seed + 2, log)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    log(f"training: {args.epochs} epochs in {t_train:.1f} s, final loss {losses[-1]:.4f}")
    test_specs = synth.training_specs(args.test, args.seed + 777777)
    res, rows = evaluate(W, test_specs, device, log=log)
    w = W.cpu().numpy().astype(np.float32)
    w.tofile(os.path.join(args.out, WEIGHTS_NAME))
    report = {
        "network": "65-64-64-1 GELU, FP32, y = log10(tau / (||A||_F ||B||_F))",
        "leaf": LEAF, "reference_bound_rel": REF_REL,
        "data": {"pairs": args.pairs, "tuples": int(len(Y)), "sweep": args.sweep,
                 "seconds": t_data, "specs_seed": args.seed},
        "training": {"epochs": args.epochs, "batch": args.batch, "lr": args.lr,
                     "quantile": args.quantile, "seconds": t_train,
                     "loss_first": losses[0], "loss_last": losses[-1]},
        "evaluation": res, "test_specs_seed": args.seed + 777777,
        "command": "python -m paper_2103_13042_gb300.tau_train " + " ".join(sys.argv[1:]),
    }
    with open(os.path.join(args.out, REPORT_NAME), "w") as f:
        json.dump(report, f, indent=1)
    log(json.dumps(res["overall"]))


if __name__ == "__main__":
    main()
