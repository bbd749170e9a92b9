"""GPU parity of the learned-tau pieces: histogram, network forward / gradient /
Adam / training loop, tau prediction, band plans.

Expected values come from the FP64 oracle (oracle/tau.py, oracle/mlp.py) on
the same seeded inputs and weights.  Tolerances: the network runs in FP32, so
forward values agree to 1e-5 relative, gradients to 1e-4 relative (scaled by
the gradient's largest entry), as the oracle's checks state.
"""
import math

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import mlp as OM
from oracle import spamm as S
from oracle import tau as OT
from tests.gpu_helpers import band_ok, dev, host, plan_mask

pytestmark = pytest.mark.gpu


def _pair(n, seed, kind="exp"):
    if kind == "exp":
        return synth.exp_decay_normal(n, 0.05, seed), synth.exp_decay_normal(n, 0.05, seed + 1)
    return synth.alg_decay_signed(n, 2.5, seed), synth.alg_decay_signed(n, 2.5, seed + 1)


def _features(rng, count):
    """Synthetic network inputs: histogram-like rows (non-negative, sum 1) and a log10 target."""
    h = rng.gamma(0.3, size=(count, 64))
    h /= h.sum(axis=1, keepdims=True)
    t = rng.uniform(-7.0, -3.0, size=(count, 1))
    return np.concatenate([h, t], axis=1)


def _boundary_triples(nA, nB, inv):
    """Triples whose bin moves when inv moves by a few ulps (order-dependent roundings)."""
    p = S.triple_products(nA, nB)
    lo = OT.hist_bin(p, inv * (1 - 8e-16))
    hi = OT.hist_bin(p, inv * (1 + 8e-16))
    return int((lo != hi).sum())


@pytest.mark.parametrize("n,leaf,kind", [(1024, 32, "exp"), (1000, 64, "alg"), (640, 128, "exp"),
                                         (96, 32, "alg")])
def test_histogram_matches_oracle(n, leaf, kind):
    a, b = _pair(n, 40 + n, kind)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    plan = P.Plan(n, leaf, P.FP32)
    got = plan.histogram(dev(nA), dev(nB))
    bd = nA.shape[0]
    ref = np.rint(OT.norm_product_histogram(nA, nB) * bd ** 3).astype(np.int64)
    assert got.sum() == bd ** 3
    slack = _boundary_triples(nA, nB, OT.inv_norm_product(nA, nB))
    assert np.abs(got - ref).sum() <= 2 * slack, (got, ref)


def test_histogram_special_values():
    """Zero blocks land in bin 63; a zero matrix puts every triple there."""
    leaf = 32
    a, b = _pair(256, 5)
    a[:64, 64:128] = 0.0
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    plan = P.Plan(256, leaf, P.FP32)
    got = plan.histogram(dev(nA), dev(nB))
    ref = np.rint(OT.norm_product_histogram(nA, nB) * 8 ** 3).astype(np.int64)
    assert np.array_equal(got, ref)
    z = np.zeros_like(nA)
    got0 = plan.histogram(dev(z), dev(nB))
    assert got0[63] == 8 ** 3 and got0[:63].sum() == 0


def test_mlp_forward_matches_oracle():
    rng = np.random.default_rng(7)
    theta = synth.mlp_init(11)
    X = _features(rng, 300)
    got = host(P.spamm_mlp_forward(dev(theta), dev(X.astype(np.float32))))
    ref, _ = OM.forward(theta.astype(np.float64), X.astype(np.float32).astype(np.float64))
    # normwise over the batch: single outputs near zero carry the rounding of
    # their O(1) partial sums, so each is compared against the batch's scale
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("q", [0.1, 0.5])
def test_mlp_grad_matches_oracle(q):
    rng = np.random.default_rng(int(q * 100))
    theta = synth.mlp_init(3)
    X = _features(rng, 97).astype(np.float32)      # not a multiple of the 32-sample chunk
    Y = rng.normal(-6.0, 1.0, size=97).astype(np.float32)
    g, loss = P.spamm_mlp_grad(dev(theta), dev(X), dev(Y), q)
    ref_loss, ref_g = OM.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                                       Y.astype(np.float64), q)
    assert abs(float(host(loss)[0]) - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
    gg = host(g).astype(np.float64)
    assert np.max(np.abs(gg - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))


def test_mlp_adam_matches_oracle():
    rng = np.random.default_rng(21)
    theta = synth.mlp_init(5).astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    W, Mg, Vg = dev(theta.astype(np.float32)), dev(m.astype(np.float32)), dev(v.astype(np.float32))
    for t in range(1, 4):
        grad = rng.normal(0, 1e-2, size=theta.size)
        P.spamm_mlp_adam(W, dev(grad.astype(np.float32)), Mg, Vg, t, 1e-3)
        theta, m, v = OM.adam_step(theta, grad.astype(np.float32).astype(np.float64), m, v, t, 1e-3)
    assert np.max(np.abs(host(W) - theta)) <= 1e-6


def test_mlp_train_loop_matches_oracle():
    """Five Adam steps of the one-launch training loop against the FP64 loop."""
    rng = np.random.default_rng(99)
    theta = synth.mlp_init(8).astype(np.float64)
    X = _features(rng, 256).astype(np.float32)
    Y = rng.normal(-6.0, 1.0, size=256).astype(np.float32)
    steps, batch, lr, q = 5, 64, 1e-3, 0.2
    idx = np.stack([rng.permutation(256)[:batch] for _ in range(steps)]).astype(np.int32)
    W = dev(theta.astype(np.float32))
    Mg = torch.zeros_like(W)
    Vg = torch.zeros_like(W)
    losses = host(P.spamm_mlp_train(W, Mg, Vg, 0, dev(X), dev(Y), dev(idx.ravel()), steps, batch,
                                    lr, q))
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for s in range(steps):
        xs, ys = X[idx[s]].astype(np.float64), Y[idx[s]].astype(np.float64)
        loss, g = OM.loss_and_grad(theta, xs, ys, q)
        assert abs(losses[s] - loss) <= 1e-4 * max(1.0, abs(loss))
        theta, m, v = OM.adam_step(theta, g, m, v, s + 1, lr)
    assert np.max(np.abs(host(W) - theta)) <= 5e-5


@pytest.mark.parametrize("target", [1e-3, 1e-6])
def test_tau_predict_matches_oracle_pipeline(target):
    leaf = 64
    a, b = _pair(1000, 77, "alg")
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    theta = synth.mlp_init(13)
    plan = P.Plan(1000, leaf, P.FP32)
    got = plan.tau_predict(dev(nA), dev(nB), target, dev(theta))
    x = OT.mlp_features(OT.norm_product_histogram(nA, nB), target)
    y, _ = OM.forward(theta.astype(np.float64), x.astype(np.float32).astype(np.float64)[None, :])
    ref = 10.0 ** y[0] * OT.frobenius_from_normmap(nA) * OT.frobenius_from_normmap(nB)
    assert got == pytest.approx(ref, rel=3e-5)


def test_batch_tau_predict_equals_single():
    leaf = 64
    specs = synth.batch_specs(4, 606, n_lo=100, n_hi=700)
    pairs = [synth.spec_matrices(sp) for sp in specs]
    theta = dev(synth.mlp_init(2))
    targets = [1e-3, 1e-4, 1e-5, 1e-7]
    batch = P.Batch([a.shape[0] for a, _ in pairs], leaf, P.BF16, graph=False)
    taus = batch.tau_predict([dev(a) for a, _ in pairs], [dev(b) for _, b in pairs], targets, theta)
    for i, (a, b) in enumerate(pairs):
        A, B = dev(a), dev(b)
        nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
        t1 = P.Plan(a.shape[0], leaf, P.BF16).tau_predict(nA, nB, targets[i], theta)
        assert taus[i] == t1
    batch.close()


@pytest.mark.parametrize("leaf", [32, 64])
def test_band_plan_matches_oracle(leaf):
    n = 700
    a, b = _pair(n, 1234, "exp")
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = S.triple_products(nA, nB)
    t_lo, t_hi = float(np.quantile(p, 0.3)), float(np.quantile(p, 0.8))
    plan = P.Plan(n, leaf, P.FP32).band(dev(nA), dev(nB), t_lo, t_hi)
    surv, _ = plan_mask(plan)
    ref = S.survives(p, t_lo) & ~S.survives(p, t_hi)
    assert np.array_equal(surv, ref)
    C = torch.full((n, n), float("nan"), device="cuda")
    plan.multiply(dev(a), dev(b), C)
    cref = S.multiply_with_skipset(a, b, leaf, ref)
    assert np.linalg.norm(host(C) - cref) <= 1e-5 * np.linalg.norm(cref)
    # the band error identity: SpAMM(t_lo) - SpAMM(t_hi) = band product
    c_lo = S.multiply_with_skipset(a, b, leaf, S.flat_survivors(nA, nB, t_lo))
    c_hi = S.multiply_with_skipset(a, b, leaf, S.flat_survivors(nA, nB, t_hi))
    # (FP64 cancellation in c_lo - c_hi is relative to ||c_lo||)
    assert np.linalg.norm((c_lo - c_hi) - cref) <= 1e-13 * np.linalg.norm(c_lo)


# --------------------------------------------------------------------------- Table 1 on the GPU

def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


@pytest.mark.parametrize("n", [1024, 2048, 4096])
def test_table1_valid_ratios_on_gpu(n):
    """The paper's printed tau values give the printed valid ratios (+-1.5 points) through the
    GPU norm map and plan (Section 4.1, Table 1; leaf 32)."""
    t = _golden("table1.json")
    col = t["n"].index(n)
    A = dev(synth.table1_matrix(n))
    nA = P.spamm_normmap(A, 32)
    plan = P.Plan(n, 32, P.FP32)
    for label, taus in t["rows"].items():
        st = plan.plan(nA, nA, taus[col]).stats()
        assert abs(st["valid_ratio"] - float(label)) <= 0.015, (n, label, st["valid_ratio"])


@pytest.mark.parametrize("target", [0.3, 0.1, 0.05])
def test_valid_ratio_search_matches_oracle(target):
    n, leaf = 1024, 32
    a = synth.table1_matrix(n)
    nA = S.normmap(a, leaf)
    plan = P.Plan(n, leaf, P.FP32)
    tau, ratio, probes = plan.tau_for_valid_ratio(dev(nA), dev(nA), target, 0.01, 20)
    ref_tau, ref_ratio, ref_probes = OT.tau_for_valid_ratio(nA, nA, target, iters=20, tol=0.01)
    assert abs(ratio - target) <= 0.01 or probes == 20
    assert ratio == pytest.approx(OT.valid_ratio_at(nA, nA, tau), abs=0)
    assert probes == ref_probes
    assert tau == pytest.approx(ref_tau, rel=1e-12)
