"""The library's tau bisection (spamm_tau_select), which judges the learned tau and replaces it
on a miss, against the oracle's bisection (oracle.tau.bisect_tau) run on the oracle's own
error: e(tau) = ||SpAMM(A, B, tau) - AB||_F / (||A||_F ||B||_F) with the FP64 flat rule and the
dense FP64 product.  Same seeded pairs, same target, same starting point: the two must take
the same decisions, so they end on the same tau after the same number of evaluations, and the
oracle confirms that tau meets the target.
"""
import math

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import spamm as S
from oracle import tau as OT
from tests.gpu_helpers import dev

pytestmark = pytest.mark.gpu


def _pair(family, n, seed):
    if family == "exp":
        return synth.exp_decay_normal(n, 0.3, seed), synth.exp_decay_normal(n, 0.3, seed + 1)
    return synth.alg_decay_signed(n, 2.5, seed), synth.alg_decay_signed(n, 2.5, seed + 1)


def _oracle_error(a, b, leaf):
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    ab = OT.frobenius_from_normmap(nA) * OT.frobenius_from_normmap(nB)
    dense = S.dense_reference(a, b)

    def err(t):
        c = S.multiply_with_skipset(a, b, leaf, S.flat_survivors(nA, nB, t))
        return S.frobenius(c - dense) / ab
    return err, ab


@pytest.mark.parametrize("n,leaf,family,eps", [(512, 32, "exp", 1e-4), (640, 64, "alg", 1e-6),
                                               (1000, 64, "exp", 1e-7), (777, 32, "alg", 1e-3)])
def test_select_equals_oracle_bisection(n, leaf, family, eps):
    a, b = _pair(family, n, 2000 + n)
    err, ab = _oracle_error(a, b, leaf)
    tau_o, ev_o = OT.bisect_tau(err, eps, tau0=eps * ab)
    A, B = dev(a), dev(b)
    gA, gB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    plan = P.Plan(n, leaf, P.FP32)
    tau_ref, gab = plan.tau_certify(gA, gB)
    assert math.isclose(gab, ab, rel_tol=1e-12)
    tau_g, ev_g, e_g = plan.tau_select(gA, gB, A, B, eps)
    assert ev_g == ev_o, (ev_g, ev_o)
    assert tau_g == pytest.approx(tau_o, rel=1e-12, abs=0.0), (tau_g, tau_o)
    assert tau_o > 0.0
    e_true = err(tau_g)
    assert e_true <= eps                                    # the oracle confirms the answer
    assert abs(e_g - e_true) <= 1e-5 * e_true + 1e-11       # and the library's own measure
    # the bracket is tight: 1.01 x tau is not admissible (unless 40 evaluations ran out)
    if ev_o < 40:
        assert err(tau_g * 1.01) > eps or tau_g * 1.01 > tau_o * 1.0100001


def test_error_measure_against_oracle():
    """spamm_tau_error at several tau equals the oracle's exact pruning error (to the FP32 band
    product's accuracy plus the certified 1e-11)."""
    n, leaf = 600, 64
    a, b = _pair("exp", n, 77)
    err, ab = _oracle_error(a, b, leaf)
    A, B = dev(a), dev(b)
    gA, gB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    plan = P.Plan(n, leaf, P.FP32)
    tau_ref, _ = plan.tau_certify(gA, gB)
    assert err(tau_ref) <= 1e-11
    T = torch.empty_like(A)
    for rel in (1e-9, 1e-6, 1e-3, 1e-1):
        t = rel * ab
        e_g = plan.tau_error(gA, gB, A, B, t, tau_ref, T)
        e_o = err(t)
        assert abs(e_g - e_o) <= 1e-5 * e_o + 1e-11, (rel, e_g, e_o)
    assert plan.tau_error(gA, gB, A, B, 0.5 * tau_ref, tau_ref, T) == 0.0


def test_select_with_network_checks_then_falls_back():
    """With the trained network: a hit returns the predicted tau after one evaluation; a miss
    costs one evaluation more than plain bisection and returns the bisection's tau.  Either
    way the oracle confirms the target."""
    W = P.load_tau_weights()
    leaf = 64
    for n, family, eps in [(768, "exp", 1e-5), (640, "alg", 1e-4), (512, "exp", 1e-7)]:
        a, b = _pair(family, n, 3000 + n)
        err, ab = _oracle_error(a, b, leaf)
        A, B = dev(a), dev(b)
        gA, gB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
        plan = P.Plan(n, leaf, P.FP32)
        tau_n, ev_n, _ = plan.tau_select(gA, gB, A, B, eps, W)
        tau_b, ev_b, _ = plan.tau_select(gA, gB, A, B, eps)
        tau_p = plan.tau_predict(gA, gB, eps, W)
        if ev_n == 1:
            assert tau_n == tau_p
        else:
            assert ev_n == 1 + ev_b and tau_n == tau_b
        assert err(tau_n) <= eps
