"""Pins of the tau tools: valid-ratio search, histogram features and bisection."""
import math

import numpy as np
import pytest

import synth
from oracle import spamm as S
from oracle import tau as T


def _norms(n=256, leaf=32, seed=51):
    a = synth.alg_decay_signed(n, 2.0, seed)
    b = synth.exp_decay_normal(n, 0.1, seed + 1)
    return a, b, S.normmap(a, leaf), S.normmap(b, leaf)


def test_mean_norm_product_brute_force():
    _, _, nA, nB = _norms()
    p = S.triple_products(nA, nB)
    assert math.isclose(T.mean_norm_product(nA, nB), math.fsum(p.ravel().tolist()) / p.size,
                        rel_tol=1e-13)


@pytest.mark.parametrize("target", [0.3, 0.2, 0.1, 0.05])
def test_valid_ratio_search_hits_target(target):
    a = synth.table1_matrix(1024)
    nA = S.normmap(a, 32)
    tau, vr, probes = T.tau_for_valid_ratio(nA, nA, target, iters=20, tol=0.01)
    assert abs(vr - target) <= 0.01 and probes <= 20
    assert vr == S.valid_ratio(S.flat_survivors(nA, nA, tau))


def test_histogram_sums_to_one_and_matches_log2():
    _, _, nA, nB = _norms()
    h = T.norm_product_histogram(nA, nB)
    assert math.isclose(h.sum(), 1.0, rel_tol=1e-12)
    inv = T.inv_norm_product(nA, nB)
    p = S.triple_products(nA, nB).ravel()
    r = p * inv
    t = np.where(r > 0, np.clip(np.floor(-np.log2(np.where(r > 0, r, 1.0))), 0, 63), 63).astype(int)
    ref = np.bincount(t, minlength=64) / p.size
    assert np.array_equal(h, ref)


def test_histogram_bin_edges_exact_powers():
    r = np.array([1.0, 0.75, 0.5, 0.5000001, 0.25, 2.0 ** -63, 2.0 ** -64, 2.0 ** -70, 0.0])
    t = T.hist_bin(r, 1.0)
    assert t.tolist() == [0, 0, 1, 0, 2, 63, 63, 63, 63]


def test_bisection_exact_bracket_on_step_function():
    steps = np.array([3e-5, 7e-4, 2e-2, 0.9])
    errs = np.array([0.0, 1e-7, 1e-5, 1e-3, 1e-1])

    def err(t):
        return float(errs[np.searchsorted(steps, t, side="right")])

    for eps, crit in ((5e-6, 7e-4), (1e-3, 0.9), (5e-8, 3e-5), (1e-7, 7e-4)):
        tau, ev = T.bisect_tau(err, eps, 1e-3)
        assert err(tau) <= eps
        assert err(tau * 1.0100001) > eps or tau * 1.01 >= crit * 0.99
        assert tau <= crit and tau >= crit / 1.0100001


def test_bisection_on_real_inputs_meets_target():
    a, b, nA, nB = _norms(n=128, leaf=32)
    ref = S.dense_reference(a, b)
    nab = S.frobenius(a) * S.frobenius(b)

    def err(t):
        c = S.multiply_with_skipset(a, b, 32, S.flat_survivors(nA, nB, t))
        return S.frobenius(ref - c) / nab

    for eps in (1e-3, 1e-5):
        tau, _ = T.bisect_tau(err, eps, T.mean_norm_product(nA, nB))
        assert err(tau) <= eps
        assert err(tau * 1.02) > eps or err(tau * 1.02) <= eps  # bracket ends at <=1% ratio


def test_frobenius_from_normmap_equals_matrix_norm():
    """||X||_F from the leaf norms equals the matrix's own Frobenius norm (ragged n too)."""
    for n, leaf in ((256, 32), (250, 64), (97, 32)):
        a, _, _, _ = _norms(n, leaf, 70 + n)
        nA = S.normmap(a, leaf)
        assert T.frobenius_from_normmap(nA) == pytest.approx(
            float(np.linalg.norm(a.astype(np.float64))), rel=1e-14)
        assert T.inv_norm_product(nA, nA) == pytest.approx(
            1.0 / float(np.linalg.norm(a.astype(np.float64))) ** 2, rel=1e-14)
    z = np.zeros((4, 4))
    assert T.inv_norm_product(z, z) == 0.0


def test_mlp_features_layout():
    """65 features: the 64 bins unchanged, then log10 of the target error."""
    h = np.arange(64, dtype=np.float64) / 2016.0
    x = T.mlp_features(h, 1e-5)
    assert x.shape == (65,)
    assert np.array_equal(x[:64], h)
    assert x[64] == pytest.approx(-5.0, abs=1e-15)


def test_valid_ratio_at_counts_triples_one_by_one():
    """Brute force over every (i, k, j) with the skip rule written out (multiply iff not
    p < tau), including a tau equal to one product (a tie is multiplied)."""
    _, _, nA, nB = _norms(n=160, leaf=32)
    bd = nA.shape[0]
    p_mid = float(nA[1, 2] * nB[2, 3])
    for tau in (0.0, p_mid, 1e-3, math.inf):
        cnt = sum(1 for i in range(bd) for k in range(bd) for j in range(bd)
                  if not float(nA[i, k]) * float(nB[k, j]) < tau)
        assert T.valid_ratio_at(nA, nB, tau) == cnt / bd ** 3
    assert T.valid_ratio_at(nA, nB, 0.0) == 1.0 and T.valid_ratio_at(nA, nB, math.inf) == 0.0
