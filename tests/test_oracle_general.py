"""Pins of the general-form oracle: rectangular C = alpha*A*B + beta*C and chained powers."""
import math

import numpy as np
import pytest

import synth
from oracle import general as G
from oracle import spamm as S


def _rect(m, n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    r = np.arange(m)[:, None] * (n / m)
    c = np.arange(n)[None, :]
    return (np.exp(-0.2 * np.abs(r - c)) * g.standard_normal((m, n))).astype(np.float32)


def test_square_alpha_one_beta_zero_is_the_square_oracle():
    a = synth.alg_decay_signed(100, 2.0, 31)
    b = synth.exp_decay_normal(100, 0.1, 32)
    for tau in (0.0, 1e-3, 1e-1):
        g = G.spamm_general(a, b, 16, tau)
        s = S.spamm(a, b, 16, tau)
        assert np.array_equal(g["surv"], s["surv"])
        assert np.array_equal(g["C"], s["C"])
        assert g["bound2"] == pytest.approx(s["bound2"], rel=1e-15, abs=0)


def test_tau_zero_is_the_dense_general_product():
    """Every triple survives; the result is alpha*A@B + beta*C (library matmul), ragged
    edges in all three dimensions."""
    a, b = _rect(70, 45, 33), _rect(45, 33, 34)
    c_in = _rect(70, 33, 35)
    alpha, beta = -1.5, 0.25
    r = G.spamm_general(a, b, 16, 0.0, alpha, beta, c_in)
    assert r["S"] == 5 * 3 * 3 and r["bound2"] == 0.0
    ref = alpha * (a.astype(np.float64) @ b.astype(np.float64)) + beta * c_in.astype(np.float64)
    assert np.max(np.abs(r["C"] - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_tau_infinite_leaves_beta_c_and_beta_zero_reads_no_c():
    a, b = _rect(40, 24, 36), _rect(24, 56, 37)
    c_in = _rect(40, 56, 38)
    r = G.spamm_general(a, b, 8, math.inf, 2.0, -0.5, c_in)
    assert r["S"] == 0 and np.array_equal(r["C"], -0.5 * c_in.astype(np.float64))
    nan_c = np.full((40, 56), np.nan, dtype=np.float32)
    r = G.spamm_general(a, b, 8, 0.0, 1.0, 0.0, nan_c)
    assert np.isfinite(r["C"]).all()


def test_hand_enumerated_rectangular_case():
    """Leaf 2; A is 2 x 3 blocks, B is 3 x 1 blocks, each block constant +-2^e, so a block
    norm is exactly 2^(e+1) and every product is a power of two.  Products by hand:
    row 0: 2^2, 2^4, 2^3; row 1: 2^5, 2^2, 2^-1.  At tau = 8 the survivors are (0,1,0),
    (0,2,0) (a tie, multiplied) and (1,0,0)."""
    ea = np.array([[0, 1, 2], [3, -1, -2]])
    sa = np.array([[1, -1, 1], [-1, 1, 1]])
    eb = np.array([0, 1, -1])
    sb = np.array([1, 1, -1])
    a = np.kron(sa * np.ldexp(1.0, ea), np.ones((2, 2))).astype(np.float32)      # 4 x 6
    b = np.kron((sb * np.ldexp(1.0, eb))[:, None], np.ones((2, 2))).astype(np.float32)  # 6 x 2
    r = G.spamm_general(a, b, 2, 8.0)
    expect = np.zeros((2, 3, 1), dtype=bool)
    expect[0, 1, 0] = expect[0, 2, 0] = expect[1, 0, 0] = True
    assert np.array_equal(r["surv"], expect)
    # row-block 0: 2 * ((-2)(2) + (4)(-0.5)) = -12; row-block 1: 2 * ((-8)(1)) = -16
    assert np.array_equal(r["C"], np.array([[-12, -12]] * 2 + [[-16, -16]] * 2, dtype=float))
    # skipped: tile (0,0) 2^2; tile (1,0) 2^2 + 2^-1
    assert r["bound2"] == math.sqrt(16.0 + 4.5 ** 2)


@pytest.mark.parametrize("m,k,n,leaf", [(70, 45, 33, 16), (24, 90, 40, 8), (50, 50, 17, 16)])
def test_rectangular_flat_rule_equals_the_recursion(m, k, n, leaf):
    """Algorithm 1 on the zero-padded square embedding forms exactly the flat survivors."""
    a, b = _rect(m, k, m + k), _rect(k, n, k + n)
    nA, nB = G.normmap_rect(a, leaf), G.normmap_rect(b, leaf)
    p = np.sort((nA[:, :, None] * nB[None, :, :]).ravel())
    for tau in (0.0, float(p[p.size // 4]), float(p[p.size // 2]), float(p[-1])):
        flat = G.spamm_general(a, b, leaf, tau)
        c_rec, s_rec = G.spamm_general_recursive(a, b, leaf, tau)
        assert np.array_equal(flat["surv"], s_rec)
        assert np.max(np.abs(flat["C"] - c_rec), initial=0.0) <= 1e-13 * max(
            1.0, np.max(np.abs(c_rec), initial=0.0))


def test_rectangular_norms_and_pruning_bound():
    """Norms against a per-block numpy norm; the pruning error stays within bound2 and the
    bound is nested in tau."""
    a, b = _rect(70, 45, 41), _rect(45, 33, 42)
    nA = G.normmap_rect(a, 16)
    assert nA.shape == (5, 3)
    assert nA[4, 2] == pytest.approx(np.linalg.norm(a[64:70, 32:45].astype(np.float64)),
                                     rel=1e-15)
    exact = a.astype(np.float64) @ b.astype(np.float64)
    prev = -1.0
    for tau in (1e-3, 1e-2, 1e-1, 1.0):
        r = G.spamm_general(a, b, 16, tau)
        err = np.linalg.norm(exact - r["C"])
        assert err <= r["bound2"] * (1 + 1e-12) + 1e-12
        assert r["bound2"] >= prev
        prev = r["bound2"]


@pytest.mark.parametrize("squaring,steps,power", [(True, 3, 8), (False, 3, 4)])
def test_power_chain_at_tau_zero_is_the_matrix_power(squaring, steps, power):
    n = 48
    a = (0.5 * synth.exp_decay_normal(n, 0.3, 43) / 2.0).astype(np.float32)
    chain = G.power_chain(a, 16, 0.0, steps, squaring)
    ref = np.linalg.matrix_power(a.astype(np.float64), power)
    got = chain[-1]["X"].astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    assert all(step["S"] == 3 ** 3 for step in chain)


def test_power_chain_steps_are_spamm_of_the_stored_fp32_matrices():
    """Each step is the square oracle on the previous step's FP32 result; the step's error
    against the exact product of its inputs is within its skipped bound plus the FP32
    rounding of the stored result."""
    n, leaf, tau = 96, 16, 1e-3
    a = synth.exp_decay_normal(n, 0.5, 44)
    chain = G.power_chain(a, leaf, tau, 3)
    x = a.astype(np.float32)
    for step in chain:
        ref = S.spamm(x, x, leaf, tau)
        assert np.array_equal(step["norms"], S.normmap(x, leaf))
        assert np.array_equal(step["C"], ref["C"]) and step["S"] == ref["S"]
        assert np.array_equal(step["X"], ref["C"].astype(np.float32))
        exact = x.astype(np.float64) @ x.astype(np.float64)
        err = np.linalg.norm(step["X"].astype(np.float64) - exact)
        assert err <= ref["bound2"] + 2.0 ** -24 * np.linalg.norm(ref["C"]) * 1.01 + 1e-300
        x = step["X"]
