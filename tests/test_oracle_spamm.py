"""Pins of the FP64 oracle's norms, skip rule, recursion and bounds.

Each test checks the oracle against something other than itself: the
hand-enumerated skip sets of tests/golden/hand_tiny.json, Table 1 of the paper
(tests/golden/table1.json), closed forms for Toeplitz inputs, the dense
product at tau = 0, and the invariants the skip rule implies.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import spamm as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- P3: hand cases

def _hand_matrices():
    g = _load("hand_tiny.json")
    E = np.array(g["E"])
    a = synth.block_constant(E, np.array(g["sign_A"]), 2)
    b = synth.block_constant(E, np.array(g["sign_B"]), 2)
    return g, E, a, b


def test_hand_norms_are_exact_powers_of_two():
    g, E, a, b = _hand_matrices()
    nA = S.normmap(a, 2)
    assert np.array_equal(nA, np.exp2(E + 1.0))


@pytest.mark.parametrize("case", range(3))
def test_hand_skip_sets(case):
    g, E, a, b = _hand_matrices()
    c = g["cases"][case]
    tau = 2.0 ** c["tau_log2"]
    res = S.spamm(a, b, 2, tau)
    expect = np.zeros((4, 4, 4), dtype=bool)
    for key, ks in c["survivors"].items():
        i, j = map(int, key.split(","))
        for k in ks:
            expect[i, k, j] = True
    assert np.array_equal(res["surv"], expect)
    assert res["S"] == c["S"]
    # the same set by integer arithmetic on the exponents: E_ik + E_kj + 2 >= log2 tau
    ints = (E[:, :, None] + E[None, :, :] + 2) >= c["tau_log2"]
    assert np.array_equal(res["surv"], ints)
    # C from the closed form: a 2x2 constant block product is 2 * ca * cb * ones
    sa, sb = np.array(g["sign_A"]), np.array(g["sign_B"])
    cexp = np.zeros((8, 8))
    for i in range(4):
        for j in range(4):
            v = sum(2.0 * sa[i, k] * sb[k, j] * 2.0 ** (E[i, k] + E[k, j])
                    for k in range(4) if expect[i, k, j])
            cexp[2 * i:2 * i + 2, 2 * j:2 * j + 2] = v
    assert np.array_equal(res["C"], cexp)
    # the recursion reaches the same set and the same C
    crec, srec = S.spamm_recursive(a, b, 2, tau)
    assert np.array_equal(srec, expect)
    assert np.array_equal(crec, cexp)


def test_nan_block_survives_and_zero_block_at_tau0():
    g, E, a, b = _hand_matrices()
    a = a.copy()
    a[0:2, 4:6] = np.nan                      # block (0, 2) of A
    res = S.spamm(a, b, 2, 1.0)
    assert res["surv"][0, 2, :].all()          # NaN product is never skipped
    assert np.isnan(res["C"][0:2]).any()
    z = a.copy()
    z[:] = 0
    res0 = S.spamm(z, b, 2, 0.0)
    assert res0["S"] == 64                     # 0 >= 0: everything survives at tau = 0
    assert not res0["C"].any()


def test_padding_n7_equals_zero_extended_n8():
    g, E, a, b = _hand_matrices()
    a7, b7 = a[:7, :7].copy(), b[:7, :7].copy()
    a8, b8 = np.zeros((8, 8), np.float32), np.zeros((8, 8), np.float32)
    a8[:7, :7], b8[:7, :7] = a7, b7
    for tau in (0.0, 0.5, 1.0, 2.0, 4.0):
        r7, r8 = S.spamm(a7, b7, 2, tau), S.spamm(a8, b8, 2, tau)
        assert np.array_equal(r7["surv"], r8["surv"])
        assert np.array_equal(r7["C"], r8["C"][:7, :7])
        c7, s7 = S.spamm_recursive(a7, b7, 2, tau)
        assert np.array_equal(s7, r7["surv"]) and np.array_equal(c7, r7["C"])


# ---------------------------------------------------------------- P5: closed-form norms

def _toeplitz_asym(n):
    """a_ij = f(i - j): (d+1)^-3 below/on the diagonal, 2 (|d|+1)^-3 above (asymmetric)."""
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    d = i - j
    return np.where(d >= 0, (np.abs(d) + 1.0) ** -3, 2.0 * (np.abs(d) + 1.0) ** -3).astype(np.float32)


def _f32_of_offset(d):
    d = np.asarray(d)
    return np.where(d >= 0, (np.abs(d) + 1.0) ** -3, 2.0 * (np.abs(d) + 1.0) ** -3).astype(np.float32)


@pytest.mark.parametrize("n,leaf", [(256, 32), (200, 32), (130, 64)])
def test_norms_closed_form_diagonal_multiplicity(n, leaf):
    """||A[I,K]||^2 = sum over diagonals m of (number of (p,q) on it) * f(offset)^2."""
    a = _toeplitz_asym(n)
    nA = S.normmap(a, leaf)
    bd = S.num_blocks(n, leaf)
    for I in range(bd):
        for K in range(bd):
            rows = np.arange(I * leaf, min(n, (I + 1) * leaf))
            cols = np.arange(K * leaf, min(n, (K + 1) * leaf))
            # entries with i - j = d: count pairs (r, c) in the block with r - c = d
            total = 0.0
            for d in range(rows[0] - cols[-1], rows[-1] - cols[0] + 1):
                lo = max(rows[0], cols[0] + d)
                hi = min(rows[-1], cols[-1] + d)
                cnt = max(0, hi - lo + 1)
                v = float(_f32_of_offset(d))
                total += cnt * v * v
            assert math.isclose(nA[I, K], math.sqrt(total), rel_tol=1e-14)
    # asymmetry is visible: a transposed block index would fail
    assert not np.allclose(nA, nA.T)


# ---------------------------------------------------------------- P1, P2

@pytest.mark.parametrize("n,leaf", [(256, 32), (200, 32), (96, 32)])
def test_tau0_is_dense_product(n, leaf):
    a = synth.exp_decay_su(n, 0.5, 11)
    b = synth.exp_decay_su(n, 0.3, 12)
    res = S.spamm(a, b, leaf, 0.0)
    bd = S.num_blocks(n, leaf)
    assert res["S"] == bd ** 3
    ref = S.dense_reference(a, b)
    assert S.frobenius(res["C"] - ref) <= 1e-13 * S.frobenius(ref)
    crec, srec = S.spamm_recursive(a, b, leaf, 0.0)
    assert srec.all()
    assert S.frobenius(crec - ref) <= 1e-13 * S.frobenius(ref)


def test_tau_inf_and_above_max():
    a = synth.exp_decay_su(128, 0.5, 13)
    b = synth.exp_decay_su(128, 0.5, 14)
    for tau in (math.inf, 1e30):
        res = S.spamm(a, b, 32, tau)
        assert res["S"] == 0 and not res["C"].any()
    nA, nB = S.normmap(a, 32), S.normmap(b, 32)
    pmax = float(S.triple_products(nA, nB).max())
    res = S.spamm(a, b, 32, np.nextafter(pmax, np.inf))
    assert res["S"] == 0
    res = S.spamm(a, b, 32, pmax)                  # tie at the maximum survives
    assert res["S"] >= 1


# ---------------------------------------------------------------- P6: invariants

@pytest.mark.parametrize("n,leaf,seed", [(256, 32, 21), (224, 32, 22), (32, 32, 23), (64, 16, 24)])
def test_recursive_equals_flat_and_invariants(n, leaf, seed):
    a = synth.exp_decay_su(n, 0.4, seed)
    b = synth.alg_decay_signed(n, 2.5, seed + 1)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    ref = S.dense_reference(a, b)
    p = S.triple_products(nA, nB)
    taus = [0.0] + sorted(set(np.quantile(p, [0.1, 0.3, 0.5, 0.7, 0.9, 0.99]).tolist())) + [math.inf]
    prev = None
    for tau in taus:
        res = S.spamm(a, b, leaf, tau)
        crec, srec = S.spamm_recursive(a, b, leaf, tau)
        assert np.array_equal(srec, res["surv"])
        assert S.frobenius(crec - res["C"]) <= 1e-13 * max(1e-300, S.frobenius(ref))
        err = S.frobenius(ref - res["C"])
        assert err <= res["bound2"] * (1 + 1e-12) + 1e-13 * S.frobenius(ref)
        assert res["bound2"] <= res["bound1"] * (1 + 1e-15)
        if prev is not None:
            assert not (res["surv"] & ~prev["surv"]).any()     # nested skip sets
            assert res["S"] <= prev["S"]
            assert res["bound1"] >= prev["bound1"] and res["bound2"] >= prev["bound2"]
        prev = res
    # V matrix: per-tile counts add up to S
    assert S.valid_counts(prev["surv"]).sum() == prev["S"]


def test_error_monotone_on_decade_grid_c1_shape():
    """On the c1 matrix family the error grows with tau over a decade grid (empirical, reading)."""
    a = synth.exp_decay_su(256, 0.5, 31)
    ref = S.dense_reference(a, a)
    errs = []
    for tau in (0.0, 1e-8, 1e-6, 1e-4, 1e-2, 1e0):
        res = S.spamm(a, a, 32, tau)
        errs.append(S.frobenius(ref - res["C"]))
    assert all(e2 >= e1 - 1e-15 for e1, e2 in zip(errs, errs[1:]))


def test_c1_block_tridiagonal_skip_set():
    """N=1024, exp(-0.5|i-j|) s u, leaf 32, tau 1e-4 and 1e-2 keep exactly the block tridiagonal.

    Off-diagonal blocks at distance >= 2 have entries below exp(-0.5*33) ~ 7e-8,
    so their norms (< 32 * 7e-8) times any norm (< 32) stay below 1e-4; the
    diagonal and first off-diagonal blocks are far above 1e-2.  Survivors are
    the (i,k,j) with |i-k| <= 1 and |k-j| <= 1: 30*9 + 2*4... counted below.
    """
    a, b = synth.workload_c1()
    nA = S.normmap(a, 32)
    bd = 32
    expect = np.zeros((bd, bd, bd), dtype=bool)
    for i in range(bd):
        for k in range(max(0, i - 1), min(bd, i + 2)):
            for j in range(max(0, k - 1), min(bd, k + 2)):
                expect[i, k, j] = True
    for tau in (1e-4, 1e-2):
        surv = S.flat_survivors(nA, nA, tau)
        assert np.array_equal(surv, expect)
    # count: sum over k of (#i adjacent to k) * (#j adjacent to k) = 2*2*2 + 30*3*3
    assert expect.sum() == 2 * 4 + 30 * 9 == 278


# ---------------------------------------------------------------- P4: Table 1

def _table1_offset_norms(n, leaf):
    """Leaf norms g(d) of the Table 1 matrix as a function of the block offset d = K - I."""
    bd = n // leaf
    g = np.zeros(2 * bd - 1)
    m = np.arange(-(leaf - 1), leaf)
    mult = (leaf - np.abs(m)).astype(np.float64)
    for idx, d in enumerate(range(-(bd - 1), bd)):
        dist = np.abs(d * leaf + m).astype(np.float64)
        v = (0.1 / (dist ** 0.1 + 1.0)).astype(np.float32).astype(np.float64)
        g[idx] = math.sqrt(math.fsum((mult * v * v).tolist()))
    return g


def _table1_ratio_closed_form(n, leaf, tau):
    """Valid ratio by counting index triples per offset pair (d1 = k - i, d2 = j - k)."""
    bd = n // leaf
    g = _table1_offset_norms(n, leaf)
    d = np.arange(-(bd - 1), bd)
    d1, d2 = d[:, None], d[None, :]
    lo = np.maximum(0, np.maximum(-d1, -d1 - d2))
    hi = np.minimum(bd - 1, np.minimum(bd - 1 - d1, bd - 1 - d1 - d2))
    cnt = np.maximum(0, hi - lo + 1)
    surv = ~((g[:, None] * g[None, :]) < tau)
    return float((cnt * surv).sum()) / bd ** 3


def test_table1_closed_form_all_sizes():
    t = _load("table1.json")
    tol = t["tolerance_pp"] / 100.0
    for label, taus in t["rows"].items():
        for n, tau in zip(t["n"], taus):
            vr = _table1_ratio_closed_form(n, 32, tau)
            assert abs(vr - float(label)) <= tol, (n, label, vr)


def test_table1_leaf_reading_rejects_16_and_64():
    t = _load("table1.json")
    tau = t["rows"]["0.10"][0]
    assert _table1_ratio_closed_form(1024, 16, tau) < 0.01
    assert _table1_ratio_closed_form(1024, 64, tau) > 0.99


@pytest.mark.parametrize("n", [1024, 2048])
def test_table1_oracle_path(n):
    """The oracle's own normmap + flat enumeration reproduce Table 1 at N = 1024, 2048."""
    t = _load("table1.json")
    a = synth.table1_matrix(n)
    nA = S.normmap(a, 32)
    col = t["n"].index(n)
    # offset-norm closed form agrees with the oracle normmap
    g = _table1_offset_norms(n, 32)
    bd = n // 32
    for I in (0, bd // 2, bd - 1):
        for K in range(bd):
            assert math.isclose(nA[I, K], g[K - I + bd - 1], rel_tol=1e-14)
    for label, taus in t["rows"].items():
        vr = S.valid_ratio(S.flat_survivors(nA, nA, taus[col]))
        assert abs(vr - float(label)) <= t["tolerance_pp"] / 100.0


# ------------------------------------------------ row-sampled forms and errors

@pytest.mark.parametrize("n,leaf,rows", [(300, 32, [0, 4, 9]), (257, 64, [0, 3, 4]),
                                         (128, 32, [1, 2])])
def test_row_sampled_forms_equal_full_oracle(n, leaf, rows):
    """normmap_rows / spamm_rows (the CPU baseline's bounded sample) equal the matching rows of
    the full norm map, flat survivor set and product, including ragged last block-rows."""
    a = synth.exp_decay_su(n, 0.3, 11 + n)
    b = synth.alg_decay_signed(n, 2.0, 12 + n)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    nA_rows = S.normmap_rows(a, leaf, rows)
    assert np.array_equal(nA_rows, nA[rows])
    p = S.triple_products(nA, nB)
    tau = float(np.quantile(p[p > 0], 0.6))
    full = S.spamm(a, b, leaf, tau)
    surv_full = S.flat_survivors(nA, nB, tau)
    part = S.spamm_rows(a, b, leaf, tau, rows, nA_rows, nB)
    for i in rows:
        strip, surv = part[i]
        lo, hi = i * leaf, min(n, (i + 1) * leaf)
        assert np.array_equal(surv, surv_full[i])
        ref = full["C"][lo:hi]
        assert np.max(np.abs(strip - ref)) <= 1e-13 * max(np.max(np.abs(ref)), 1e-300)


def test_errors_three_normalisations():
    """Eq. 5 errors: a known perturbation gives ||E||_F in absolute and both relative forms."""
    ref = np.diag([3.0, 4.0])
    c = ref.copy()
    c[0, 1] = 1e-3                       # E = ref - c has one entry of magnitude 1e-3
    e = S.errors(c, ref, 2.0, 5.0)
    assert e["abs"] == pytest.approx(1e-3, rel=1e-15)
    assert e["rel_c"] == pytest.approx(1e-3 / 5.0, rel=1e-15)    # ||ref||_F = 5
    assert e["rel_ab"] == pytest.approx(1e-3 / 10.0, rel=1e-15)
    z = S.errors(ref, ref, 0.0, 0.0)
    assert z["abs"] == 0.0 and z["rel_c"] == 0.0 and z["rel_ab"] == 0.0


def test_needed_b_rows_give_the_same_sampled_rows():
    """spamm_rows with B's norm map restricted to the needed block rows equals spamm_rows with
    the full map (decisions and values), on a decay pair whose far blocks are exactly zero."""
    n, leaf = 600, 32
    a = synth.exp_decay_normal(n, 2.0, 31)    # |i-j| beyond ~60 underflows to exact zeros
    b = synth.exp_decay_normal(n, 2.0, 32)
    bd = S.num_blocks(n, leaf)
    rows = [0, 7, bd - 1]
    nA_rows = S.normmap_rows(a, leaf, rows)
    full = S.normmap(b, leaf)
    for tau in (1e-30, 1e-6):
        part = S.normmap_needed(b, leaf, nA_rows, tau)
        ks = S.needed_b_rows(nA_rows, tau)
        assert 0 < ks.size < bd
        assert np.array_equal(part[ks], full[ks])
        r_full = S.spamm_rows(a, b, leaf, tau, rows, nA_rows, full)
        r_part = S.spamm_rows(a, b, leaf, tau, rows, nA_rows, part)
        for i in rows:
            assert np.array_equal(r_full[i][0], r_part[i][0])
            assert np.array_equal(r_full[i][1], r_part[i][1])
    # tau = 0 needs every row (a zero block survives at tau = 0)
    assert S.needed_b_rows(nA_rows, 0.0).size == bd


def test_blocked_norms_agree_with_exactly_rounded_norms():
    """normmap_blocked (numpy pairwise FP64 sums) within 1e-14 relative of normmap (math.fsum,
    exactly rounded) on wide-range, ragged and exactly-zero blocks; zero blocks stay 0."""
    g = np.random.Generator(np.random.PCG64(404))
    x = (g.standard_normal((333, 333)) * np.exp2(g.integers(-60, 60, (333, 333)))).astype(np.float32)
    x[:64, 100:200] = 0.0
    for leaf in (32, 64, 128):
        exact = S.normmap(x, leaf)
        fast = S.normmap_blocked(x, leaf)
        assert np.array_equal(exact == 0, fast == 0)
        nz = exact > 0
        assert np.max(np.abs(fast[nz] - exact[nz]) / exact[nz]) <= 1e-14
    y = synth.near_sparse(300, 405)
    assert np.max(np.abs(S.normmap_blocked(y, 64) / S.normmap(y, 64) - 1.0)) <= 1e-14
