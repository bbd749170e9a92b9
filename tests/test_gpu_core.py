"""GPU parity of the norm map, the pair test / work queues and the FP32 multiply.

Every expected value comes from the CPU oracle on the same seeded inputs.
"""
import math

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import precision as OP
from oracle import spamm as S
from oracle import tau as OT
from tests.gpu_helpers import band_ok, dev, host, plan_mask

pytestmark = pytest.mark.gpu

NORM_REL_TOL = 3e-13       # the normmap's stated accuracy
FP32_REL_TOL = 1e-5        # FP32 path vs FP64 oracle, relative Frobenius


def _pair(family, n, seed):
    if family == "exp":
        return synth.exp_decay_su(n, 0.5, seed), synth.exp_decay_su(n, 0.5, seed + 1)
    if family == "alg":
        return synth.alg_decay_signed(n, 3.0, seed), synth.alg_decay_signed(n, 3.0, seed + 1)
    if family == "sparse":
        return synth.near_sparse(n, seed), synth.near_sparse(n, seed + 1)
    if family == "normal":
        return synth.exp_decay_normal(n, 0.05, seed), synth.exp_decay_normal(n, 0.05, seed + 1)
    raise ValueError(family)


# --------------------------------------------------------------------------- norm map

@pytest.mark.parametrize("n,leaf,family", [
    (1024, 32, "exp"), (200, 32, "alg"), (1001, 32, "normal"), (1000, 64, "sparse"),
    (640, 128, "alg"), (130, 128, "normal"), (777, 64, "exp"), (64, 64, "normal"),
])
def test_normmap_parity(n, leaf, family):
    a, _ = _pair(family, n, 100 + n)
    got = host(P.spamm_normmap(dev(a), leaf))
    ref = S.normmap(a, leaf)
    assert got.shape == ref.shape
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero])
    rel = np.abs(got[~zero] - ref[~zero]) / ref[~zero]
    assert rel.max(initial=0.0) <= NORM_REL_TOL


def test_normmap_special_values():
    a = synth.exp_decay_normal(256, 0.1, 7)
    a[0:3, 70:72] = np.nan                 # block (0, 1) at leaf 64
    a[100, 200] = np.inf                   # block (1, 3)
    a[128:192, 0:64] = 0.0                 # block (2, 0)
    got = host(P.spamm_normmap(dev(a), 64))
    assert np.isnan(got[0, 1])
    assert not np.isfinite(got[1, 3])
    assert got[2, 0] == 0.0
    ref = S.normmap(a, 64)
    fin = np.isfinite(ref)
    assert np.allclose(got[fin], ref[fin], rtol=NORM_REL_TOL, atol=0)


@pytest.mark.parametrize("leaf", [32, 64, 128])
def test_normmap_wide_dynamic_range(leaf):
    """Entries spread over 2^-100 .. 2^20 (log-uniform, random signs), blocks dominated by one
    entry, and blocks of tiny entries only: the exact-square sums keep the 3e-13 accuracy."""
    g = np.random.default_rng(leaf)
    n = 4 * leaf + 3
    a = (np.exp2(g.uniform(-100, 20, size=(n, n))) * g.choice([-1.0, 1.0], size=(n, n))).astype(np.float32)
    a[:leaf, :leaf] = np.float32(1e-30)            # tiny entries only
    a[0, 0] = np.float32(3.0e5)                     # then one dominant entry elsewhere
    a[leaf:2 * leaf, leaf:2 * leaf] *= np.float32(1e-12)
    a[leaf + 1, leaf + 2] = np.float32(7.0e9)
    got = host(P.spamm_normmap(dev(a), leaf))
    ref = S.normmap(a, leaf)
    rel = np.abs(got - ref) / ref
    assert rel.max() <= NORM_REL_TOL, rel.max()


@pytest.mark.parametrize("n,leaf,shift", [(1, 32, 0), (2, 32, 4), (3, 32, 12), (5, 32, 28),
                                           (7, 64, 4), (33, 32, 20), (130, 128, 4), (131, 128, 8),
                                           (1001, 64, 12), (1027, 64, 28), (2049, 128, 4),
                                           (1024, 32, 4), (1028, 64, 8)])
def test_normmap_offset_views(n, leaf, shift):
    """X 16-byte aligned but not on a 128-byte line (a view `shift` floats into a buffer), tiny
    and ragged n: the staged copies are clipped to X's first byte and last 16-byte boundary."""
    a, _ = _pair("normal", n, 900 + n)
    buf = torch.full((n * n + 64,), float("nan"), dtype=torch.float32, device="cuda")
    X = buf[shift:shift + n * n].view(n, n)
    X.copy_(torch.from_numpy(a).cuda())
    assert X.data_ptr() % 16 == 0
    got = host(P.spamm_normmap(X, leaf))
    ref = S.normmap(a, leaf)
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero])
    assert np.max(np.abs(got[~zero] - ref[~zero]) / ref[~zero], initial=0.0) <= NORM_REL_TOL
    assert P.spamm_last_device_status() == 0


def test_normmap_c2_full_size():
    a, _ = synth.workload_c2()
    got = host(P.spamm_normmap(dev(a), 64))
    ref = S.normmap(a, 64)
    assert np.max(np.abs(got - ref) / ref) <= NORM_REL_TOL


# --------------------------------------------------------------------------- plan

def _plan(nA_dev, nB_dev, n, leaf, tau, precision=P.FP32, target=1e-5):
    return P.Plan(n, leaf, precision).plan(nA_dev, nB_dev, tau, target)


@pytest.mark.parametrize("n,leaf,family", [(1024, 32, "exp"), (1000, 64, "alg"),
                                           (512, 32, "sparse"), (640, 128, "normal")])
def test_plan_exact_on_oracle_norms(n, leaf, family):
    """Fed the oracle's norm maps, the pair test is exactly the FP64 test (no band)."""
    a, b = _pair(family, n, 200 + n)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = S.triple_products(nA, nB)
    pos = p[p > 0]
    taus = [0.0, math.inf] + [float(np.quantile(pos, q)) for q in (0.01, 0.3, 0.7, 0.95, 0.999)]
    taus += [float(pos.max()), float(np.median(pos))]          # exact ties with products
    for tau in taus:
        plan = _plan(dev(nA), dev(nB), n, leaf, tau)
        surv, _ = plan_mask(plan)
        ref = S.flat_survivors(nA, nB, tau)
        assert np.array_equal(surv, ref), tau
        st = plan.stats()
        assert st["survivors"] == int(ref.sum())
        assert st["valid_ratio"] == S.valid_ratio(ref)
        V = S.valid_counts(ref)
        assert st["max_tile_survivors"] == int(V.max())
        assert st["nonempty_tiles"] == int((V > 0).sum())
        b1, b2 = S.skipped_bounds(nA, nB, ref)
        assert math.isclose(st["skipped_bound1"], b1, rel_tol=1e-5, abs_tol=1e-300)
        assert math.isclose(st["skipped_bound2"], b2, rel_tol=1e-5, abs_tol=1e-300)
        assert math.isclose(st["norm_a"], OT.frobenius_from_normmap(nA), rel_tol=1e-14)


@pytest.mark.parametrize("n,leaf,prec", [(16384, 32, P.FP32), (31000, 64, P.BF16_SPLIT)])
def test_plan_large_grid_counts(n, leaf, prec):
    """bd = 512 / 485: the pair-test kernel stages 12 * bd screens of shared memory, which with
    its static shared memory passes the default 48 KB limit; survivors per tile against numpy
    on the same maps."""
    bd = P.num_blocks(n, leaf)
    rng = np.random.default_rng(500)
    nA = rng.lognormal(0.0, 2.0, size=(bd, bd))
    nB = rng.lognormal(0.0, 2.0, size=(bd, bd))
    tau = float(np.exp(3.0))
    plan = P.Plan(n, leaf, prec).plan(dev(nA), dev(nB), tau, 1e-5)
    tp, kk = plan.export()
    got = np.diff(tp.astype(np.int64)).reshape(bd, bd)
    ref = np.empty((bd, bd), dtype=np.int64)
    for i in range(bd):
        ref[i] = (nA[i, :, None] * nB >= tau).sum(axis=0)   # sum over k of the tile (i, j)
    assert np.array_equal(got, ref)
    assert plan.stats()["survivors"] == int(ref.sum())


def test_plan_hand_ties_scaled():
    """Hand skip sets of tests/golden/hand_tiny.json at leaf 32: norms are 2^(E+5) exactly."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_tiny.json")))
    E = np.array(g["E"])
    a = synth.block_constant(E, np.array(g["sign_A"]), 32)
    b = synth.block_constant(E, np.array(g["sign_B"]), 32)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, 32), P.spamm_normmap(B, 32)
    assert np.array_equal(host(nA), np.exp2(E + 5.0))
    for case in g["cases"]:
        tau = 2.0 ** (case["tau_log2"] + 8)        # products scale by 2^(5+5-2)
        plan = _plan(nA, nB, 128, 32, tau)
        surv, _ = plan_mask(plan)
        expect = np.zeros((4, 4, 4), dtype=bool)
        for key, ks in case["survivors"].items():
            i, j = map(int, key.split(","))
            expect[i, ks, j] = True
        assert np.array_equal(surv, expect)
        C = host(plan.multiply(A, B, torch.empty_like(A)))
        assert np.array_equal(C.astype(np.float64), S.multiply_with_skipset(a, b, 32, expect))


@pytest.mark.parametrize("n,leaf,family", [(1024, 32, "exp"), (777, 64, "normal"),
                                           (512, 64, "sparse")])
def test_plan_on_gpu_norms_band(n, leaf, family):
    """End to end from the GPU norm maps: disagreements only inside the 1e-12 tau band."""
    a, b = _pair(family, n, 300 + n)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = S.triple_products(nA, nB)
    gA, gB = P.spamm_normmap(dev(a), leaf), P.spamm_normmap(dev(b), leaf)
    for tau in [float(np.quantile(p[p > 0], q)) for q in (0.2, 0.5, 0.9)] + [float(p.max())]:
        surv, _ = plan_mask(_plan(gA, gB, n, leaf, tau))
        assert band_ok(surv, S.flat_survivors(nA, nB, tau), p, tau)


def test_plan_order_and_offsets():
    a, b = _pair("alg", 1024, 401)
    nA, nB = S.normmap(a, 32), S.normmap(b, 32)
    plan = _plan(dev(nA), dev(nB), 1024, 32, 1e-6)
    tp, kk = plan.export()
    cnt = np.diff(tp)
    assert tp[0] == 0 and np.all(cnt >= 0)
    assert np.array_equal(cnt, S.valid_counts(S.flat_survivors(nA, nB, 1e-6)).ravel())


# --------------------------------------------------------------------------- FP32 multiply

def _fp32_case(a, b, leaf, tau):
    A, B = dev(a), dev(b)
    C, plan = P.spamm(A, B, leaf, tau)
    surv, _ = plan_mask(plan)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    ref = S.multiply_with_skipset(a, b, leaf, surv)
    got = host(C).astype(np.float64)
    err = S.frobenius(got - ref)
    scale = S.frobenius(ref)
    assert err <= FP32_REL_TOL * scale + 1e-30
    assert err <= OP.accumulation_bound(nA, nB, surv, OP.FP32, leaf) + 1e-30
    # tile by tile: each output tile within its own share of the accumulation bound (a tile
    # written wrongly or in the wrong place fails here even when it is tiny next to ||C||_F;
    # tiles without survivors must be exact zeros)
    t = OP.accumulation_tile_bounds(nA, nB, surv, OP.FP32, leaf)
    assert np.all(OP.tile_errors(got, ref, leaf) <= t), "a tile exceeds its own bound"
    return got, ref, surv


@pytest.mark.parametrize("tau", [0.0, 1e-4, 1e-2])
def test_multiply_fp32_c1(tau):
    a, b = synth.workload_c1()
    got, ref, surv = _fp32_case(a, b, 32, tau)
    if tau > 0:
        assert surv.sum() == 278          # block tridiagonal, as the oracle pins
    if tau == 0.0:
        dense = S.dense_reference(a, b)
        assert S.frobenius(got - dense) <= FP32_REL_TOL * S.frobenius(dense)


@pytest.mark.parametrize("n,leaf,family,q", [(1000, 64, "alg", 0.5), (1001, 32, "normal", 0.3),
                                             (640, 128, "sparse", 0.5), (130, 64, "exp", 0.0),
                                             (96, 32, "normal", 0.9)])
def test_multiply_fp32_ragged(n, leaf, family, q):
    a, b = _pair(family, n, 500 + n)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = S.triple_products(nA, nB)
    tau = float(np.quantile(p, q)) if q > 0 else 0.0
    _fp32_case(a, b, leaf, tau)


def test_multiply_all_skipped_writes_zeros():
    a, b = _pair("alg", 300, 601)
    A, B = dev(a), dev(b)
    C = torch.full_like(A, 7.0)
    nA, nB = P.spamm_normmap(A, 64), P.spamm_normmap(B, 64)
    plan = _plan(nA, nB, 300, 64, math.inf)
    plan.multiply(A, B, C)
    assert plan.stats()["survivors"] == 0
    assert not host(C).any()


def test_multiply_fp32_c2_full_size_sampled():
    """N = 8192, leaf 64, tau = 1e-4: skip set vs oracle, C on sampled tiles vs FP64."""
    a, b = synth.workload_c2()
    leaf, tau = 64, 1e-4
    A, B = dev(a), dev(b)
    C, plan = P.spamm(A, B, leaf, tau)
    surv, _ = plan_mask(plan)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p_fn = lambda: S.triple_products(nA, nB)
    assert band_ok(surv, S.flat_survivors(nA, nB, tau), p_fn(), tau)
    got = host(C)
    pa, pb = S.padded64(a, leaf), S.padded64(b, leaf)
    g = np.random.Generator(np.random.PCG64(9))
    bd = plan.bd
    tiles = [(i, i) for i in range(0, bd, 16)] + [tuple(g.integers(0, bd, 2)) for _ in range(24)]
    tiles += [(i, min(bd - 1, i + 1)) for i in range(0, bd, 32)]
    for i, j in tiles:
        ref = np.zeros((leaf, leaf))
        for k in np.nonzero(surv[i, :, j])[0]:
            ref += S.block(pa, leaf, i, k) @ S.block(pb, leaf, k, j)
        blk = got[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf].astype(np.float64)
        nr = S.frobenius(ref)
        assert S.frobenius(blk - ref) <= FP32_REL_TOL * max(nr, 1e-300) or (nr == 0 and not blk.any())


# --------------------------------------------------------------------------- reductions

def test_frobenius_diff():
    g = np.random.Generator(np.random.PCG64(11))
    x = g.standard_normal(1_000_003).astype(np.float32)
    y = (x + 1e-3 * g.standard_normal(x.size)).astype(np.float32)
    X, Y = dev(x), dev(y)
    d = P.spamm_frobenius_diff(X, Y)
    ref = S.frobenius(x.astype(np.float64) - y.astype(np.float64))
    assert math.isclose(d, ref, rel_tol=1e-12)
    assert math.isclose(P.spamm_frobenius_diff(X), S.frobenius(x), rel_tol=1e-12)
    assert P.spamm_last_device_status() == 0


@pytest.mark.parametrize("n,leaf", [(8192, 64), (1001, 32), (2048, 128)])
def test_normmap_pair_equals_two_calls(n, leaf):
    """One launch over both operands gives the bits of two single-operand launches."""
    a = synth.exp_decay_normal(n, 0.05, 701)
    b = synth.alg_decay_signed(n, 2.5, 702)
    A, B = dev(a), dev(b)
    pA, pB = P.spamm_normmap_pair(A, B, leaf)
    sA, sB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    torch.cuda.synchronize()
    assert torch.equal(pA, sA) and torch.equal(pB, sB)
    assert P.spamm_last_device_status() == 0
