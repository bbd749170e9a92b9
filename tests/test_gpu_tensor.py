"""GPU parity of the tcgen05 multiply in every reduced-precision mode.

For each mode the GPU result is compared with the oracle's FP64 evaluation of
the same rounded operands (power-of-two block scaling, RNE rounding, hi+lo
splits) on the GPU's skip set and split flags: the difference must stay inside
the FP32-accumulation bound.  Against the exact product the error must stay
inside the mode's a-priori bound.  Split flags are checked against the
oracle's dominant-triple rule.
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
from tests.gpu_helpers import dev, host, plan_mask

pytestmark = pytest.mark.gpu

MODES = [("bf16", OP.BF16), ("fp16", OP.FP16), ("bf16_split", OP.BF16_SPLIT),
         ("fp16_split", OP.FP16_SPLIT), ("tf32x3", OP.TF32X3)]


def _pair(family, n, seed):
    if family == "alg":
        return synth.alg_decay_signed(n, 2.5, seed), synth.alg_decay_signed(n, 2.5, seed + 1)
    if family == "exp":
        return synth.exp_decay_normal(n, 0.02, seed), synth.exp_decay_normal(n, 0.02, seed + 1)
    if family == "sparse":
        return synth.near_sparse(n, seed), synth.near_sparse(n, seed + 1)
    raise ValueError(family)


def _run(a, b, leaf, tau, mode, target):
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    plan = P.Plan(a.shape[0], leaf, mode).plan(nA, nB, tau, target)
    C = torch.full_like(A, float("nan"))
    plan.multiply(A, B, C)
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    surv, flags = plan_mask(plan)
    return host(C).astype(np.float64), surv, flags, plan.stats(), host(nA), host(nB)


@pytest.mark.parametrize("name,mode", MODES)
@pytest.mark.parametrize("n,leaf,family,q", [(1000, 64, "alg", 0.6), (640, 128, "exp", 0.3),
                                             (512, 64, "sparse", 0.5), (200, 128, "alg", 0.0)])
def test_tc_matches_emulation(name, mode, n, leaf, family, q):
    a, b = _pair(family, n, 900 + n + leaf)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = S.triple_products(nA, nB)
    tau = float(np.quantile(p[p > 0], q)) if q > 0 else 0.0
    got, surv, flags, st, gA, gB = _run(a, b, leaf, tau, mode, 1e-6)
    assert np.isfinite(got).all()
    emu = OP.emulated_multiply(a, b, leaf, surv, mode, flags)
    acc_bound = OP.accumulation_bound(nA, nB, surv, mode, leaf)
    assert S.frobenius(got - emu) <= acc_bound + 1e-30, (S.frobenius(got - emu), acc_bound)
    exact = S.multiply_with_skipset(a, b, leaf, surv)
    fl = flags if mode in (OP.BF16_SPLIT, OP.FP16_SPLIT) else None
    assert S.frobenius(got - exact) <= OP.apriori_bound(nA, nB, surv, mode, leaf, fl) + 1e-30
    # tile by tile: each output tile within its own share of both bounds
    t_acc = OP.accumulation_tile_bounds(nA, nB, surv, mode, leaf)
    assert np.all(OP.tile_errors(got, emu, leaf) <= t_acc), "a tile exceeds its accumulation share"
    t_ap = OP.apriori_tile_bounds(nA, nB, surv, mode, leaf, fl)
    assert np.all(OP.tile_errors(got, exact, leaf) <= t_ap), "a tile exceeds its a-priori share"


@pytest.mark.parametrize("name,mode", [("bf16_split", OP.BF16_SPLIT), ("fp16_split", OP.FP16_SPLIT)])
@pytest.mark.parametrize("target", [1e-3, 1e-5, 1e-7])
def test_split_flags_follow_oracle_rule(name, mode, target):
    n, leaf = 1024, 64
    a, b = _pair("alg", n, 1234)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    tau = 1e-6
    A, B = dev(a), dev(b)
    plan = P.Plan(n, leaf, mode).plan(dev(nA), dev(nB), tau, target)   # oracle norms: exact test
    surv, flags = plan_mask(plan)
    st = plan.stats()
    ref_surv = S.flat_survivors(nA, nB, tau)
    assert np.array_equal(surv, ref_surv)
    na, nb = OT.frobenius_from_normmap(nA), OT.frobenius_from_normmap(nB)
    _, b2 = S.skipped_bounds(nA, nB, ref_surv)
    fmt = OP.mode_format(mode)
    m = OP.flag_exponent(nA, nB, ref_surv, fmt, target, st["skipped_bound2"], na, nb)
    assert st["flag_exponent"] == m
    assert np.array_equal(flags, OP.flag_mask(nA, nB, ref_surv, m, na, nb))
    assert st["flagged"] == int(flags.sum())


@pytest.mark.parametrize("name,mode", MODES)
def test_tc_all_skipped_and_tau0(name, mode):
    a, b = _pair("alg", 384, 77)
    leaf = 64
    got, surv, _, st, _, _ = _run(a, b, leaf, math.inf, mode, 1e-5)
    assert st["survivors"] == 0 and not got.any()
    got, surv, flags, st, _, _ = _run(a, b, leaf, 0.0, mode, 1e-5)
    assert surv.all()
    dense = S.dense_reference(a, b)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    fl = flags if mode in (OP.BF16_SPLIT, OP.FP16_SPLIT) else None
    assert S.frobenius(got - dense) <= OP.apriori_bound(nA, nB, surv, mode, leaf, fl) * 1.0001
    t_ap = OP.apriori_tile_bounds(nA, nB, surv, mode, leaf, fl)
    assert np.all(OP.tile_errors(got, dense, leaf) <= t_ap * 1.0001)


def test_bf16_split_c2_full_size_sampled():
    """N = 8192, leaf 64, tau = 1e-4, BF16 with split products on dominant blocks."""
    a, b = synth.workload_c2()
    leaf, tau, target = 64, 1e-4, 1e-5
    got, surv, flags, st, gA, gB = _run(a, b, leaf, tau, OP.BF16_SPLIT, target)
    bd = st["bd"]
    pa, pb = S.padded64(a, leaf), S.padded64(b, leaf)
    ea, ha, la = {}, {}, {}
    g = np.random.Generator(np.random.PCG64(5))
    tiles = [(i, i) for i in range(0, bd, 8)] + [(i, min(bd - 1, i + 1)) for i in range(0, bd, 16)]
    tiles += [tuple(g.integers(0, bd, 2)) for _ in range(16)]

    def q(mat, i, k):
        key = (id(mat), i, k)
        if key not in ea:
            e, h, l_ = OP.quantize_block(S.block(mat, leaf, i, k).astype(np.float32), "bf16", True)
            ea[key], ha[key], la[key] = e, h.astype(np.float64), l_.astype(np.float64)
        return ea[key], ha[key], la[key]

    for i, j in tiles:
        emu = np.zeros((leaf, leaf))
        exact = np.zeros((leaf, leaf))
        for k in np.nonzero(surv[i, :, j])[0]:
            e1, h1, l1 = q(pa, i, k)
            e2, h2, l2 = q(pb, k, j)
            prod = h1 @ h2
            if flags[i, k, j]:
                prod = prod + 2.0 ** -8 * (h1 @ l2 + l1 @ h2)
            emu += math.ldexp(1.0, int(e1 + e2)) * prod
            exact += S.block(pa, leaf, i, k) @ S.block(pb, leaf, k, j)
        blk = got[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf]
        scale = max(S.frobenius(exact), 1e-300)
        assert S.frobenius(blk - emu) <= 1e-5 * scale + 1e-30
    # whole-matrix relative error against the FP64 pruned product stays near the target
    assert st["skipped_bound2"] / (st["norm_a"] * st["norm_b"]) <= 1e-5


@pytest.mark.parametrize("name,mode", [("fp32", OP.FP32), ("bf16_split", OP.BF16_SPLIT),
                                       ("tf32x3", OP.TF32X3)])
def test_plan_multiply_equals_plan_then_multiply(name, mode):
    """The one-call form (zero-fill started after the counting half) gives the same bits."""
    n, leaf = 777, 64
    a, b = _pair("alg", n, 4321)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    p = S.triple_products(S.normmap(a, leaf), S.normmap(b, leaf))
    tau = float(np.quantile(p[p > 0], 0.7))
    C1 = torch.full_like(A, float("nan"))
    C2 = torch.full_like(A, float("nan"))
    pl = P.Plan(n, leaf, mode)
    pl.plan(nA, nB, tau, 1e-6).multiply(A, B, C1)
    pl.plan_multiply(nA, nB, tau, A, B, C2, 1e-6)
    torch.cuda.synchronize()
    assert torch.equal(C1, C2)
    assert torch.isfinite(C2).all()


@pytest.mark.parametrize("name,mode", [("bf16", OP.BF16), ("bf16_split", OP.BF16_SPLIT),
                                       ("tf32x3", OP.TF32X3), ("fp16", OP.FP16)])
@pytest.mark.parametrize("ea,eb", [(97, -22), (-60, 40), (100, 20)])
def test_tc_wide_magnitudes(name, mode, ea, eb):
    """Operands far from 1 (A ~ 2^ea, B ~ 2^eb, C representable): BF16 and TF32 blocks are
    scaled on a 2^32 grid, so the exponent sum of a product can leave [-126, 127] (2^97 x 2^-22:
    128) while C stays finite; FP16 keeps the exact block exponent.  The result must match the
    oracle's emulation with exact exponents under the accumulation bound."""
    n, leaf = 384, 64
    a0, b0 = _pair("exp", n, 4242)
    a = (a0 * 2.0 ** ea).astype(np.float32)
    b = (b0 * 2.0 ** eb).astype(np.float32)
    assert np.isfinite(a).all() and np.isfinite(b).all()
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = S.triple_products(nA, nB)
    tau = float(np.quantile(p[p > 0], 0.5))
    got, surv, flags, st, _, _ = _run(a, b, leaf, tau, mode, 1e-6)
    assert np.isfinite(got).all()
    emu = OP.emulated_multiply(a, b, leaf, surv, mode, flags)
    t_acc = OP.accumulation_tile_bounds(nA, nB, surv, mode, leaf)
    assert np.all(OP.tile_errors(got, emu, leaf) <= t_acc)
    assert S.frobenius(got - emu) <= OP.accumulation_bound(nA, nB, surv, mode, leaf)


@pytest.mark.parametrize("name,mode", [("fp32", OP.FP32), ("bf16", OP.BF16)])
@pytest.mark.parametrize("t", [-2, 0, 3])
def test_empty_tiles_match_the_plan_at_ties(name, mode, t):
    """The one-call form writes the empty tiles from the counting half's per-tile counts,
    beside the rest of the plan, the two-call form from the finished plan's order: both must
    give the oracle's empty tiles, ties at tau included.  Blocks of constant value 2^a
    have the exact norm leaf 2^a, so with tau = leaf^2 2^t many products equal tau exactly;
    zero blocks and a NaN block are mixed in.  Tiles the oracle's flat rule leaves empty are
    zero, the others equal the two-call result bit for bit."""
    leaf, bd = 64, 8                                     # (the tensor modes take 64 and 128)
    n = leaf * bd
    g = np.random.Generator(np.random.PCG64(100 + t))
    ea = g.integers(-3, 4, size=(bd, bd))
    eb = g.integers(-3, 4, size=(bd, bd))
    a = np.kron(np.exp2(ea), np.ones((leaf, leaf))).astype(np.float32)
    b = np.kron(np.exp2(eb), np.ones((leaf, leaf))).astype(np.float32)
    a[0:leaf, 2 * leaf:3 * leaf] = 0.0
    b[5 * leaf:6 * leaf, :leaf] = 0.0
    a[3 * leaf + 1, 6 * leaf + 2] = np.nan
    tau = float(leaf * leaf * 2.0 ** t)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, tau)
    p = nA[:, :, None] * nB[None, :, :]
    assert np.any(p == tau)                              # ties present
    A, B = dev(a), dev(b)
    gA, gB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    C1 = torch.full_like(A, 7.0)
    C2 = torch.full_like(A, 7.0)
    pl = P.Plan(n, leaf, mode)
    pl.plan(gA, gB, tau, 1e-6).multiply(A, B, C1)
    pl.plan_multiply(gA, gB, tau, A, B, C2, 1e-6)
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    assert torch.equal(C1.view(torch.int32), C2.view(torch.int32))
    got = host(C2)
    nonempty = surv.any(axis=1)                          # [i, j]
    for i in range(bd):
        for j in range(bd):
            blk = got[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf]
            if not nonempty[i, j]:
                assert not blk.any(), (i, j)
            else:
                assert not np.all(blk == 7.0), (i, j)


@pytest.mark.parametrize("mode", [OP.BF16, OP.FP16])
def test_plan_schedules_give_the_same_bits(mode):
    """A plan's multiply under the per-tile static, dynamic and grouped schedules: the same bits,
    for the square form and (grouped falling back to per-tile) for a general plan with alpha and
    beta; an unknown schedule is refused."""
    n, leaf = 1000, 128
    a, b = _pair("sparse", n, 515)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    p = S.triple_products(S.normmap(a, leaf), S.normmap(b, leaf))
    tau = float(np.quantile(p[p > 0], 0.4))
    pl = P.Plan(n, leaf, mode).plan(nA, nB, tau, 1e-6)
    out = {}
    for sched in ("static", "dynamic", "groups"):
        C = torch.full_like(A, float("nan"))
        pl.set_schedule(sched).multiply(A, B, C)
        torch.cuda.synchronize()
        assert P.spamm_last_device_status() == 0
        out[sched] = C
    assert torch.equal(out["static"], out["dynamic"]) and torch.equal(out["static"], out["groups"])
    with pytest.raises(P.SpammError):
        pl.set_schedule("panels")
    gp = P.GeneralPlan(n, n, n, leaf, mode)
    C0 = dev(synth.near_sparse(n, 516))
    res = []
    for sched in ("static", "groups"):
        C = C0.clone()
        gp.set_schedule(sched).plan_multiply(nA, nB, tau, A, B, C, alpha=2.0, beta=0.5)
        torch.cuda.synchronize()
        res.append(C)
    assert torch.equal(res[0], res[1])
