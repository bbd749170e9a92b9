"""GPU parity of the batched path: one launch of each kernel over many instances.

Each instance of a batch must give exactly what the single-instance entry
points give it alone (same kernels, same arithmetic, so bit-identical C, norm
maps, work queues and statistics), and the single path is itself checked
against the oracle; the FP32 batch is also compared with the oracle directly.
"""
import math

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import spamm as S
from tests.gpu_helpers import band_ok, dev, host, plan_mask

pytestmark = pytest.mark.gpu

FP32_REL_TOL = 1e-5
NORM_REL_TOL = 3e-13


def _instances(count, seed, n_lo, n_hi, q):
    """Seeded uneven-size decay instances; tau at quantile q of each one's norm products."""
    specs = synth.batch_specs(count, seed, n_lo=n_lo, n_hi=n_hi)
    out = []
    for t, sp in enumerate(specs):
        a, b = synth.spec_matrices(sp)
        out.append((a, b))
    return specs, out


def _taus(pairs, leaf, q):
    taus = []
    for a, b in pairs:
        p = S.triple_products(S.normmap(a, leaf), S.normmap(b, leaf))
        taus.append(float(np.quantile(p[p > 0], q)))
    return taus


def _single(a, b, leaf, tau, prec, target):
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    plan = P.Plan(a.shape[0], leaf, prec).plan(nA, nB, tau, target)
    C = torch.full_like(A, float("nan"))
    plan.multiply(A, B, C)
    tp, kk = plan.export()
    return host(C), host(nA), host(nB), tp, kk, plan.stats()


CASES = [(32, P.FP32, 0.7), (64, P.FP32, 0.5), (64, P.BF16, 0.6), (128, P.BF16_SPLIT, 0.4),
         (64, P.FP16_SPLIT, 0.8), (128, P.TF32X3, 0.5)]


@pytest.mark.parametrize("leaf,prec,q", CASES)
def test_batch_equals_single_instances(leaf, prec, q):
    specs, pairs = _instances(7, 4242 + leaf + prec, 40, 900, q)
    taus = _taus(pairs, leaf, q)
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    Cs = [torch.full_like(A, float("nan")) for A in As]
    batch = P.Batch([a.shape[0] for a, _ in pairs], leaf, prec, graph=False)
    batch.run(As, Bs, Cs, taus, target_rel_err=1e-6)
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    stats = batch.stats()
    for i, (a, b) in enumerate(pairs):
        c1, nA1, nB1, tp1, kk1, st1 = _single(a, b, leaf, taus[i], prec, 1e-6)
        nA, nB, tp, kk = batch.export(i)
        assert np.array_equal(nA, nA1) and np.array_equal(nB, nB1), f"instance {i}: norm maps"
        assert np.array_equal(tp, tp1) and np.array_equal(kk, kk1), f"instance {i}: queues"
        c = host(Cs[i])
        assert np.isfinite(c).all(), f"instance {i}: C not written completely"
        assert np.array_equal(c, c1), f"instance {i}: C differs from the single-instance call"
        for key in ("survivors", "nonempty_tiles", "flagged", "max_tile_survivors",
                    "flag_exponent", "bd"):
            assert stats[i][key] == st1[key], (i, key)
        for key in ("valid_ratio", "skipped_bound1", "skipped_bound2", "norm_a", "norm_b"):
            assert stats[i][key] == pytest.approx(st1[key], rel=1e-12, abs=0), (i, key)
    batch.close()


@pytest.mark.parametrize("leaf", [32, 64])
def test_batch_fp32_against_oracle(leaf):
    specs, pairs = _instances(6, 777 + leaf, 50, 700, 0.6)
    taus = _taus(pairs, leaf, 0.6)
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    Cs = [torch.full_like(A, float("nan")) for A in As]
    batch = P.Batch([a.shape[0] for a, _ in pairs], leaf, P.FP32, graph=True)
    batch.run(As, Bs, Cs, taus)
    torch.cuda.synchronize()
    stats = batch.stats()
    for i, (a, b) in enumerate(pairs):
        oA, oB = S.normmap(a, leaf), S.normmap(b, leaf)
        gA, gB, tp, kk = batch.export(i)
        zero = oA == 0
        assert np.array_equal(gA[zero], oA[zero])
        assert np.max(np.abs(gA[~zero] - oA[~zero]) / oA[~zero], initial=0) <= NORM_REL_TOL
        bd = oA.shape[0]
        surv = np.zeros((bd, bd, bd), dtype=bool)
        for t in range(bd * bd):
            ti, tj = divmod(t, bd)
            surv[ti, (kk[tp[t]:tp[t + 1]] & 0x3FF).astype(np.int64), tj] = True
        ref_surv = S.flat_survivors(oA, oB, taus[i])
        assert band_ok(surv, ref_surv, S.triple_products(oA, oB), taus[i])
        assert stats[i]["survivors"] == int(surv.sum())
        ref = S.multiply_with_skipset(a, b, leaf, surv)
        err = np.linalg.norm(host(Cs[i]) - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err <= FP32_REL_TOL, (i, err)
    batch.close()


def test_batch_graph_replay_with_new_pointers_and_tau():
    leaf = 64
    specs, pairs = _instances(5, 99, 64, 600, 0.5)
    ns = [a.shape[0] for a, _ in pairs]
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    g = P.Batch(ns, leaf, P.BF16_SPLIT, graph=True)
    e = P.Batch(ns, leaf, P.BF16_SPLIT, graph=False)
    for q in (0.3, 0.7, 0.3):
        taus = _taus(pairs, leaf, q)
        Cg = [torch.full_like(A, float("nan")) for A in As]   # new outputs every run
        Ce = [torch.full_like(A, float("nan")) for A in As]
        g.run(As, Bs, Cg, taus, 1e-6)
        e.run(As, Bs, Ce, taus, 1e-6)
        torch.cuda.synchronize()
        for i in range(len(As)):
            assert torch.equal(Cg[i], Ce[i]), (q, i)
        sg, se = g.stats(), e.stats()
        assert [s["survivors"] for s in sg] == [s["survivors"] for s in se]
    g.close()
    e.close()


def test_multiply_batched_one_shot():
    leaf = 64
    specs, pairs = _instances(4, 5150, 100, 500, 0.5)
    taus = _taus(pairs, leaf, 0.5)
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    Cs = [torch.full_like(A, float("nan")) for A in As]
    stats = P.spamm_multiply_batched(As, Bs, Cs, taus, leaf, P.BF16)
    for i, (a, b) in enumerate(pairs):
        c1, *_rest, st1 = _single(a, b, leaf, taus[i], P.BF16, 1e-5)
        assert np.array_equal(host(Cs[i]), c1)
        assert stats[i]["survivors"] == st1["survivors"]


def test_batch_degenerate_taus():
    """tau = 0 keeps every triple (C = AB up to FP32 rounding), tau = inf skips all (C = 0)."""
    leaf = 32
    pairs = [(synth.exp_decay_su(n, 0.5, 11 + n), synth.exp_decay_su(n, 0.5, 12 + n))
             for n in (33, 96, 130)]
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    Cs = [torch.full_like(A, float("nan")) for A in As]
    batch = P.Batch([33, 96, 130], leaf, P.FP32, graph=False)
    batch.run(As, Bs, Cs, [0.0, math.inf, 0.0])
    torch.cuda.synchronize()
    st = batch.stats()
    for i, (a, b) in enumerate(pairs):
        bd = -(-a.shape[0] // leaf)
        if i == 1:
            assert st[i]["survivors"] == 0
            assert not host(Cs[i]).any()
        else:
            assert st[i]["survivors"] == bd ** 3
            ref = S.dense_reference(a, b)
            assert np.linalg.norm(host(Cs[i]) - ref) / np.linalg.norm(ref) <= FP32_REL_TOL
    batch.close()


def test_batch_rejects_bad_problems():
    A = torch.zeros(64, 64, device="cuda")
    B = torch.zeros(64, 64, device="cuda")
    C = torch.zeros(64, 64, device="cuda")
    batch = P.Batch([64, 64], 32, P.FP32, graph=False)
    with pytest.raises(P.SpammError) as e:      # output of one instance is the input of another
        batch.run([A, C], [B, B], [C, torch.zeros_like(C)], [0.0, 0.0])
    assert e.value.code == 1
    with pytest.raises(P.SpammError) as e:      # two instances write the same output
        batch.run([A, A], [B, B], [C, C], [0.0, 0.0])
    assert e.value.code == 1
    with pytest.raises(P.SpammError) as e:      # shape differs from creation
        batch.run([A, torch.zeros(65, 65, device="cuda")], [B, B],
                  [C, torch.zeros(65, 65, device="cuda")], [0.0, 0.0])
    assert e.value.code == 1
    with pytest.raises(P.SpammError) as e:      # NaN tau
        batch.run([A, A], [B, B], [C, torch.zeros_like(C)], [0.0, float("nan")])
    assert e.value.code == 1
    batch.close()


@pytest.mark.parametrize("prec", [P.FP32, P.BF16_SPLIT])
def test_dynamic_schedule_and_timings(prec):
    """The dynamic multiply schedule gives the same C as the static one; phase timings exist."""
    leaf = 64
    specs, pairs = _instances(6, 31337, 64, 800, 0.5)
    taus = _taus(pairs, leaf, 0.5)
    ns = [a.shape[0] for a, _ in pairs]
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    Cs = [torch.full_like(A, float("nan")) for A in As]
    Cd = [torch.full_like(A, float("nan")) for A in As]
    st = P.Batch(ns, leaf, prec, graph=False)
    dy = P.Batch(ns, leaf, prec, graph=True, dynamic=True)
    tm = P.Batch(ns, leaf, prec, graph=True, dynamic=True, timing=True)
    st.run(As, Bs, Cs, taus, 1e-6)
    for _ in range(2):   # a second run re-uses the counter: it must be reset
        dy.run(As, Bs, Cd, taus, 1e-6)
        torch.cuda.synchronize()
        for i in range(len(As)):
            assert torch.equal(Cs[i], Cd[i]), i
    Ct = [torch.full_like(A, float("nan")) for A in As]
    tm.run(As, Bs, Ct, taus, 1e-6)
    t = tm.timings()
    assert t["normmap"] > 0 and t["plan"] > 0 and t["multiply"] > 0 and t["round"] >= 0, t
    if prec != P.FP32:
        assert t["round"] > 0, t
    for i in range(len(As)):
        assert torch.equal(Cs[i], Ct[i]), i
    for b in (st, dy, tm):
        b.close()


def test_autotune_returns_a_measured_candidate():
    specs, pairs = _instances(5, 2718, 128, 700, 0.5)
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    Cs = [torch.zeros_like(A) for A in As]
    taus = _taus(pairs, 64, 0.5)
    best, allc = P.spamm_batch_autotune(As, Bs, Cs, taus, P.BF16, reps=2)
    assert len(allc) == 5
    assert {(c["leaf"], c["schedule"]) for c in allc} == {(64, "static"), (64, "dynamic"),
                                                          (128, "static"), (128, "dynamic"),
                                                          (128, "groups")}
    assert best["ms"] == min(c["ms"] for c in allc if c["ms"] >= 0)


def _groups_vs_static(As, Bs, taus, prec):
    ns = [A.shape[0] for A in As]
    Cs = [torch.full_like(A, float("nan")) for A in As]
    Cg = [torch.full_like(A, float("nan")) for A in As]
    st = P.Batch(ns, 128, prec, graph=False)
    gr = P.Batch(ns, 128, prec, graph=True, groups=True)
    st.run(As, Bs, Cs, taus, 1e-6)
    for _ in range(2):   # graph capture, then replay
        for C in Cg:
            C.fill_(float("nan"))
        gr.run(As, Bs, Cg, taus, 1e-6)
        torch.cuda.synchronize()
        assert P.spamm_last_device_status() == 0
        for i in range(len(As)):
            assert torch.equal(Cs[i], Cg[i]), i
    stats = gr.stats()
    st.close()
    gr.close()
    return Cg, stats


@pytest.mark.parametrize("prec", [P.BF16, P.FP16])
def test_groups_schedule_equals_per_tile_decay(prec):
    """Grouped multiply (four tiles of a block row share A) against the per-tile schedule,
    bit for bit: uneven decay instances (block columns not a multiple of four, ragged last
    tiles), FP16 with exact block exponents (several accumulator runs per tile: partial sums
    kept in C) and BF16 on the 2^32 grid."""
    specs, pairs = _instances(6, 777 + prec, 200, 1300, 0.5)
    taus = _taus(pairs, 128, 0.5)
    As = [dev(a) for a, _ in pairs]
    Bs = [dev(b) for _, b in pairs]
    _groups_vs_static(As, Bs, taus, prec)


@pytest.mark.parametrize("n,q", [(1000, 0.5), (700, 0.2), (1536, 0.9)])
def test_groups_schedule_near_sparse_against_oracle(n, q):
    """Near-sparse BF16 at leaf 128 (the dense-ish skip sets the grouped multiply is for):
    bit-equal to the per-tile schedule, and every tile within its accumulation share of the
    oracle's emulation of the rounded operands."""
    from oracle import precision as OP
    a, b = synth.near_sparse(n, 51 + n), synth.near_sparse(n, 52 + n)
    leaf = 128
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = S.triple_products(nA, nB)
    tau = float(np.quantile(p[p > 0], q))
    A, B = dev(a), dev(b)
    Cg, _ = _groups_vs_static([A], [B], [tau], P.BF16)
    gA, gB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    plan = P.Plan(n, leaf, P.BF16).plan(gA, gB, tau, 1e-6)
    surv, _ = plan_mask(plan)
    got = host(Cg[0]).astype(np.float64)
    emu = OP.emulated_multiply(a, b, leaf, surv, OP.BF16)
    t_acc = OP.accumulation_tile_bounds(nA, nB, surv, OP.BF16, leaf)
    assert np.all(OP.tile_errors(got, emu, leaf) <= t_acc)


def test_groups_schedule_wide_magnitudes():
    """A ~ 2^97, B ~ 2^-22: exponent sums past 127 on the BF16 grid (two-factor scaling)."""
    n = 640
    a = (synth.exp_decay_normal(n, 0.01, 61) * 2.0 ** 97).astype(np.float32)
    b = (synth.exp_decay_normal(n, 0.01, 62) * 2.0 ** -22).astype(np.float32)
    taus = _taus([(a, b)], 128, 0.3)
    Cg, _ = _groups_vs_static([dev(a)], [dev(b)], taus, P.BF16)
    assert bool(torch.isfinite(Cg[0]).all())


def test_groups_schedule_edges():
    """Grouped multiply: no survivors at all (tau = inf: the end-of-work path only, C all
    zeros), every triple kept (tau = 0), and more than 32 block columns of k (several mask
    words per tile, n = 4224: 33 blocks, a ragged last block) next to a small instance."""
    a, b = synth.near_sparse(640, 71), synth.near_sparse(640, 72)
    A, B = dev(a), dev(b)
    Cg, st = _groups_vs_static([A], [B], [math.inf], P.BF16)
    assert st[0]["survivors"] == 0 and not bool(Cg[0].any())
    Cg, st = _groups_vs_static([A], [B], [0.0], P.BF16)
    assert st[0]["survivors"] == 5 ** 3
    big = synth.exp_decay_normal(4224, 0.002, 73), synth.exp_decay_normal(4224, 0.002, 74)
    taus = _taus([big, (a, b)], 128, 0.6)
    _groups_vs_static([dev(big[0]), A], [dev(big[1]), B], taus, P.FP16)
