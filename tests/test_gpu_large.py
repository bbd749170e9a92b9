"""Full-size parity at N = 32768, the largest single-GPU configuration, through the C ABI.

Exponential decay a_ij = exp(-alpha |i-j|) z_ij, z ~ N(0,1), A and B independent (the
benchmark's seeds), on sampled output block rows:
  * the GPU norm map equals the oracle's exactly rounded norms (Eq. 2) on the sampled rows
    of A and on every row of B that can decide their triples (3e-13 relative; zeros exact);
  * the GPU skip set on those rows equals the oracle's flat rule (up to the 1e-12 tau band);
  * C on those rows: FP32 within 1e-5 relative and every tile inside its accumulation
    share; FP16 and TF32x3 every tile inside its a-priori share of the oracle's FP64 rows;
  * certified exactness: the oracle's rows at tau_ref = 1e-30 skip products whose sum
    (bound1 over the sampled rows) is below 1e-17 of those rows' norm, so they are AB's
    rows to FP64 resolution; the GPU's error against them stays inside the pruning bound
    plus the rounding bound.
Near-sparse ReLU(N(0,1)) with 70% of the rest zeroed, BF16 at leaf 128, tau from the
oracle's valid-ratio search (50%), per-tile and grouped schedules bit-equal: 64 sampled output
tiles plus every diagonal tile against the oracle (FP64 block norms by pairwise sums, pinned
against the exactly rounded ones); the rest of C is parity unpinned (sampled).
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
from tests.gpu_helpers import band_ok, dev, host

pytestmark = pytest.mark.gpu

N = 32768
FP32_REL_TOL = 1e-5


def _decay(n, alpha):
    return (synth.exp_decay_normal(n, alpha, synth.config_seed(2, operand="A")),
            synth.exp_decay_normal(n, alpha, synth.config_seed(2, operand="B")))


@pytest.fixture(scope="module")
def decay_n32768():
    return _decay(N, 0.5)


def _row_survivors(plan, rows):
    """GPU survivors of the given block rows as {i: surv[k, j]} from the exported queues."""
    tp, kk = plan.export()
    bd = plan.bd
    out = {}
    for i in rows:
        s = np.zeros((bd, bd), dtype=bool)
        for j in range(bd):
            t = i * bd + j
            ks = (kk[tp[t]:tp[t + 1]] & 0x3FF).astype(np.int64)
            s[ks, j] = True
        out[i] = s
    return out


def _norms_close(gpu, ref, rel=3e-13):
    assert np.array_equal(gpu == 0, ref == 0)
    nz = ref > 0
    assert np.all(np.abs(gpu[nz] - ref[nz]) <= rel * ref[nz])


def _decay_rows_case(a, b, leaf, tau, modes, rows):
    n = a.shape[0]
    assert np.isfinite(a).all() and np.isfinite(b).all()
    A, B = dev(a), dev(b)
    gA, gB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    nA_rows = S.normmap_rows(a, leaf, rows)
    nB = S.normmap_needed(b, leaf, nA_rows, tau)
    ks = S.needed_b_rows(nA_rows, tau)
    assert 0 < ks.size < nB.shape[0]
    _norms_close(host(gA)[rows], nA_rows)
    _norms_close(host(gB)[ks], nB[ks])
    ref = S.spamm_rows(a, b, leaf, tau, rows, nA_rows, nB)
    # certified reference rows: at tau_ref the skipped products of these rows sum to far
    # below FP64 resolution of the rows themselves
    tau_ref = 1e-30
    exact = S.spamm_rows(a, b, leaf, tau_ref, rows, nA_rows, nB)
    skipped_ref = sum(float(np.sum(np.where(exact[i][1], 0.0, nA_rows[r][:, None] * nB)))
                      for r, i in enumerate(rows))
    norm_rows = math.sqrt(sum(float(np.sum(exact[i][0] ** 2)) for i in rows))
    assert skipped_ref <= 1e-17 * norm_rows
    C = torch.empty_like(A)
    for mode in modes:
        plan = P.Plan(n, leaf, mode).plan(gA, gB, tau, 1e-5)
        C.fill_(float("nan"))
        plan.multiply(A, B, C)
        torch.cuda.synchronize()
        assert P.spamm_last_device_status() == 0
        gsurv = _row_survivors(plan, rows)
        surv = np.stack([ref[i][1] for i in rows])
        for r, i in enumerate(rows):
            p = nA_rows[r][:, None] * nB
            assert band_ok(gsurv[i], ref[i][1], p, tau)
            assert np.array_equal(gsurv[i], ref[i][1])       # no product sits on this tau
        if mode == OP.FP32:
            t = OP.accumulation_tile_bounds(nA_rows, nB, surv, OP.FP32, leaf)
        else:
            t = OP.apriori_tile_bounds(nA_rows, nB, surv, mode, leaf)
        err2_exact, err_bound = 0.0, 0.0
        for r, i in enumerate(rows):
            strip = slice(i * leaf, min(n, (i + 1) * leaf))
            got = C[strip].double().cpu().numpy()
            want = ref[i][0]
            assert np.isfinite(got).all()
            assert np.all(OP.tile_errors(got, want, leaf)[0] <= t[r]), (mode, i)
            if mode == OP.FP32:
                assert S.frobenius(got - want) <= FP32_REL_TOL * S.frobenius(want)
            # against AB's rows: the pruning (skipped products of the row) plus the rounding
            skipped = np.where(ref[i][1], 0.0, nA_rows[r][:, None] * nB).sum(axis=0)
            err2_exact += float(np.sum((got - exact[i][0]) ** 2))
            err_bound += float(np.sum((skipped + t[r]) ** 2))
        assert math.sqrt(err2_exact) <= math.sqrt(err_bound) + 1e-12 * norm_rows
        del plan


def test_decay_n32768_sampled_rows(decay_n32768):
    """alpha = 0.5 (the benchmark's default input), tau = 1e-6, both leaf sizes; rows at the
    edges and inside."""
    a, b = decay_n32768
    for leaf, modes in ((128, (OP.FP32, OP.FP16, OP.TF32X3)), (64, (OP.FP16, OP.BF16_SPLIT))):
        bd = S.num_blocks(N, leaf)
        rows = [0, 1, bd // 3, bd // 2 + 1, bd - 2, bd - 1]
        _decay_rows_case(a, b, leaf, 1e-6, modes, rows)


def test_decay_n32768_error_targeted_tau(decay_n32768):
    """The same input at tau = 0.32, the threshold that a pruning error of 5e-6 of
    ||A||_F ||B||_F selects for it (about 2 300 survivors, pruning the dominant error): FP16
    and FP32 at leaf 128 on rows at the edges and in the middle."""
    a, b = decay_n32768
    bd = S.num_blocks(N, 128)
    _decay_rows_case(a, b, 128, 0.32, (OP.FP32, OP.FP16), [0, bd // 2, bd - 1])


@pytest.mark.parametrize("alpha,tau", [(0.1, 1e-6), (1.0, 1e-2)])
def test_decay_other_rates_sampled_rows(alpha, tau):
    """The other decay rates of the configuration at N = 16384 (alpha = 0.1 keeps about 60
    blocks of each row non-negligible; alpha = 1.0 is nearly block diagonal)."""
    a, b = _decay(16384, alpha)
    leaf = 128
    bd = S.num_blocks(16384, leaf)
    _decay_rows_case(a, b, leaf, tau, (OP.FP32, OP.FP16), [0, bd // 2, bd - 1])


@pytest.fixture(scope="module")
def near_sparse_n32768():
    return (synth.near_sparse(N, synth.config_seed(2, operand="A")),
            synth.near_sparse(N, synth.config_seed(2, operand="B")))


def test_near_sparse_n32768_sampled_tiles(near_sparse_n32768):
    a, b = near_sparse_n32768
    leaf = 128
    bd = S.num_blocks(N, leaf)
    nA, nB = S.normmap_blocked(a, leaf), S.normmap_blocked(b, leaf)
    tau, ratio, _ = OT.tau_for_valid_ratio(nA, nB, 0.5)
    assert abs(ratio - 0.5) <= 0.01
    A, B = dev(a), dev(b)
    gA, gB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    rel = np.abs(host(gA) / nA - 1.0).max()
    assert rel <= 1e-12, rel
    plan = P.Plan(N, leaf, P.BF16).plan(gA, gB, tau)
    st = plan.stats()
    assert abs(st["valid_ratio"] - ratio) <= 1e-6
    C = torch.full_like(A, float("nan"))
    plan.multiply(A, B, C)
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    # the grouped schedule (the autotuner's pick for this input) gives the same bits
    Cg = torch.full_like(A, float("nan"))
    plan.set_schedule("groups").multiply(A, B, Cg)
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    assert torch.equal(C, Cg)
    del Cg
    tp, kk = plan.export()
    g = np.random.Generator(np.random.PCG64(32768))
    tiles = [(i, i) for i in range(bd)] + [tuple(int(x) for x in g.integers(0, bd, 2))
                                            for _ in range(64)]
    kmax = max(int(S.survives(nA[i, :, None] * nB, tau).sum(axis=0).max()) for i in range(bd))
    gacc = OP.accumulation_coeff(OP.BF16, leaf, kmax)
    c_plain = OP.triple_error_coeff(OP.BF16, False, leaf)
    for i, j in tiles:
        p = nA[i, :] * nB[:, j]
        surv_o = S.survives(p, tau)
        t = i * bd + j
        surv_g = np.zeros(bd, dtype=bool)
        surv_g[(kk[tp[t]:tp[t + 1]] & 0x3FF).astype(np.int64)] = True
        assert band_ok(surv_g, surv_o, p, tau), (i, j)
        exact = np.zeros((leaf, leaf))
        for k in np.nonzero(surv_g)[0]:
            exact += S.block64(a, leaf, i, k) @ S.block64(b, leaf, k, j)
        got = C[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf].double().cpu().numpy()
        bound = float(np.sum(np.where(surv_g, (c_plain + gacc) * p, 0.0)))
        assert S.frobenius(got - exact) <= bound, (i, j)
