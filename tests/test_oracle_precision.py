"""Pins of the reduced-precision emulation (operand rounding, scaling, splits, bounds)."""
import math

import numpy as np
import pytest

import synth
from oracle import precision as P
from oracle import spamm as S


def _rne_frexp(x, sig_bits):
    """Independent RNE: scale the frexp significand to sig_bits integer bits, np.rint (half-even)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(np.ldexp(m, sig_bits)), e - sig_bits)


def _samples(seed=1, n=20000):
    g = np.random.Generator(np.random.PCG64(seed))
    x = (g.standard_normal(n) * np.exp2(g.integers(-30, 30, n))).astype(np.float32)
    # exact ties: values halfway between representable neighbours
    ties = (np.arange(1, 200, dtype=np.float64) * 2 + 1) * 2.0 ** -9   # odd multiples of 2^-9
    return np.concatenate([x, ties.astype(np.float32), -ties.astype(np.float32),
                           np.float32([0.0, -0.0, 1.0, 3.4e38])])


def test_bf16_rounding_matches_frexp_rint():
    x = _samples()
    got = P.round_bf16(x).astype(np.float64)
    ref = _rne_frexp(x, 8)
    finite = np.abs(ref) < 3.3e38
    assert np.array_equal(got[finite], ref[finite])
    assert np.isinf(P.round_bf16(np.float32([3.4e38])))[0]   # rounds past bf16 max


def test_tf32_rounding_matches_frexp_rint():
    x = _samples(2)
    assert np.array_equal(P.round_tf32(x).astype(np.float64), _rne_frexp(x, 11))


def test_fp16_library_rounding_agrees_with_bit_rounding_in_normal_range():
    x = _samples(3)
    x = x[(np.abs(x) >= 2.0 ** -14) & (np.abs(x) < 65000)]
    assert np.array_equal(P.round_fp16(x), P.round_tf32(x))    # both keep 11 significant bits


def test_block_exponent_range():
    g = np.random.Generator(np.random.PCG64(4))
    for _ in range(200):
        blk = (g.standard_normal((8, 8)) * 2.0 ** g.integers(-60, 60)).astype(np.float32)
        e = P.block_exponent(blk)
        mx = float(np.max(np.abs(blk))) * 2.0 ** -e
        assert 0.5 <= mx < 1.0
    assert P.block_exponent(np.zeros((4, 4), np.float32)) == 0


@pytest.mark.parametrize("fmt", ["bf16", "fp16", "tf32"])
def test_split_residual_is_second_order(fmt):
    g = np.random.Generator(np.random.PCG64(5))
    blk = (g.standard_normal((64, 64)) * 3.0).astype(np.float32)
    e, hi, lo = P.quantize_block(blk, fmt, True)
    scaled = blk.astype(np.float64) * 2.0 ** -e
    u = {"bf16": P.U_BF16, "fp16": P.U_FP16, "tf32": P.U_TF32}[fmt]
    r1 = np.abs(scaled - hi)
    assert (r1 <= u * np.abs(scaled) + 2.0 ** -25).all()
    r2 = np.abs(scaled - hi - lo.astype(np.float64) * 2.0 ** -P.lo_shift(fmt))
    assert (r2 <= u * u * np.abs(scaled) + 2.0 ** -36).all()


@pytest.mark.parametrize("mode", [P.BF16, P.FP16, P.TF32X3, P.BF16_SPLIT, P.FP16_SPLIT])
def test_exactly_representable_inputs_give_exact_products(mode):
    """Small integers times powers of two are exact in every format: emulation == FP64 product."""
    g = np.random.Generator(np.random.PCG64(6))
    n, leaf = 128, 32
    a = (g.integers(-8, 9, (n, n)) * 2.0 ** g.integers(-3, 3, (n, n))).astype(np.float32)
    b = (g.integers(-8, 9, (n, n)) * 2.0 ** g.integers(-3, 3, (n, n))).astype(np.float32)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, float(np.median(S.triple_products(nA, nB))))
    flags = surv.copy() if mode in (P.BF16_SPLIT, P.FP16_SPLIT) else None
    emu = P.emulated_multiply(a, b, leaf, surv, mode, flags)
    assert np.array_equal(emu, S.multiply_with_skipset(a, b, leaf, surv))


@pytest.mark.parametrize("mode", [P.BF16, P.FP16, P.TF32X3, P.BF16_SPLIT, P.FP16_SPLIT])
def test_apriori_bound_holds_for_emulation(mode):
    n, leaf = 256, 64
    a = synth.alg_decay_signed(n, 2.0, 41)
    b = synth.exp_decay_normal(n, 0.05, 42)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    for tau in (0.0, 1e-3):
        surv = S.flat_survivors(nA, nB, tau)
        flags = None
        if mode in (P.BF16_SPLIT, P.FP16_SPLIT):
            flags = P.flag_mask(nA, nB, surv, -4, S.frobenius(a), S.frobenius(b))
            assert flags.any() and (surv & ~flags).any()
        emu = P.emulated_multiply(a, b, leaf, surv, mode, flags)
        exact = S.multiply_with_skipset(a, b, leaf, surv)
        err = S.frobenius(emu - exact)
        bound = P.apriori_bound(nA, nB, surv, mode, leaf, flags)
        assert err <= bound
        # the bound is not vacuous: within a factor 1e4 of the measured error
        assert err > 0 and bound < 1e4 * err


def test_split_beats_plain_by_orders_of_magnitude():
    n, leaf = 128, 64
    a = synth.exp_decay_normal(n, 0.02, 43)
    b = synth.exp_decay_normal(n, 0.02, 44)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 0.0)
    exact = S.multiply_with_skipset(a, b, leaf, surv)
    for plain, split, u in ((P.BF16, P.BF16_SPLIT, P.U_BF16), (P.FP16, P.FP16_SPLIT, P.U_FP16)):
        e1 = S.frobenius(P.emulated_multiply(a, b, leaf, surv, plain) - exact)
        e2 = S.frobenius(P.emulated_multiply(a, b, leaf, surv, split, surv) - exact)
        assert e2 < 2 * u * e1          # the split removes one factor u


def test_flag_exponent_definition_brute_force():
    """The returned binade is the largest m whose unflagged hi-only bound fits the budget."""
    n, leaf = 256, 32
    a = synth.alg_decay_signed(n, 2.0, 45)
    b = synth.alg_decay_signed(n, 2.0, 46)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    na, nb = S.frobenius(a), S.frobenius(b)
    surv = S.flat_survivors(nA, nB, 1e-6)
    _, b2 = S.skipped_bounds(nA, nB, surv)
    p = S.triple_products(nA, nB)[surv]
    inv = 1.0 / (na * nb)
    c1 = 2 * P.U_BF16 + P.U_BF16 ** 2
    prev_m = None
    for target in (1e-2, 1e-3, 1e-4, 1e-5, 1e-7):
        m = P.flag_exponent(nA, nB, surv, "bf16", target, b2, na, nb)
        budget = 0.5 * (target * na * nb - b2)
        def fits(mm):
            return budget >= 0 and c1 * math.fsum(p[np.floor(np.log2(p * inv)) < mm].tolist()) <= budget
        if budget < 0:
            assert m == P.FLAG_BIN_MIN - 1
        else:
            assert fits(m) and (m == 1 or not fits(m + 1))
        if prev_m is not None:
            assert m <= prev_m                 # tighter targets flag more
        prev_m = m


def test_relative_bin_is_floor_log2():
    g = np.random.Generator(np.random.PCG64(7))
    p = np.exp2(g.uniform(-150, 0, 5000))
    p = np.concatenate([p, np.exp2(np.arange(-150, 1, dtype=np.float64)), [0.0]])
    b = P.relative_bin(p, 1.0)
    ref = np.where(p > 0, np.maximum(np.floor(np.log2(np.where(p > 0, p, 1.0))), P.FLAG_BIN_MIN),
                   P.FLAG_BIN_MIN)
    assert np.array_equal(b, ref.astype(np.int64))


@pytest.mark.parametrize("fmt,split", [("bf16", False), ("bf16", True), ("fp16", False),
                                       ("fp16", True), ("tf32", True)])
def test_quantize_matrix_reconstructs_each_block(fmt, split):
    """Every leaf block of the zero-padded matrix (ragged n) is recovered from its images: the
    scale exponent puts the block maximum in [0.5, 1), hi * 2^e is within u of each entry (plus
    FP16's subnormal floor) and hi + lo within about u^2; padding quantises to exact zeros."""
    n, leaf = 70, 32
    g = np.random.default_rng(7)
    x = (g.standard_normal((n, n)) * np.exp2(g.integers(-12, 12, (n, n)))).astype(np.float32)
    ex, hi, lo = P.quantize_matrix(x, leaf, fmt, split)
    bd = S.num_blocks(n, leaf)
    u = {"bf16": P.U_BF16, "fp16": P.U_FP16, "tf32": P.U_TF32}[fmt]
    pad = np.zeros((bd * leaf, bd * leaf))
    pad[:n, :n] = x
    for i in range(bd):
        for k in range(bd):
            blk = pad[i * leaf:(i + 1) * leaf, k * leaf:(k + 1) * leaf]
            mx = np.max(np.abs(blk))
            if mx > 0:
                assert 0.5 <= mx * 2.0 ** -float(ex[i, k]) < 1.0
            scale = 2.0 ** float(ex[i, k])
            floor = 2.0 ** -24 * scale if fmt == "fp16" else 0.0     # FP16 subnormal spacing
            h = hi[i, k].astype(np.float64) * scale
            assert np.all(np.abs(blk - h) <= u * np.abs(blk) + floor)
            if split:
                rec = (hi[i, k].astype(np.float64)
                       + lo[i, k].astype(np.float64) * 2.0 ** -P.lo_shift(fmt)) * scale
                assert np.all(np.abs(blk - rec) <= 2 * u * u * np.abs(blk) + 2 * floor)
            outside = np.zeros_like(blk, dtype=bool)
            outside[max(0, n - i * leaf):, :] = True
            outside[:, max(0, n - k * leaf):] = True
            assert np.all(h[outside] == 0.0)


@pytest.mark.parametrize("mode", [P.BF16, P.FP16, P.BF16_SPLIT, P.FP16_SPLIT, P.TF32X3])
def test_triple_error_coeff_bounds_single_products(mode):
    """The per-triple coefficient bounds the rounding error of single block products measured
    in FP64 on random blocks spanning several binades: ||AB - Q(A)Q(B)||_F <= c ||A|| ||B||."""
    leaf = 32
    fmt, split = P.mode_format(mode), P.mode_is_split(mode)
    c = P.triple_error_coeff(mode, split, leaf)
    g = np.random.default_rng(mode)
    worst = 0.0
    for _ in range(20):
        a = (g.standard_normal((leaf, leaf)) * np.exp2(g.integers(-6, 6, (leaf, leaf)))).astype(np.float32)
        b = (g.standard_normal((leaf, leaf)) * np.exp2(g.integers(-6, 6, (leaf, leaf)))).astype(np.float32)
        ea, ha, la = P.quantize_block(a, fmt, split)
        eb, hb, lb = P.quantize_block(b, fmt, split)
        qa = ha.astype(np.float64) + (la.astype(np.float64) * 2.0 ** -P.lo_shift(fmt) if split else 0)
        qb = hb.astype(np.float64) + (lb.astype(np.float64) * 2.0 ** -P.lo_shift(fmt) if split else 0)
        exact = a.astype(np.float64) @ b.astype(np.float64)
        # the split product omits lo*lo, as the tensor-core mode does
        got = (qa @ qb if not split else
               (ha.astype(np.float64) @ qb + la.astype(np.float64) * 2.0 ** -P.lo_shift(fmt)
                @ hb.astype(np.float64))) * 2.0 ** float(ea + eb)
        err = np.linalg.norm(exact - got) / (np.linalg.norm(a) * np.linalg.norm(b))
        worst = max(worst, err)
    assert worst <= c
    assert worst >= c * 1e-3   # the bound is not vacuous by orders of magnitude


# ---------------------------------------------------------------------------
# The accumulation bound against simulated FP32 accumulation chains
# ---------------------------------------------------------------------------

def _to_f32(x, toward_zero):
    """FP32 rounding of FP64 values: to nearest, or toward zero (a truncating adder)."""
    y = x.astype(np.float32)
    if toward_zero:
        y = np.where(np.abs(y.astype(np.float64)) > np.abs(x), np.nextafter(y, np.float32(0)), y)
    return y


def _elementwise(blocks, leaf):
    return np.kron(blocks, np.ones((leaf, leaf), dtype=blocks.dtype))


def _fma_chain_fp32(a, b, leaf, surv):
    """One FP32 FMA chain per output entry over every surviving k and inner index, k ascending
    (a product of two FP32 values is exact in FP64, so each step rounds once, then to FP32)."""
    n = a.shape[0]
    bd = S.num_blocks(n, leaf)
    m = bd * leaf
    A = np.zeros((m, m), np.float32)
    B = np.zeros((m, m), np.float32)
    A[:n, :n], B[:n, :n] = a, b
    c = np.zeros((m, m), np.float32)
    for k in range(bd):
        keep = _elementwise(surv[:, k, :], leaf)
        for p in range(k * leaf, (k + 1) * leaf):
            step = _to_f32(c + np.outer(A[:, p].astype(np.float64), B[p, :]), False)
            c = np.where(keep, step, c)
    return c[:n, :n]


def _tensor_chain(a, b, leaf, surv, mode, flags, toward_zero):
    """The tensor-core modes' accumulation model: per surviving k, a fresh FP32 sum of the
    leaf hi*hi terms (then 2^-s_lo hi*lo and lo*hi on split triples), each add rounded; then
    one rounded add of 2^(ea+eb) times that sum into C."""
    n = a.shape[0]
    bd = S.num_blocks(n, leaf)
    m = bd * leaf
    fmt = P.mode_format(mode)
    split = P.mode_is_split(mode)
    ea, ha, la = P.quantize_matrix(a, leaf, fmt, split)
    eb, hb, lb = P.quantize_matrix(b, leaf, fmt, split)
    sl = 2.0 ** -P.lo_shift(fmt)
    c = np.zeros((m, m), np.float32)
    for k in range(bd):
        keep = _elementwise(surv[:, k, :], leaf)
        if mode == P.TF32X3:
            use = np.ones((m, m), bool)
        elif split:
            use = _elementwise(flags[:, k, :], leaf)
        hA = np.concatenate([ha[i, k] for i in range(bd)], 0).astype(np.float64)
        hB = np.concatenate([hb[k, j] for j in range(bd)], 1).astype(np.float64)
        terms = [(hA[:, p], hB[p, :], 1.0, None) for p in range(leaf)]
        if split:
            lA = np.concatenate([la[i, k] for i in range(bd)], 0).astype(np.float64)
            lB = np.concatenate([lb[k, j] for j in range(bd)], 1).astype(np.float64)
            terms += [(hA[:, p], lB[p, :], sl, use) for p in range(leaf)]
            terms += [(lA[:, p], hB[p, :], sl, use) for p in range(leaf)]
        s = np.zeros((m, m), np.float32)
        for x, y, w, mask in terms:
            step = _to_f32(s + w * np.outer(x, y), toward_zero)
            s = step if mask is None else np.where(mask, step, s)
        scale = _elementwise(np.ldexp(1.0, (ea[:, k, None] + eb[None, k, :]).astype(np.int64)),
                             leaf)
        c = np.where(keep, _to_f32(c + scale * s, toward_zero), c)
    return c[:n, :n]


def _positive(n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.uniform(0.5, 1.0, (n, n)).astype(np.float32)


def test_accumulation_bound_covers_an_fp32_fma_chain():
    """All-positive inputs make the rounding errors of one long chain add up; the simulated
    chain stays inside the bound, and the bound is not vacuous (within 100x of it)."""
    n, leaf = 200, 64
    a, b = _positive(n, 71), _positive(n, 72)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 0.0)
    ref = S.multiply_with_skipset(a, b, leaf, surv)
    err = np.linalg.norm(_fma_chain_fp32(a, b, leaf, surv).astype(np.float64) - ref)
    bound = P.accumulation_bound(nA, nB, surv, P.FP32, leaf)
    assert 0.01 * bound < err <= bound


@pytest.mark.parametrize("mode", [P.FP16, P.BF16_SPLIT, P.TF32X3])
def test_accumulation_bound_covers_truncating_tensor_chains(mode):
    """Rounding toward zero on positive data is the worst ordinary case of the model: it stays
    inside the bound, yet breaks a bound that drops the per-k product length (3 leaf), so that
    term is needed."""
    n, leaf = 200, 64
    a, b = _positive(n, 73), _positive(n, 74)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 0.0)
    flags = surv.copy() if mode == P.BF16_SPLIT else None
    emu = P.emulated_multiply(a, b, leaf, surv, mode, flags)
    bound = P.accumulation_bound(nA, nB, surv, mode, leaf)
    for toward_zero in (False, True):
        sim = _tensor_chain(a, b, leaf, surv, mode, flags, toward_zero).astype(np.float64)
        err = np.linalg.norm(sim - emu)
        assert err <= bound
    kmax = int(surv.sum(axis=1).max())
    if P.mode_is_split(mode):
        assert err > bound * (kmax + 4) / (3 * leaf + kmax + 4)


@pytest.mark.parametrize("mode", [P.BF16, P.FP16_SPLIT, P.TF32X3])
def test_accumulation_bound_on_pruned_signed_inputs(mode):
    """A decaying signed pair under pruning (uneven survivor counts per tile, ragged edge)."""
    n, leaf = 150, 64
    a = synth.exp_decay_normal(n, 0.02, 75)
    b = synth.exp_decay_normal(n, 0.02, 76)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    p = np.sort((nA[:, :, None] * nB[None, :, :]).ravel())
    surv = S.flat_survivors(nA, nB, float(p[p.size // 3]))
    assert 0 < surv.sum() < surv.size
    flags = surv.copy() if mode == P.FP16_SPLIT else None
    emu = P.emulated_multiply(a, b, leaf, surv, mode, flags)
    bound = P.accumulation_bound(nA, nB, surv, mode, leaf)
    for toward_zero in (False, True):
        sim = _tensor_chain(a, b, leaf, surv, mode, flags, toward_zero).astype(np.float64)
        assert np.linalg.norm(sim - emu) <= bound


# --------------------------------------------------------------------------- per-tile bounds

def _decay_pair(n=320, seed=81, alpha=0.05):
    return synth.exp_decay_normal(n, alpha, seed), synth.exp_decay_normal(n, alpha, seed + 1)


@pytest.mark.parametrize("mode", [P.BF16, P.FP16_SPLIT, P.TF32X3])
def test_tile_bounds_are_the_shares_of_the_totals(mode):
    a, b = _decay_pair()
    leaf = 64
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 1e-3)
    flags = surv.copy() if mode == P.FP16_SPLIT else None
    t_ap = P.apriori_tile_bounds(nA, nB, surv, mode, leaf, flags)
    t_ac = P.accumulation_tile_bounds(nA, nB, surv, mode, leaf)
    assert t_ap.shape == (nA.shape[0],) * 2
    assert math.isclose(math.sqrt(math.fsum((t_ap * t_ap).ravel().tolist())),
                        P.apriori_bound(nA, nB, surv, mode, leaf, flags), rel_tol=1e-12)
    assert math.isclose(math.sqrt(math.fsum((t_ac * t_ac).ravel().tolist())),
                        P.accumulation_bound(nA, nB, surv, mode, leaf), rel_tol=1e-12)
    # a tile without survivors has a zero bound, so a check against it demands exact zeros
    assert np.all(t_ap[~surv.any(axis=1)] == 0.0)


@pytest.mark.parametrize("mode", [P.BF16, P.FP16, P.TF32X3, P.BF16_SPLIT])
def test_apriori_tile_bounds_hold_tile_by_tile(mode):
    """Every tile of the emulated product (even the off-diagonal ones, many decades below
    ||C||_F) stays within its own a-priori share."""
    a, b = _decay_pair(alpha=0.1)
    leaf = 64
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 0.0)
    flags = None
    if mode == P.BF16_SPLIT:
        flags = P.flag_mask(nA, nB, surv, -6, S.frobenius(a), S.frobenius(b))
    emu = P.emulated_multiply(a, b, leaf, surv, mode, flags)
    exact = S.multiply_with_skipset(a, b, leaf, surv)
    err = P.tile_errors(emu, exact, leaf)
    t = P.apriori_tile_bounds(nA, nB, surv, mode, leaf, flags)
    assert np.all(err <= t)
    assert t.max() / t.min() > 1e3          # the tiles span several decades


@pytest.mark.parametrize("mode", [P.FP16, P.BF16_SPLIT])
def test_accumulation_tile_bounds_cover_simulated_chains(mode):
    n, leaf = 200, 64
    a, b = synth.exp_decay_normal(n, 0.02, 77), synth.exp_decay_normal(n, 0.02, 78)
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 0.0)
    flags = surv.copy() if mode == P.BF16_SPLIT else None
    emu = P.emulated_multiply(a, b, leaf, surv, mode, flags)
    t = P.accumulation_tile_bounds(nA, nB, surv, mode, leaf)
    for toward_zero in (False, True):
        sim = _tensor_chain(a, b, leaf, surv, mode, flags, toward_zero).astype(np.float64)
        assert np.all(P.tile_errors(sim, emu, leaf) <= t)
    sim = _fma_chain_fp32(a, b, leaf, surv).astype(np.float64)
    ref = S.multiply_with_skipset(a, b, leaf, surv)
    assert np.all(P.tile_errors(sim, ref, leaf) <= P.accumulation_tile_bounds(nA, nB, surv,
                                                                              P.FP32, leaf))


def test_tile_check_catches_an_error_the_total_misses():
    """A planted mistake in a small off-diagonal tile (its entries written with the wrong sign)
    keeps the whole-matrix error inside the total bound but breaks that tile's own bound."""
    a, b = _decay_pair()
    leaf = 64
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 0.0)
    emu = P.emulated_multiply(a, b, leaf, surv, P.BF16)
    exact = S.multiply_with_skipset(a, b, leaf, surv)
    bad = emu.copy()
    bad[0:leaf, 3 * leaf:4 * leaf] *= -1.0            # tile (0, 3): far from the diagonal
    total = P.apriori_bound(nA, nB, surv, P.BF16, leaf)
    assert S.frobenius(bad - exact) <= total
    t = P.apriori_tile_bounds(nA, nB, surv, P.BF16, leaf)
    assert not np.all(P.tile_errors(bad, exact, leaf) <= t)
    assert np.all(P.tile_errors(emu, exact, leaf) <= t)


def test_tile_bounds_of_sampled_rows_match_the_full_map():
    """The row form (nA holding only some block rows) gives those rows of the full result,
    up to g, which the sampled rows' own largest survivor count can only lower."""
    a, b = _decay_pair(alpha=0.1)
    leaf = 64
    nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
    surv = S.flat_survivors(nA, nB, 1e-6)
    rows = [0, 3]
    full = P.apriori_tile_bounds(nA, nB, surv, P.FP16, leaf)
    part = P.apriori_tile_bounds(nA[rows], nB, surv[rows], P.FP16, leaf)
    assert part.shape == (2, nB.shape[1])
    assert np.all(part <= full[rows]) and np.allclose(part, full[rows], rtol=1e-3)
    emu = P.emulated_multiply(a, b, leaf, surv, P.FP16)
    exact = S.multiply_with_skipset(a, b, leaf, surv)
    for r, i in enumerate(rows):
        strip = slice(i * leaf, (i + 1) * leaf)
        assert np.all(P.tile_errors(emu[strip], exact[strip], leaf)[0] <= part[r])


def test_c2_error_table_is_consistent():
    """The stored accuracy table of the N = 8192 configuration (written by
    `python -m oracle.c2_error_table`, oracle only): every mode's error stays inside the
    pruning bound plus its a-priori bound, the pruning error inside bound2, survivors grow as
    tau falls, and TF32x3 stays at the pruning error (its rounding is far below it)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "c2_error_table.json")
    t = json.load(open(path))
    rows = t["rows"]
    assert [r["tau"] for r in rows] == sorted((r["tau"] for r in rows), reverse=True)
    assert all(a["S"] <= b["S"] for a, b in zip(rows, rows[1:]))
    for r in rows:
        assert r["pruning_rel"] <= r["bound2_rel"] * (1 + 1e-9)
        for name, m in r["modes"].items():
            assert m["rel_err"] <= r["bound2_rel"] + m["apriori_rel"], (r["tau"], name)
            assert m["rounding_rel"] <= m["apriori_rel"], (r["tau"], name)
        assert r["modes"]["tf32x3"]["rounding_rel"] < 0.1 * r["modes"]["fp16"]["rounding_rel"]
