"""Reduced-precision SpAMM emulated in FP64 (oracle for the tensor-core modes).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper runs its tensor-core multiply on FP16 operands with FP32
accumulation (Section 3.3, Algorithm 3).  The modes emulated here extend that:

* every leaf block X[I,K] gets a power-of-two scale 2^e, e the frexp exponent
  of max |X[I,K]| (so the scaled maximum lies in [0.5, 1); a zero block has
  e = 0); the scaled block is X * 2^-e computed in FP32;
* ``hi`` = RNE rounding of the scaled block to the operand format
  (BF16: 8 significant bits, FP16: 11 with IEEE half range and subnormals,
  TF32: 11 significant bits with the FP32 exponent range);
* split modes also keep ``lo`` = RNE((scaled - hi) * 2^s_lo), s_lo = 8 (BF16)
  or 11 (FP16, TF32), so the low part stays clear of the FP16 subnormal range;
* a leaf product is 2^(ea+eb) * hi_a hi_b for plain triples and
  2^(ea+eb) * (hi_a hi_b + 2^-s_lo (hi_a lo_b + lo_a hi_b)) for split triples.

``Mode`` numbering matches the C ABI's precision enum.
"""
from __future__ import annotations

import math

import numpy as np

from . import spamm as S

FP32, TF32X3, BF16, FP16, BF16_SPLIT, FP16_SPLIT = range(6)
MODE_NAMES = {FP32: "fp32", TF32X3: "tf32x3", BF16: "bf16", FP16: "fp16",
              BF16_SPLIT: "bf16_split", FP16_SPLIT: "fp16_split"}

# unit roundoff u of each operand format (half an ulp of 1)
U_BF16 = 2.0 ** -8
U_FP16 = 2.0 ** -11
U_TF32 = 2.0 ** -11
# accumulation: FP32 adds; tensor-core adders may truncate, so use a full ulp
U_ACC = 2.0 ** -23
# bound on the absolute rounding error of a scaled FP16 value in the subnormal range
FP16_SUBNORMAL_HALF_ULP = 2.0 ** -25


def mode_format(mode: int) -> str:
    return {TF32X3: "tf32", BF16: "bf16", BF16_SPLIT: "bf16",
            FP16: "fp16", FP16_SPLIT: "fp16"}[mode]


def mode_is_split(mode: int) -> bool:
    return mode in (TF32X3, BF16_SPLIT, FP16_SPLIT)


def lo_shift(fmt: str) -> int:
    return {"bf16": 8, "fp16": 11, "tf32": 11}[fmt]


# ---------------------------------------------------------------------------
# Rounding to the operand formats (round to nearest, ties to even)
# ---------------------------------------------------------------------------

def _rne_drop_bits(x32: np.ndarray, drop: int) -> np.ndarray:
    """Round FP32 values to nearest-even after dropping the low ``drop`` significand bits.

    Works on the IEEE bit pattern: adding (2^(drop-1) - 1) plus the lowest kept
    bit and truncating is round-to-nearest-even for every finite value,
    including subnormals; the carry into the exponent field handles the
    binade change and overflow to infinity.  NaN is passed through.
    """
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    keep_lsb = (bits >> np.uint64(drop)) & np.uint64(1)
    rounded = (bits + np.uint64((1 << (drop - 1)) - 1) + keep_lsb) & np.uint64(
        (0xFFFFFFFF >> drop) << drop)
    out = rounded.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(x32), x32, out)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """RNE to bfloat16 (8 significant bits, FP32 exponent range); returned as FP32."""
    return _rne_drop_bits(x, 16)


def round_tf32(x: np.ndarray) -> np.ndarray:
    """RNE to TF32 (11 significant bits, FP32 exponent range); returned as FP32."""
    return _rne_drop_bits(x, 13)


def round_fp16(x: np.ndarray) -> np.ndarray:
    """RNE to IEEE binary16 (numpy's conversion: subnormals, overflow to inf)."""
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def round_to(fmt: str, x: np.ndarray) -> np.ndarray:
    return {"bf16": round_bf16, "fp16": round_fp16, "tf32": round_tf32}[fmt](x)


# ---------------------------------------------------------------------------
# Per-block power-of-two scaling and hi/lo operand blocks
# ---------------------------------------------------------------------------

def block_exponent(blk: np.ndarray) -> int:
    """frexp exponent of max|block|: max * 2^-e lies in [0.5, 1).  Zero block -> 0."""
    m = float(np.max(np.abs(blk))) if blk.size else 0.0
    if m == 0.0 or not math.isfinite(m):
        return 0
    return math.frexp(m)[1]


def quantize_block(blk32: np.ndarray, fmt: str, split: bool):
    """(e, hi, lo) of one FP32 block; lo is None unless ``split``.

    scaled = blk * 2^-e in FP32 (np.ldexp on float32 rounds like an FP32
    multiply by a power of two), hi = RNE(scaled), lo = RNE((scaled - hi) * 2^s_lo).
    """
    blk32 = np.asarray(blk32, dtype=np.float32)
    e = block_exponent(blk32)
    scaled = np.ldexp(blk32, np.int32(-e)).astype(np.float32)
    hi = round_to(fmt, scaled)
    lo = None
    if split:
        resid = (scaled - hi).astype(np.float32)          # exact in FP32
        lo = round_to(fmt, np.ldexp(resid, np.int32(lo_shift(fmt))).astype(np.float32))
    return e, hi, lo


def quantize_matrix(x: np.ndarray, leaf: int, fmt: str, split: bool):
    """Block grid of (e, hi, lo) for every leaf block of the zero-padded matrix."""
    n = x.shape[0]
    bd = S.num_blocks(n, leaf)
    p = np.zeros((bd * leaf, bd * leaf), dtype=np.float32)
    p[:n, :n] = x
    ex = np.zeros((bd, bd), dtype=np.int64)
    hi = np.zeros((bd, bd, leaf, leaf), dtype=np.float32)
    lo = np.zeros((bd, bd, leaf, leaf), dtype=np.float32) if split else None
    for i in range(bd):
        for k in range(bd):
            e, h, l_ = quantize_block(p[i * leaf:(i + 1) * leaf, k * leaf:(k + 1) * leaf],
                                      fmt, split)
            ex[i, k] = e
            hi[i, k] = h
            if split:
                lo[i, k] = l_
    return ex, hi, lo


# ---------------------------------------------------------------------------
# Dominant-triple flags for the split modes
# ---------------------------------------------------------------------------

FLAG_BIN_MIN = -200     # relative products below 2^-200 share the lowest bin


def relative_bin(p: np.ndarray, inv_ab: float) -> np.ndarray:
    """floor(log2(r)) of r = fl(p * inv_ab), clamped below at FLAG_BIN_MIN (r = 0 -> min)."""
    r = np.asarray(p, dtype=np.float64) * inv_ab
    m, e = np.frexp(r)                     # r = m 2^e, m in [0.5, 1)
    b = (e - 1).astype(np.int64)           # floor(log2 r) for r > 0
    return np.where(r > 0, np.maximum(b, FLAG_BIN_MIN), FLAG_BIN_MIN)


def inv_ab(norm_a: float, norm_b: float) -> float:
    ab = norm_a * norm_b
    return 1.0 / ab if ab > 0 else 0.0


def flag_exponent(nA, nB, surv, fmt: str, target_rel: float, bound2: float,
                  norm_a: float, norm_b: float) -> int:
    """Smallest relative-product binade that gets the hi+lo product.

    Triples with floor(log2(p/(||A|| ||B||))) >= m are flagged.  m is the
    largest integer in [FLAG_BIN_MIN - 1, 1] such that the hi-only error
    bound of the unflagged survivors, (2u + u^2) * sum_{bin < m} p, stays
    within half of the budget left after pruning,
    0.5 * (target_rel * ||A|| ||B|| - bound2).  A negative budget flags all.
    """
    u = {"bf16": U_BF16, "fp16": U_FP16, "tf32": U_TF32}[fmt]
    c1 = 2 * u + u * u
    ab = norm_a * norm_b
    budget = 0.5 * (target_rel * ab - bound2)
    if not budget >= 0:
        return FLAG_BIN_MIN - 1
    p = triple_products_surv(nA, nB, surv)
    bins = relative_bin(p, inv_ab(norm_a, norm_b))
    w = {}
    for b_, v in zip(bins.tolist(), p.tolist()):
        w.setdefault(b_, []).append(v)
    wsum = {b_: math.fsum(v) for b_, v in w.items()}
    best = FLAG_BIN_MIN - 1
    for m in range(FLAG_BIN_MIN - 1, 2):
        below = math.fsum(v for b_, v in wsum.items() if b_ < m)
        if c1 * below <= budget:
            best = m
    return best


def triple_products_surv(nA, nB, surv) -> np.ndarray:
    """Norm products of the surviving triples (any order)."""
    out = []
    for i in range(nA.shape[0]):
        p = nA[i, :, None] * nB
        out.append(p[surv[i]])
    return np.concatenate(out) if out else np.zeros(0)


def flag_mask(nA, nB, surv, m: int, norm_a: float, norm_b: float) -> np.ndarray:
    """flag[i,k,j] = surviving and relative bin >= m."""
    inv = inv_ab(norm_a, norm_b)
    out = np.zeros_like(surv)
    for i in range(nA.shape[0]):
        p = nA[i, :, None] * nB
        out[i] = surv[i] & (relative_bin(p, inv) >= m)
    return out


# ---------------------------------------------------------------------------
# Emulated multiply and the a-priori error bound
# ---------------------------------------------------------------------------

def emulated_multiply(a, b, leaf: int, surv, mode: int, flags=None) -> np.ndarray:
    """FP64 evaluation of the mode's rounded operands over the survivors.

    For TF32X3 every survivor takes the split product; for BF16_SPLIT /
    FP16_SPLIT the survivors in ``flags``; for BF16 / FP16 none.
    """
    n = a.shape[0]
    fmt = mode_format(mode)
    split = mode_is_split(mode)
    ea, ha, la = quantize_matrix(a, leaf, fmt, split)
    eb, hb, lb = quantize_matrix(b, leaf, fmt, split)
    bd = S.num_blocks(n, leaf)
    sl = 2.0 ** -lo_shift(fmt)
    c = np.zeros((bd * leaf, bd * leaf))
    for i in range(bd):
        for j in range(bd):
            ks = np.nonzero(surv[i, :, j])[0]
            if ks.size == 0:
                continue
            acc = np.zeros((leaf, leaf))
            for k in ks:
                h_a, h_b = ha[i, k].astype(np.float64), hb[k, j].astype(np.float64)
                prod = h_a @ h_b
                use_split = split and (mode == TF32X3 or (flags is not None and flags[i, k, j]))
                if use_split:
                    prod = prod + sl * (h_a @ lb[k, j].astype(np.float64)
                                        + la[i, k].astype(np.float64) @ h_b)
                acc += math.ldexp(1.0, int(ea[i, k] + eb[k, j])) * prod
            c[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf] = acc
    return c[:n, :n]


def triple_error_coeff(mode: int, split_triple: bool, leaf: int) -> float:
    """c such that ||A_ik B_kj - (mode's product)||_F <= c ||A_ik||_F ||B_kj||_F.

    Operand rounding: a = hi + e, |e| <= u|a| gives 2u + u^2.  Split:
    a = hi + lo + d with |d| <= u^2 |a| and |lo| <= u(1+u)|a| gives
    3u^2 + 2u^3 + 2u^4.  FP16 adds the subnormal floor: a scaled entry can
    lose up to 2^-25 absolutely, at most leaf * 2^-24 relative to the block
    norm (the scaled maximum is >= 0.5), i.e. u_eff = u + leaf 2^-24 per
    operand (and per lo part).  FP32 has no operand rounding.
    """
    if mode == FP32:
        return 0.0
    fmt = mode_format(mode)
    u = {"bf16": U_BF16, "fp16": U_FP16, "tf32": U_TF32}[fmt]
    sub = leaf * 2.0 ** -24 if fmt == "fp16" else 0.0
    if split_triple:
        # residual after hi+lo: per entry <= u * |scaled - hi| (+ subnormal floor of lo,
        # scaled back by 2^-s_lo), so u2 = u*(u + sub)
        u2 = u * (u + sub) + sub * 2.0 ** -lo_shift(fmt)
        ul = (u + sub) * (1 + u) + sub * 2.0 ** -lo_shift(fmt)
        return 2 * u2 + u2 * u2 + ul * ul
    ue = u + sub
    return 2 * ue + ue * ue


def accumulation_coeff(mode: int, leaf: int, kmax: int) -> float:
    """Relative bound g of the FP32 accumulation per surviving triple.

    FP32 mode (one FMA chain over every surviving k and every inner index):
    g = 1.01 (leaf kmax + 1) 2^-24.  Tensor-core modes (per-k products of at
    most 2 leaf + leaf terms, then one scaled add per k, adders possibly
    truncating): g = 1.01 (3 leaf + kmax + 4) 2^-23.  Both follow the
    standard |fl(sum) - sum| <= n u sum|terms| argument, with sum|terms|
    bounded in Frobenius norm by the norm products.
    """
    if mode == FP32:
        return 1.01 * (leaf * kmax + 1) * 2.0 ** -24
    return 1.01 * (3 * leaf + kmax + 4) * U_ACC


def apriori_bound(nA, nB, surv, mode: int, leaf: int, flags=None) -> float:
    """Tile-orthogonal bound on ||C_mode - C_exact(surv)||_F.

    sqrt(sum_ij (sum_{k surv} (c_ikj + g) p_ikj)^2), where c_ikj is
    :func:`triple_error_coeff` and g is :func:`accumulation_coeff`
    (kmax = most survivors of any tile).
    """
    bd = nA.shape[0]
    kmax = int(surv.sum(axis=1).max()) if surv.any() else 0
    g = accumulation_coeff(mode, leaf, kmax)
    c_plain = triple_error_coeff(mode, False, leaf)
    c_split = triple_error_coeff(mode, True, leaf) if mode != FP32 else 0.0
    tot = []
    for i in range(bd):
        p = nA[i, :, None] * nB
        coeff = np.full_like(p, c_plain)
        if mode == TF32X3:
            coeff[:] = c_split
        elif flags is not None and mode in (BF16_SPLIT, FP16_SPLIT):
            coeff = np.where(flags[i], c_split, c_plain)
        t = np.where(surv[i], (coeff + g) * p, 0.0).sum(axis=0)
        tot.append(t)
    tot = np.concatenate(tot)
    return math.sqrt(math.fsum((tot * tot).tolist()))


def accumulation_bound(nA, nB, surv, mode: int, leaf: int) -> float:
    """Bound on ||GPU result - FP64 evaluation of the same rounded operands||_F (c = 0)."""
    bd = nA.shape[0]
    kmax = int(surv.sum(axis=1).max()) if surv.any() else 0
    g = accumulation_coeff(mode, leaf, kmax)
    if mode_is_split(mode):
        g *= 2.0   # the hi*lo cross products add as much again, each below the hi*hi size
    tot = []
    for i in range(bd):
        p = nA[i, :, None] * nB
        tot.append(np.where(surv[i], g * p, 0.0).sum(axis=0))
    tot = np.concatenate(tot)
    return math.sqrt(math.fsum((tot * tot).tolist()))


# ---------------------------------------------------------------------------
# The same bounds tile by tile.  Both totals above are tile-orthogonal: each is
# sqrt(sum over output tiles of t_ij^2) with t_ij a bound on the Frobenius
# error of tile (i, j) alone.  These return the t_ij themselves ([bd, bd]), so
# a test can hold every tile to its own share instead of only the total (on a
# decay matrix the off-diagonal tiles are orders of magnitude below ||C||_F,
# and a whole-matrix check cannot see an error there).
# ---------------------------------------------------------------------------

def apriori_tile_bounds(nA, nB, surv, mode: int, leaf: int, flags=None) -> np.ndarray:
    """t_ij = sum over surviving k of (c_ikj + g) p_ikj: bound on the tile's ||C_mode - C_exact||_F,
    with c_ikj and g as in :func:`apriori_bound` (g from the largest survivor count).

    nA may hold only some block rows ([r, bd]; surv and flags then [r, bd, bd]): the result
    is [r, bd] for those rows, g taken from their largest survivor count."""
    rows = nA.shape[0]
    kmax = int(surv.sum(axis=1).max()) if surv.any() else 0
    g = accumulation_coeff(mode, leaf, kmax)
    c_plain = triple_error_coeff(mode, False, leaf)
    c_split = triple_error_coeff(mode, True, leaf) if mode != FP32 else 0.0
    out = np.zeros((rows, nB.shape[1]))
    for i in range(rows):
        p = nA[i, :, None] * nB                      # [k, j]
        if mode == TF32X3:
            coeff = np.full_like(p, c_split)
        elif flags is not None and mode in (BF16_SPLIT, FP16_SPLIT):
            coeff = np.where(flags[i], c_split, c_plain)
        else:
            coeff = np.full_like(p, c_plain)
        out[i] = np.where(surv[i], (coeff + g) * p, 0.0).sum(axis=0)
    return out


def accumulation_tile_bounds(nA, nB, surv, mode: int, leaf: int) -> np.ndarray:
    """t_ij = sum over surviving k of g p_ikj (doubled in split modes, as in
    :func:`accumulation_bound`): bound on the tile's distance from the FP64 evaluation of
    the same rounded operands (block rows as for :func:`apriori_tile_bounds`)."""
    rows = nA.shape[0]
    kmax = int(surv.sum(axis=1).max()) if surv.any() else 0
    g = accumulation_coeff(mode, leaf, kmax)
    if mode_is_split(mode):
        g *= 2.0
    out = np.zeros((rows, nB.shape[1]))
    for i in range(rows):
        p = nA[i, :, None] * nB
        out[i] = np.where(surv[i], g * p, 0.0).sum(axis=0)
    return out


def tile_errors(x: np.ndarray, y: np.ndarray, leaf: int) -> np.ndarray:
    """||X[i,j] - Y[i,j]||_F per leaf tile of two equally shaped r x c matrices
    ([ceil(r/leaf), ceil(c/leaf)], FP64; ragged edge tiles cover their in-range entries)."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    r, c = d.shape
    br, bc = -(-r // leaf), -(-c // leaf)
    p = np.zeros((br * leaf, bc * leaf))
    p[:r, :c] = d * d
    return np.sqrt(p.reshape(br, leaf, bc, leaf).sum(axis=(1, 3)))
