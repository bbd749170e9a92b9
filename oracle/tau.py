"""Choosing tau: valid-ratio search (Section 3.5.2), norm-product histogram, bisection.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from . import spamm as S

HIST_BINS = 64


# ---------------------------------------------------------------------------
# Valid ratio and its tau search (Section 3.5.2)
# ---------------------------------------------------------------------------

def mean_norm_product(nA: np.ndarray, nB: np.ndarray) -> float:
    """ave = mean of nA[i,k] nB[k,j] over all BDIM^3 triples.

    The sum factorises: sum_k (sum_i nA[i,k]) (sum_j nB[k,j]).
    """
    bd = nA.shape[0]
    col = nA.sum(axis=0)          # sum_i nA[i, k]
    row = nB.sum(axis=1)          # sum_j nB[k, j]
    return math.fsum((col * row).tolist()) / bd ** 3


def valid_ratio_at(nA, nB, tau: float) -> float:
    """Fraction of surviving leaf triples at threshold tau (Section 3.5.2 formula)."""
    bd = nA.shape[0]
    cnt = 0
    for i in range(bd):
        cnt += int(S.survives(nA[i, :, None] * nB, tau).sum())
    return cnt / bd ** 3


def tau_for_valid_ratio(nA, nB, target: float, iters: int = 20, tol: float = 0.01):
    """Binary search for tau whose valid ratio is within ``tol`` of ``target``.

    Search space [0, k * ave], ave the mean norm product; the first probe is
    tau = ave; k starts at 1 and grows by one while k * ave still leaves a
    valid ratio above the target.  Stops after ``iters`` probes or within
    ``tol`` (absolute, in ratio units).  Returns (tau, valid_ratio, probes).
    """
    ave = mean_norm_product(nA, nB)
    k = 1
    while valid_ratio_at(nA, nB, k * ave) > target and k < 10 ** 6:
        k += 1
    lo, hi = 0.0, k * ave
    tau = min(ave, hi)
    vr = valid_ratio_at(nA, nB, tau)
    probes = 1
    while abs(vr - target) > tol and probes < iters:
        if vr > target:
            lo = tau
        else:
            hi = tau
        tau = 0.5 * (lo + hi)
        vr = valid_ratio_at(nA, nB, tau)
        probes += 1
    return tau, vr, probes


# ---------------------------------------------------------------------------
# Log histogram of block-norm products (learned-tau features)
# ---------------------------------------------------------------------------

def frobenius_from_normmap(nX: np.ndarray) -> float:
    """||X||_F recovered from its leaf norms: sqrt(sum nX[I,K]^2)."""
    return math.sqrt(math.fsum((nX * nX).ravel().tolist()))


def inv_norm_product(nA, nB) -> float:
    """fl(1 / fl(||A||_F ||B||_F)), both norms from the normmaps."""
    ab = frobenius_from_normmap(nA) * frobenius_from_normmap(nB)
    return 1.0 / ab if ab > 0 else 0.0


def hist_bin(p: np.ndarray, inv: float) -> np.ndarray:
    """Bin t = clamp(floor(-log2 r), 0, 63) of r = fl(p * inv); r = 0 -> 63.

    With r = m 2^e (frexp, m in [0.5, 1)): -log2 r lies in (-e, 1 - e], so
    floor(-log2 r) = -e, or 1 - e when m is exactly 0.5.
    """
    r = np.asarray(p, dtype=np.float64) * inv
    m, e = np.frexp(r)
    t = -e.astype(np.int64) + (m == 0.5)
    t = np.clip(t, 0, HIST_BINS - 1)
    return np.where(r > 0, t, HIST_BINS - 1)


def norm_product_histogram(nA, nB) -> np.ndarray:
    """64-bin histogram of log2(p / (||A|| ||B||)) over all BDIM^3 triples, summing to 1."""
    bd = nA.shape[0]
    inv = inv_norm_product(nA, nB)
    counts = np.zeros(HIST_BINS, dtype=np.int64)
    for i in range(bd):
        t = hist_bin(nA[i, :, None] * nB, inv)
        counts += np.bincount(t.ravel(), minlength=HIST_BINS)
    return counts / float(bd ** 3)


def mlp_features(hist: np.ndarray, target_rel_err: float) -> np.ndarray:
    """MLP input: the 64 bins followed by log10 of the target relative error."""
    return np.concatenate([np.asarray(hist, dtype=np.float64), [math.log10(target_rel_err)]])


# ---------------------------------------------------------------------------
# Bisection on the achieved error (fallback and arbiter of learned tau)
# ---------------------------------------------------------------------------

def bisect_tau(err_fn, eps: float, tau0: float, max_steps: int = 40, ratio: float = 1.01):
    """Largest tested tau whose error stays <= eps.

    Brackets in log tau: ``lo`` (error <= eps, tau = 0 counts as exact) and
    ``hi`` (error > eps).  From ``tau0`` the bracket expands by factors of 10,
    then bisects geometrically until hi / lo <= ratio or ``max_steps``
    evaluations.  Returns (tau, evaluations).
    """
    evals = 0

    def ok(t):
        nonlocal evals
        evals += 1
        return err_fn(t) <= eps

    lo, hi = 0.0, float(tau0)
    if ok(hi):
        lo = hi
        hi = hi * 10.0
        while evals < max_steps and ok(hi):
            lo, hi = hi, hi * 10.0
        if evals >= max_steps:
            return lo, evals
    else:
        t = hi / 10.0
        while evals < max_steps and t > 0:
            if ok(t):
                lo = t
                break
            hi, t = t, t / 10.0
        if lo == 0.0:
            return 0.0, evals
    while hi / lo > ratio and evals < max_steps:
        mid = math.sqrt(lo * hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo, evals
