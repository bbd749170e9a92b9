"""FP64 oracle for SpAMM: norms, Algorithm 1, the flat skip rule, errors and bounds.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation (Section 3, notation paragraph): leaf size ``leaf`` (the paper's
LoNum), ``bd = ceil(n / leaf)`` blocks per dimension (BDIM), block (I, K) is
the leaf x leaf sub-matrix starting at row I*leaf, column K*leaf; matrices are
zero padded to bd*leaf.  ``nA[I, K] = ||A[I, K]||_F`` (Eq. 2).

Skip rule (Algorithm 1 tests, Algorithm 2 bitmap): a block product is
multiplied when ``||A_ik||_F * ||B_kj||_F >= tau``.  Read as "skip iff the
product is < tau", so a tie is multiplied and a NaN product is never skipped.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# Block grid and norms (Section 3 notation; Eq. 2)
# ---------------------------------------------------------------------------

def num_blocks(n: int, leaf: int) -> int:
    """BDIM = ceil(n / LoNum): blocks per dimension after zero padding."""
    return -(-n // leaf)


def padded64(x: np.ndarray, leaf: int) -> np.ndarray:
    """Float64 copy of ``x`` zero padded to a multiple of ``leaf`` (Section 3 notation)."""
    n = x.shape[0]
    m = num_blocks(n, leaf) * leaf
    p = np.zeros((m, m), dtype=np.float64)
    p[:n, :n] = x
    return p


def block(p: np.ndarray, leaf: int, i: int, k: int) -> np.ndarray:
    """Sub-matrix X[i, k] of a padded matrix (starts at row i*leaf, column k*leaf)."""
    return p[i * leaf:(i + 1) * leaf, k * leaf:(k + 1) * leaf]


def leaf_sumsq(x: np.ndarray, leaf: int) -> np.ndarray:
    """Sum of squares of every leaf block, correctly rounded to FP64.

    Squares of FP32 entries are exact in FP64 (48-bit significands); the sum of
    a block is formed by ``math.fsum`` (exactly rounded), so the result is the
    FP64 value nearest the exact sum of squares.
    """
    p = padded64(x, leaf)
    bd = num_blocks(x.shape[0], leaf)
    s = np.empty((bd, bd), dtype=np.float64)
    for i in range(bd):
        for k in range(bd):
            blk = block(p, leaf, i, k)
            s[i, k] = math.fsum((blk * blk).ravel().tolist())
    return s


def normmap(x: np.ndarray, leaf: int) -> np.ndarray:
    """Eq. 2 per leaf block: normmap[I, K] = sqrt(sum of squares of X[I, K]) (Section 3.1)."""
    return np.sqrt(leaf_sumsq(x, leaf))


def frobenius(x: np.ndarray) -> float:
    """||X||_F with an exactly rounded sum of squares."""
    x64 = np.asarray(x, dtype=np.float64)
    return math.sqrt(math.fsum((x64 * x64).ravel().tolist()))


# ---------------------------------------------------------------------------
# Flat leaf-level rule (Section 3.1 re-design; Algorithm 2 bitmap)
# ---------------------------------------------------------------------------

def survives(p: np.ndarray | float, tau: float):
    """Multiply iff the norm product is >= tau (Algorithm 1 tests).  NaN survives."""
    return ~(np.asarray(p) < tau)


def flat_survivors(nA: np.ndarray, nB: np.ndarray, tau: float) -> np.ndarray:
    """Boolean mask surv[i, k, j] = !(nA[i,k] * nB[k,j] < tau) over all leaf triples."""
    bd = nA.shape[0]
    surv = np.zeros((bd, bd, bd), dtype=bool)
    for i in range(bd):
        prod = nA[i, :, None] * nB          # prod[k, j] = nA[i,k] * nB[k,j]
        surv[i] = survives(prod, tau)
    return surv


def triple_products(nA: np.ndarray, nB: np.ndarray) -> np.ndarray:
    """p[i, k, j] = nA[i,k] * nB[k,j] (FP64) for all triples (small bd only)."""
    return nA[:, :, None] * nB[None, :, :]


def multiply_with_skipset(a: np.ndarray, b: np.ndarray, leaf: int,
                          surv: np.ndarray) -> np.ndarray:
    """C[i,j] = sum over k with surv[i,k,j] of A[i,k] B[k,j], FP64, beta = 0 (Section 3.3).

    Returns the n x n result (padding removed).  k is visited in increasing order.
    """
    n = a.shape[0]
    pa, pb = padded64(a, leaf), padded64(b, leaf)
    bd = num_blocks(n, leaf)
    c = np.zeros_like(pa)
    for i in range(bd):
        for j in range(bd):
            ks = np.nonzero(surv[i, :, j])[0]
            if ks.size == 0:
                continue
            acc = np.zeros((leaf, leaf))
            for k in ks:
                acc += block(pa, leaf, i, k) @ block(pb, leaf, k, j)
            c[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf] = acc
    return c[:n, :n]


def dense_reference(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The exact product AB in FP64 (library matmul on FP64 copies)."""
    return np.asarray(a, dtype=np.float64) @ np.asarray(b, dtype=np.float64)


# ---------------------------------------------------------------------------
# Recursive quadtree SpAMM (Eq. 1 split, Algorithm 1)
# ---------------------------------------------------------------------------

class Quadtree:
    """Norms of every quadtree node (Eq. 1), built from the leaf sums of squares.

    The leaf grid is padded with zero blocks to ``bq = 2^h`` leaves per side.
    ``sumsq[t]`` holds the sums of squares of the nodes that span 2^t x 2^t
    leaves; a parent's sum is ((s00 + s01) + s10) + s11 of its four children,
    so a child's norm never exceeds its parent's in floating point either.
    """

    def __init__(self, leaf_s: np.ndarray):
        bd = leaf_s.shape[0]
        self.height = max(0, math.ceil(math.log2(bd))) if bd > 1 else 0
        bq = 1 << self.height
        s0 = np.zeros((bq, bq), dtype=np.float64)
        s0[:bd, :bd] = leaf_s
        self.sumsq = [s0]
        for _ in range(self.height):
            c = self.sumsq[-1]
            parent = ((c[0::2, 0::2] + c[0::2, 1::2]) + c[1::2, 0::2]) + c[1::2, 1::2]
            self.sumsq.append(parent)
        self.norms = [np.sqrt(s) for s in self.sumsq]


def spamm_recursive(a: np.ndarray, b: np.ndarray, leaf: int, tau: float):
    """Algorithm 1 on the quadtree of leaf blocks.

    Returns ``(C, surv)``: the FP64 product (n x n) and the boolean mask of leaf
    triples (i, k, j), i, k, j < bd, whose leaf product was formed.

    At a node pair (A node at (ai, ak), B node at (ak, bj), scale t) the four
    output quadrants are C_ij = T0 + T1 with T_k = SpAMM(A_ik, B_kj) when
    ||A_ik||_F ||B_kj||_F >= tau, else 0; at the leaf scale C = AB.  The root
    pair itself is not tested.  With a single leaf block (bd = 1) the root is
    the leaf; the flat rule of Section 3.1 tests that one pair, and so does
    this function, so that both forms agree for every bd.
    """
    n = a.shape[0]
    pa, pb = padded64(a, leaf), padded64(b, leaf)
    bd = num_blocks(n, leaf)
    qa, qb = Quadtree(leaf_sumsq(a, leaf)), Quadtree(leaf_sumsq(b, leaf))
    surv = np.zeros((bd, bd, bd), dtype=bool)

    def leaf_product(i, k, j):
        if i < bd and k < bd and j < bd:
            surv[i, k, j] = True
            return block(pa, leaf, i, k) @ block(pb, leaf, k, j)
        return None  # a padded leaf: all zeros

    def rec(t, ai, ak, bj):
        """SpAMM of A node (ai, ak) and B node (ak, bj) at scale t; None stands for 0."""
        if t == 0:
            return leaf_product(ai, ak, bj)
        half = (1 << (t - 1)) * leaf
        out = None
        for i in range(2):
            for j in range(2):
                terms = []
                for k in range(2):
                    ca, cb = (2 * ai + i, 2 * ak + k), (2 * ak + k, 2 * bj + j)
                    if not (qa.norms[t - 1][ca] * qb.norms[t - 1][cb] < tau):
                        terms.append(rec(t - 1, ca[0], ca[1], cb[1]))
                    else:
                        terms.append(None)
                t0, t1 = terms
                if t0 is None and t1 is None:
                    cij = None
                elif t0 is None:
                    cij = t1
                elif t1 is None:
                    cij = t0
                else:
                    cij = t0 + t1
                if cij is not None:
                    if out is None:
                        out = np.zeros((2 * half, 2 * half))
                    out[i * half:(i + 1) * half, j * half:(j + 1) * half] = cij
        return out

    h = qa.height
    if h == 0:
        # Single leaf: apply the leaf-level test (Section 3.1 form).
        root = (leaf_product(0, 0, 0)
                if not (qa.norms[0][0, 0] * qb.norms[0][0, 0] < tau) else None)
    else:
        root = rec(h, 0, 0, 0)
    c = np.zeros((bd * leaf, bd * leaf))
    if root is not None:
        m = min(root.shape[0], bd * leaf)
        c[:m, :m] = root[:m, :m]
    return c[:n, :n], surv


# ---------------------------------------------------------------------------
# Statistics, errors (Eq. 5) and skipped-product bounds
# ---------------------------------------------------------------------------

def valid_counts(surv: np.ndarray) -> np.ndarray:
    """V[i, j] = number of surviving k for output tile (i, j) (Section 3.5.1)."""
    return surv.sum(axis=1)


def valid_ratio(surv: np.ndarray) -> float:
    """valid ratio = sum V / BDIM^3 (Section 3.5.2)."""
    return float(surv.sum()) / surv.size


def skipped_bounds(nA: np.ndarray, nB: np.ndarray, surv: np.ndarray):
    """(bound1, bound2) over the skipped leaf triples.

    bound1 = sum of p_ikj over skipped triples;
    bound2 = sqrt(sum_ij (sum_{k skipped} p_ikj)^2).
    ||AB - C||_F <= bound2 <= bound1 by the triangle inequality per tile,
    sub-multiplicativity of the Frobenius norm and orthogonality of tiles.
    """
    bd = nA.shape[0]
    b1 = []
    tile = np.zeros((bd, bd))
    for i in range(bd):
        p = nA[i, :, None] * nB                  # [k, j]
        sk = np.where(surv[i], 0.0, p)
        tile[i] = sk.sum(axis=0)
        b1.append(math.fsum(sk.ravel().tolist()))
    return math.fsum(b1), math.sqrt(math.fsum((tile * tile).ravel().tolist()))


def errors(c: np.ndarray, ref: np.ndarray, norm_a: float, norm_b: float):
    """Eq. 5 error E = AB - SpAMM(A, B, tau) in the three normalisations used.

    Returns dict(abs=||E||_F, rel_c=||E||_F/||AB||_F, rel_ab=||E||_F/(||A||_F ||B||_F)).
    """
    e = np.asarray(ref, dtype=np.float64) - np.asarray(c, dtype=np.float64)
    ae = frobenius(e)
    rc = frobenius(ref)
    return {"abs": ae, "rel_c": ae / rc if rc > 0 else (0.0 if ae == 0 else math.inf),
            "rel_ab": ae / (norm_a * norm_b) if norm_a * norm_b > 0 else
            (0.0 if ae == 0 else math.inf)}


def spamm(a: np.ndarray, b: np.ndarray, leaf: int, tau: float):
    """Convenience: flat-rule SpAMM.  Returns dict with C, surv, nA, nB and statistics."""
    nA, nB = normmap(a, leaf), normmap(b, leaf)
    surv = flat_survivors(nA, nB, tau)
    c = multiply_with_skipset(a, b, leaf, surv)
    b1, b2 = skipped_bounds(nA, nB, surv)
    return {"C": c, "surv": surv, "nA": nA, "nB": nB, "S": int(surv.sum()),
            "valid_ratio": valid_ratio(surv), "bound1": b1, "bound2": b2}


# ---------------------------------------------------------------------------
# Block-row samples (bounded CPU timing of the same workload)
# ---------------------------------------------------------------------------

def normmap_rows(x: np.ndarray, leaf: int, rows) -> np.ndarray:
    """Eq. 2 norms of the leaf blocks in block-rows ``rows`` only ([len(rows), bd])."""
    n = x.shape[0]
    bd = num_blocks(n, leaf)
    out = np.zeros((len(rows), bd))
    for r, i in enumerate(rows):
        strip = np.zeros((leaf, bd * leaf))
        lo, hi = i * leaf, min(n, (i + 1) * leaf)
        strip[:hi - lo, :n] = x[lo:hi]
        for k in range(bd):
            blk = strip[:, k * leaf:(k + 1) * leaf]
            out[r, k] = math.sqrt(math.fsum((blk * blk).ravel().tolist()))
    return out


def block64(x: np.ndarray, leaf: int, i: int, k: int) -> np.ndarray:
    """FP64 copy of leaf block X[i, k] of an unpadded n x n matrix, zero padded to leaf x leaf
    (the same values as ``block(padded64(x), ...)`` without copying the whole matrix)."""
    n = x.shape[0]
    out = np.zeros((leaf, leaf))
    r0, c0 = i * leaf, k * leaf
    r1, c1 = min(n, r0 + leaf), min(n, c0 + leaf)
    out[:r1 - r0, :c1 - c0] = x[r0:r1, c0:c1]
    return out


def spamm_rows(a: np.ndarray, b: np.ndarray, leaf: int, tau: float, rows,
               nA_rows: np.ndarray, nB: np.ndarray) -> dict:
    """Block-rows ``rows`` of C by the flat rule: {i: (C strip [leaf, n], surviving (k, j))}."""
    n = a.shape[0]
    bd = num_blocks(n, leaf)
    out = {}
    for r, i in enumerate(rows):
        lo, hi = i * leaf, min(n, (i + 1) * leaf)
        a_strip = np.zeros((leaf, bd * leaf))
        a_strip[:hi - lo, :n] = a[lo:hi]
        surv = survives(nA_rows[r][:, None] * nB, tau)          # [k, j]
        c = np.zeros((leaf, bd * leaf))
        for j in range(bd):
            for k in np.nonzero(surv[:, j])[0]:
                c[:, j * leaf:(j + 1) * leaf] += (a_strip[:, k * leaf:(k + 1) * leaf]
                                                  @ block64(b, leaf, k, j))
        out[i] = (c[:hi - lo, :n], surv)
    return out


def normmap_blocked(x: np.ndarray, leaf: int) -> np.ndarray:
    """Eq. 2 for every leaf block with numpy's FP64 pairwise summation of the exact squares:
    the form for matrices too large for :func:`normmap`'s exactly rounded sums (one leaf-row
    strip at a time).  Not exactly rounded: each sum is within about log2(leaf^2) 2^-53
    relative of the exact one, far inside the 1e-12 band in which skip decisions may differ."""
    n = x.shape[0]
    bd = num_blocks(n, leaf)
    out = np.empty((bd, bd))
    for i in range(bd):
        lo, hi = i * leaf, min(n, (i + 1) * leaf)
        strip = np.zeros((leaf, bd * leaf))
        strip[:hi - lo, :n] = x[lo:hi]
        blocks = (strip * strip).reshape(leaf, bd, leaf).transpose(1, 0, 2).reshape(bd, -1)
        out[i] = np.sqrt(blocks.sum(axis=1))      # contiguous rows: pairwise sums
    return out


def needed_b_rows(nA_rows: np.ndarray, tau: float):
    """Block rows k of B's norm map that can decide a triple of the given block rows of C.

    For tau > 0, a triple (i, k, j) with nA[i, k] = 0 has p = 0 * nB[k, j] = 0 < tau for
    every finite nB[k, j], so it is skipped whatever row k of B holds; only the k with a
    non-zero (or non-finite) nA[i, k] in some sampled row are needed.  Every k is needed
    for tau = 0.  (With a non-finite entry in row k of B, p would be NaN and survive: the
    caller checks that B is finite before relying on this.)
    """
    if not tau > 0.0:
        return np.arange(nA_rows.shape[1])
    return np.nonzero(np.any(nA_rows != 0.0, axis=0))[0]


def normmap_needed(b: np.ndarray, leaf: int, nA_rows: np.ndarray, tau: float) -> np.ndarray:
    """B's [bd, bd] norm map with only the rows :func:`needed_b_rows` computed (Eq. 2, exactly
    rounded sums) and the others 0.  For the sampled block rows of C, :func:`spamm_rows` makes
    the same decisions with it as with the full map when tau > 0 and B is finite (checked)."""
    n = b.shape[0]
    bd = num_blocks(n, leaf)
    ks = needed_b_rows(nA_rows, tau)
    if tau > 0.0 and ks.size < bd and not np.isfinite(b).all():
        ks = np.arange(bd)
    out = np.zeros((bd, bd))
    if ks.size:
        out[ks] = normmap_rows(b, leaf, ks)
    return out
