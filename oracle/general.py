"""FP64 oracle for the general SpAMM forms: C = alpha*A*B + beta*C on rectangular
operands, and chained products for matrix powers.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 2 states the problem as C = alpha*A*B + beta*C with general A, B, C and
then fixes alpha = 1, beta = 0 and square N x N operands for the rest of the
paper.  This module keeps the general statement:

* A is M x K, B is K x N, C is M x N, all zero padded to whole leaf blocks; the
  block grids are bm x bk (A) and bk x bn (B), bm = ceil(M/leaf) and so on.
* The skip rule is the square one, triple by triple: block product
  A[i,k] B[k,j] is formed iff !(nA[i,k] * nB[k,j] < tau), nA, nB the Eq. 2 norms.
* result = alpha * sum over surviving k of A[i,k] B[k,j]  +  beta * C_in.
  With beta = 0 the old C is not read (so NaN or Inf in it do not propagate),
  as in a BLAS GEMM.

Algorithm 1 recurses on square quadtrees; a rectangular pair is the square
pair zero-padded to a common size, whose extra blocks have norm 0.  Since the
norm of a node bounds the norms of its children, the recursion forms exactly
the leaf triples that pass their own test (the same argument as for the square
form), so the flat rule above is what the recursion computes.

The chained form serves matrix powers, the use of the ergo experiment in
Section 4.3, which does not say how the power is formed; both readings are kept:
repeated squaring, X_{t+1} = SpAMM(X_t, X_t, tau), and repeated multiplication,
X_{t+1} = SpAMM(X_t, A, tau).  X_0 = A; each X_t is stored in FP32 as a GPU
chain stores it, and the norm map of X_{t+1} is taken from that stored matrix.
"""
from __future__ import annotations

import math

import numpy as np

from . import spamm as S


def grid(rows: int, cols: int, leaf: int) -> tuple[int, int]:
    """Block grid (ceil(rows/leaf), ceil(cols/leaf)) of a zero-padded rows x cols matrix."""
    return S.num_blocks(rows, leaf), S.num_blocks(cols, leaf)


def padded_rect(x: np.ndarray, leaf: int) -> np.ndarray:
    """FP64 copy of ``x`` zero padded to whole leaf blocks in both dimensions."""
    r, c = x.shape
    gr, gc = grid(r, c, leaf)
    p = np.zeros((gr * leaf, gc * leaf), dtype=np.float64)
    p[:r, :c] = x
    return p


def normmap_rect(x: np.ndarray, leaf: int) -> np.ndarray:
    """Eq. 2 for every leaf block of a rectangular matrix: sqrt of the exactly rounded sum
    of squares (FP32 squares are exact in FP64; math.fsum rounds the sum once)."""
    p = padded_rect(x, leaf)
    gr, gc = grid(x.shape[0], x.shape[1], leaf)
    out = np.empty((gr, gc), dtype=np.float64)
    for i in range(gr):
        for k in range(gc):
            blk = p[i * leaf:(i + 1) * leaf, k * leaf:(k + 1) * leaf]
            out[i, k] = math.sqrt(math.fsum((blk * blk).ravel().tolist()))
    return out


def survivors_rect(nA: np.ndarray, nB: np.ndarray, tau: float) -> np.ndarray:
    """surv[i, k, j] = !(nA[i,k] * nB[k,j] < tau) for nA [bm, bk], nB [bk, bn]."""
    if nA.shape[1] != nB.shape[0]:
        raise ValueError("inner block counts differ")
    surv = np.zeros((nA.shape[0], nA.shape[1], nB.shape[1]), dtype=bool)
    for i in range(nA.shape[0]):
        surv[i] = S.survives(nA[i, :, None] * nB, tau)
    return surv


def product_rect(a: np.ndarray, b: np.ndarray, leaf: int, surv: np.ndarray) -> np.ndarray:
    """sum over surviving k of A[i,k] B[k,j] in FP64, k ascending; M x N (padding removed)."""
    m, kdim = a.shape
    n = b.shape[1]
    pa, pb = padded_rect(a, leaf), padded_rect(b, leaf)
    bm, bk = grid(m, kdim, leaf)
    bn = S.num_blocks(n, leaf)
    c = np.zeros((bm * leaf, bn * leaf))
    for i in range(bm):
        for j in range(bn):
            acc = np.zeros((leaf, leaf))
            for k in np.nonzero(surv[i, :, j])[0]:
                acc += (pa[i * leaf:(i + 1) * leaf, k * leaf:(k + 1) * leaf]
                        @ pb[k * leaf:(k + 1) * leaf, j * leaf:(j + 1) * leaf])
            c[i * leaf:(i + 1) * leaf, j * leaf:(j + 1) * leaf] = acc
    return c[:m, :n]


def skipped_bound_rect(nA: np.ndarray, nB: np.ndarray, surv: np.ndarray) -> float:
    """sqrt(sum over tiles of (sum of skipped p_ikj)^2): bounds ||AB - product_rect||_F."""
    tiles = []
    for i in range(nA.shape[0]):
        p = nA[i, :, None] * nB
        tiles.append(np.where(surv[i], 0.0, p).sum(axis=0))
    t = np.concatenate(tiles)
    return math.sqrt(math.fsum((t * t).tolist()))


def spamm_general(a: np.ndarray, b: np.ndarray, leaf: int, tau: float, alpha: float = 1.0,
                  beta: float = 0.0, c_in: np.ndarray | None = None) -> dict:
    """C = alpha * SpAMM(A, B, tau) + beta * C_in (Section 2 statement), FP64.

    Returns dict(C, surv, nA, nB, S, bound2) where bound2 bounds
    ||alpha AB - alpha SpAMM(A, B)||_F / |alpha|."""
    if a.shape[1] != b.shape[0]:
        raise ValueError("inner dimensions differ")
    nA, nB = normmap_rect(a, leaf), normmap_rect(b, leaf)
    surv = survivors_rect(nA, nB, tau)
    c = alpha * product_rect(a, b, leaf, surv)
    if beta != 0.0:
        if c_in is None or c_in.shape != c.shape:
            raise ValueError("beta != 0 needs C_in of shape M x N")
        c = c + beta * np.asarray(c_in, dtype=np.float64)
    return {"C": c, "surv": surv, "nA": nA, "nB": nB, "S": int(surv.sum()),
            "bound2": skipped_bound_rect(nA, nB, surv)}


def spamm_general_recursive(a: np.ndarray, b: np.ndarray, leaf: int, tau: float):
    """Algorithm 1 on the zero-padded square embedding of a rectangular pair.

    Returns (A B restricted to the surviving triples, surv [bm, bk, bn]) taken from the
    square recursion (oracle.spamm.spamm_recursive) on matrices of side max(M, K, N)."""
    m, kdim = a.shape
    n = b.shape[1]
    side = max(m, kdim, n)
    sa = np.zeros((side, side), dtype=np.float32)
    sb = np.zeros((side, side), dtype=np.float32)
    sa[:m, :kdim] = a
    sb[:kdim, :n] = b
    c, surv = S.spamm_recursive(sa, sb, leaf, tau)
    bm, bk = grid(m, kdim, leaf)
    bn = S.num_blocks(n, leaf)
    return c[:m, :n], surv[:bm, :bk, :bn]


def power_chain(a: np.ndarray, leaf: int, tau: float, steps: int,
                squaring: bool = True) -> list[dict]:
    """Chained SpAMM from X_0 = A (square): X_{t+1} = fl32(SpAMM(X_t, X_t, tau)) when
    ``squaring`` (X_t = A^(2^t) up to pruning and rounding), else fl32(SpAMM(X_t, A, tau))
    (X_t = A^(t+1)).

    Entry t of the result describes the product that made X_{t+1}: dict(X = X_{t+1} as FP32,
    C = its FP64 value before the FP32 rounding, surv, norms = the norm map of X_t it was
    planned with, S, bound2)."""
    a32 = np.asarray(a, dtype=np.float32)
    x = a32
    out = []
    for _ in range(steps):
        r = S.spamm(x, x if squaring else a32, leaf, tau)
        x_next = r["C"].astype(np.float32)
        out.append({"X": x_next, "C": r["C"], "surv": r["surv"], "norms": r["nA"],
                    "S": r["S"], "bound2": r["bound2"]})
        x = x_next
    return out
