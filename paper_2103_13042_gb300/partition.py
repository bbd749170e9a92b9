"""Multi-GPU partitions of the product (Section 3.4, Algorithm 4): host logic only.

Row blocks: rank r of W computes output block rows [r0, r1) of C = SpAMM(A, B) from its rows of A
(a row-major view of A) and all of B, with B's norm map computed on every rank.  Each output
tile depends only on its own block row of A and on B, so the ranks exchange nothing.
Algorithm 4 gives the rows of GPU i as a range of i M / N to (i + 1) M / N (printed garbled),
read here as half-open; the split is taken on leaf-block boundaries so that no block row is cut
and every rank's norm map holds whole block rows of A's.

By instance: the instances of a batch are dealt to the ranks longest first (n^3 as the work of
an instance), each to the rank with the least work so far, so the ranks finish together.
"""
from __future__ import annotations


def row_blocks(n: int, leaf: int, world: int) -> list[tuple[int, int]]:
    """[(r0, r1)] per rank: output rows of each rank, whole leaf blocks, covering [0, n) in
    order; a rank gets an empty range when there are fewer block rows than ranks."""
    if n < 1 or leaf < 1 or world < 1:
        raise ValueError("n, leaf and world must be positive")
    bm = -(-n // leaf)
    out = []
    for r in range(world):
        b0, b1 = r * bm // world, (r + 1) * bm // world
        out.append((min(n, b0 * leaf), min(n, b1 * leaf)))
    return out


def instances_by_rank(ns, world: int) -> list[list[int]]:
    """Indices of the batch's instances per rank: longest first (n^3), each to the rank with the
    least work so far (ties to the lower rank); every rank's list in increasing index order."""
    if world < 1:
        raise ValueError("world must be positive")
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(ns)), key=lambda q: (-float(ns[q]) ** 3, q)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += float(ns[i]) ** 3
    return [sorted(x) for x in out]
