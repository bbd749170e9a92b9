"""The multi-GPU partitions (row blocks of Algorithm 4, instances of a batch), on the CPU: the
row ranges cover the output exactly on leaf boundaries, the instance deal is balanced, and two
gloo ranks that each compute their own block rows (the oracle standing in for each rank's GPU)
reproduce the whole product with no exchange on the data path (the gather is the test's)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2103_13042_gb300 import partition as PT  # noqa: E402


@pytest.mark.parametrize("n,leaf,world", [(1000, 64, 3), (32768, 128, 8), (100, 32, 8), (64, 64, 2)])
def test_row_blocks_cover_on_leaf_boundaries(n, leaf, world):
    rb = PT.row_blocks(n, leaf, world)
    assert len(rb) == world and rb[0][0] == 0 and rb[-1][1] == n
    for (a0, a1), (b0, _) in zip(rb, rb[1:]):
        assert a1 == b0 and a0 <= a1
    for r0, r1 in rb:
        assert r0 % leaf == 0 and (r1 % leaf == 0 or r1 == n)
    bm = -(-n // leaf)
    sizes = [-(-(r1 - r0) // leaf) for r0, r1 in rb]
    assert sum(sizes) == bm and max(sizes) - min(sizes) <= 1


def test_instances_by_rank_balanced():
    g = np.random.Generator(np.random.PCG64(3))
    ns = [int(x) for x in np.exp(g.uniform(np.log(256), np.log(4096), 256)).round()]
    parts = PT.instances_by_rank(ns, 8)
    assert sorted(i for p in parts for i in p) == list(range(256))
    loads = [sum(ns[i] ** 3 for i in p) for p in parts]
    assert max(loads) <= 1.05 * (sum(loads) / 8) + max(ns) ** 3
    assert PT.instances_by_rank([5, 9], 4) == [[1], [0], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import synth
    from oracle import spamm as S
    from paper_2103_13042_gb300 import partition as P2
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, leaf, tau = 300, 32, 1e-3
    a = synth.exp_decay_normal(n, 0.1, 5)
    b = synth.exp_decay_normal(n, 0.1, 6)
    r0, r1 = P2.row_blocks(n, leaf, world)[rank]
    rows = list(range(r0 // leaf, -(-r1 // leaf)))
    nB = S.normmap(b, leaf)                         # replicated on every rank
    part = S.spamm_rows(a, b, leaf, tau, rows, S.normmap_rows(a, leaf, rows), nB)
    mine = np.concatenate([part[i][0] for i in rows]) if rows else np.zeros((0, n))
    got = [None] * world
    dist.all_gather_object(got, (r0, r1, mine))     # the test's check, not the data path
    if rank == 0:
        full = np.zeros((n, n))
        for s0, s1, blk in got:
            full[s0:s1] = blk
        want = S.spamm(a, b, leaf, tau)["C"]
        q.put(bool(np.array_equal(full, want)))
    dist.barrier()
    dist.destroy_process_group()


def test_row_block_ranks_reproduce_the_product():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ok = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ok
