"""The multi-GPU form is replicas: each rank runs its own product, the job's time is the
slowest rank's and its throughput the sum over ranks.  The aggregation runs here on CPU
ranks (gloo, world size 2); on GPUs the same calls run over NCCL."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.slowest_rank_ms(1.0 + 2.0 * rank, world, torch.device("cpu"))
    thr = bench.job_throughput(100.0, ms, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, thr))


def test_slowest_rank_and_job_throughput_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.0, 3.0]          # every rank sees the slowest time
    assert res[0][2] == pytest.approx(100.0 * 2 / 3e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(2.5, 1, None) == 2.5
    assert bench.job_throughput(10.0, 2.0, 1) == pytest.approx(5000.0)


def test_reference_arm_other_ranks_exit_silently():
    """Under torchrun only rank 0 runs the reference arm; the others exit 0 with no output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    """Rank 0 of the reference arm times the oracle on the host cores and prints one JSON line
    with the contract's keys (a small case here: the N = 2048 algebraic-decay workload, at
    least 8 output block-rows per step, one per worker process)."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "c2", "--n", "2048", "--steps", "1", "--warmup", "3",
                        "--ref-rows", "8"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["warmup"] >= 3 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["unit"].startswith("TFLOP/s")
    assert d["dtype"] == "f64" and d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["nproc"] >= cb["cores"] and cb["single_thread"]["cores"] == 1
    assert " of 32 output block rows" in cb["sample"] and d["config"]["n"] == 2048
    # the step is a bounded sample of the job (fewer block rows than the whole product); its
    # wall time also holds the single-thread leg, so it is not compared with the extrapolation
    import re
    sampled = int(re.search(r"(\d+) of 32 output block rows", cb["sample"]).group(1))
    assert 1 <= sampled < 32 and d["ms_per_step_full_job_extrapolated"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
