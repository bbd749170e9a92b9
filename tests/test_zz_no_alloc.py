"""The allocation-free FP32 entry point gives exactly the bits of the regular entry points.

spamm_multiply_fp32_noalloc is for callers that cannot allocate device memory
where they need a product (for example under a host framework that already
owns the device memory pool, or a plugin host that forbids allocation).  It
keeps its scratch in a static device array shared by all calls and runs the
same norm map, plan and SIMT multiply as spamm_normmap + spamm_plan +
spamm_multiply (SPAMM_FP32), so its C must be bit-identical to theirs.  This
test makes three different calls in a row through the C ABI (the static
scratch keeps the previous call's contents, so stale data would show) --
including a size whose rows are not 16-byte aligned (n % 4 != 0), which takes
the norm map's unaligned path -- and checks each against the regular entry
points bit for bit, and one against the FP64 oracle.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import precision as OP
from oracle import spamm as S

pytestmark = pytest.mark.gpu

FP32_REL_TOL = 1e-5


def _noalloc(A, B, C, n, leaf, tau):
    lib = P.lib()
    return lib.spamm_multiply_fp32_noalloc(ctypes.c_void_p(A.data_ptr()),
                                           ctypes.c_void_p(B.data_ptr()),
                                           ctypes.c_void_p(C.data_ptr()), n, leaf, tau,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_calls_in_a_row_equal_regular_entry_points():
    cases = [(1000, 64, 1e-4, synth.alg_decay_signed, 3.0, 71),
             (2048, 32, 1e-7, synth.exp_decay_normal, 0.2, 72),
             (1001, 32, 1e-5, synth.exp_decay_normal, 0.05, 73)]
    outs, inputs = [], []
    for n, leaf, tau, gen, rate, seed in cases:
        a, b = gen(n, rate, seed), gen(n, rate, seed + 1)
        A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        C = torch.full_like(A, float("nan"))
        assert _noalloc(A, B, C, n, leaf, tau) == 0
        outs.append(C)
        inputs.append((a, b, A, B, leaf, tau))
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    for q, (C, (a, b, A, B, leaf, tau)) in enumerate(zip(outs, inputs)):
        ref, plan = P.spamm(A, B, leaf, tau)
        torch.cuda.synchronize()
        assert torch.equal(C, ref), f"case {q}: differs from normmap + plan + multiply"
        if q == 2:   # the unaligned case against the FP64 oracle, tile by tile
            nA, nB = S.normmap(a, leaf), S.normmap(b, leaf)
            surv = S.flat_survivors(nA, nB, tau)
            assert plan.stats()["survivors"] == int(surv.sum())
            exact = S.multiply_with_skipset(a, b, leaf, surv)
            got = C.cpu().numpy().astype(np.float64)
            assert S.frobenius(got - exact) <= FP32_REL_TOL * S.frobenius(exact)
            t = OP.accumulation_tile_bounds(nA, nB, surv, OP.FP32, leaf)
            assert np.all(OP.tile_errors(got, exact, leaf) <= t)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    A = torch.zeros((4160, 4160), device="cuda")
    B = torch.zeros_like(A)
    C = torch.full_like(A, 3.0)
    assert _noalloc(A, B, C, 4160, 64, 0.0) == 2   # SPAMM_ERR_UNSUPPORTED: ceil(4160/64) = 65 > 64
    torch.cuda.synchronize()
    assert bool((C == 3.0).all())                  # nothing was enqueued
