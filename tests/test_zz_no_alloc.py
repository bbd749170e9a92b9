"""The allocation-free FP32 entry point agrees with the regular entry points.

spamm_multiply_fp32_noalloc is for callers that cannot allocate device memory
where they need a product (for example under a host framework that already
owns the device memory pool).  It keeps its scratch in a static device array
shared by all calls, so this test makes two different calls in a row through
the C ABI and checks both against normmap + plan + multiply.  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import spamm as S

pytestmark = pytest.mark.gpu

FP32_REL_TOL = 1e-5


def _regular(A, B, leaf, tau):
    C, _ = P.spamm(A, B, leaf, tau)
    torch.cuda.synchronize()
    return C.cpu().numpy().astype(np.float64)


def test_noalloc_two_calls_match_regular_entry_points():
    lib = P.lib()
    cases = [(1000, 64, 1e-4, synth.alg_decay_signed, 3.0, 71),
             (2048, 32, 1e-7, synth.exp_decay_normal, 0.2, 72)]
    outs, inputs = [], []
    for n, leaf, tau, gen, rate, seed in cases:
        A = torch.from_numpy(gen(n, rate, seed)).cuda()
        B = torch.from_numpy(gen(n, rate, seed + 1)).cuda()
        C = torch.full_like(A, float("nan"))
        rc = lib.spamm_multiply_fp32_noalloc(ctypes.c_void_p(A.data_ptr()),
                                             ctypes.c_void_p(B.data_ptr()),
                                             ctypes.c_void_p(C.data_ptr()), n, leaf, tau,
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        outs.append(C)
        inputs.append((A, B, leaf, tau))
    torch.cuda.synchronize()
    for C, (A, B, leaf, tau) in zip(outs, inputs):
        got = C.cpu().numpy().astype(np.float64)
        ref = _regular(A, B, leaf, tau)
        assert np.isfinite(got).all()
        assert S.frobenius(got - ref) <= FP32_REL_TOL * S.frobenius(ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = P.lib()
    A = torch.zeros((4160, 4160), device="cuda")
    B = torch.zeros_like(A)
    C = torch.full_like(A, 3.0)
    rc = lib.spamm_multiply_fp32_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                         ctypes.c_void_p(C.data_ptr()), 4160, 64, 0.0, None)
    assert rc == 2                      # SPAMM_ERR_UNSUPPORTED: ceil(4160/64) = 65 > 64
    torch.cuda.synchronize()
    assert bool((C == 3.0).all())       # nothing was enqueued
