"""Edge cases through the C ABI: degenerate sizes, special values, argument errors, plan reuse,
ragged tensor-core shapes, and the bounded-wait self-test (failure detection without a fault)."""
import math

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import precision as OP
from oracle import spamm as S
from tests.gpu_helpers import dev, host, plan_mask

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,leaf", [(P.FP32, 32), (P.BF16, 64), (P.TF32X3, 128)])
def test_one_by_one(prec, leaf):
    a = np.array([[3.0]], dtype=np.float32)
    b = np.array([[-2.5]], dtype=np.float32)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    assert host(nA)[0, 0] == 3.0 and host(nB)[0, 0] == 2.5
    C = torch.full_like(A, float("nan"))
    P.Plan(1, leaf, prec).plan_multiply(nA, nB, 7.5, A, B, C)     # tie: multiplied
    assert host(C)[0, 0] == -7.5
    P.Plan(1, leaf, prec).plan_multiply(nA, nB, 7.5000001, A, B, C)   # skipped: zero
    assert host(C)[0, 0] == 0.0


@pytest.mark.parametrize("prec", [P.FP32, P.BF16_SPLIT])
def test_zero_matrices(prec):
    n, leaf = 200, 64
    A = torch.zeros(n, n, device="cuda")
    B = torch.zeros(n, n, device="cuda")
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    for tau, surv in ((0.0, 4 ** 3), (1e-30, 0)):
        C = torch.full_like(A, float("nan"))
        pl = P.Plan(n, leaf, prec)
        pl.plan_multiply(nA, nB, tau, A, B, C, 1e-5)
        assert pl.stats()["survivors"] == surv
        assert not host(C).any()


def test_nan_block_propagates():
    """A NaN block's norm is NaN: its triples always survive and NaN reaches exactly the rows
    of C that the block multiplies into (as in a GEMM)."""
    n, leaf = 256, 64
    a = synth.exp_decay_normal(n, 0.5, 3)
    b = synth.exp_decay_normal(n, 0.5, 4)
    a[70, 130] = np.nan                         # block (1, 2)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    assert math.isnan(host(nA)[1, 2])
    C = torch.full_like(A, 0.0)
    pl = P.Plan(n, leaf, P.FP32)
    pl.plan_multiply(nA, nB, 1e30, A, B, C)       # only the NaN triples survive
    surv, _ = plan_mask(pl)
    assert surv[1, 2, :].all() and surv.sum() == 4
    c = host(C)
    assert np.isnan(c[70]).all()
    assert not np.isnan(np.delete(c, 70, axis=0)).any()


def test_argument_errors():
    n = 128
    A = torch.zeros(n, n, device="cuda")
    B = torch.zeros(n, n, device="cuda")
    C = torch.zeros(n, n, device="cuda")
    nA, nB = P.spamm_normmap(A, 64), P.spamm_normmap(B, 64)
    with pytest.raises(P.SpammError) as e:
        P.Plan(n, 32, P.BF16)                     # tensor cores need leaf 64 or 128
    assert e.value.code == 2
    pl = P.Plan(n, 64, P.FP32)
    with pytest.raises(P.SpammError) as e:
        pl.plan(nA, nB, float("nan"))
    assert e.value.code == 1
    with pytest.raises(P.SpammError) as e:
        pl.plan(nA, nB, -1.0)
    assert e.value.code == 1
    pl.plan(nA, nB, 0.5)
    with pytest.raises(P.SpammError) as e:
        pl.multiply(A, B, A)                       # output aliases an input
    assert e.value.code == 1
    flat = torch.zeros(n * n + 1, device="cuda")
    with pytest.raises(P.SpammError) as e:
        pl.multiply(flat[1:].view(n, n), B, C)     # 4-byte misaligned
    assert e.value.code == 1
    with pytest.raises(P.SpammError) as e:
        P.spamm_normmap(A, 48)                     # leaf
    assert e.value.code == 2


def test_plan_reuse_across_tau():
    n, leaf = 500, 64
    a = synth.alg_decay_signed(n, 2.5, 8)
    b = synth.alg_decay_signed(n, 2.5, 9)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    oA, oB = S.normmap(a, leaf), S.normmap(b, leaf)
    pl = P.Plan(n, leaf, P.FP32)
    C = torch.empty_like(A)
    for tau in (1e-1, 1e-4, 1e-2, 0.0, 1e-3):
        pl.plan_multiply(nA, nB, tau, A, B, C)
        surv = S.flat_survivors(oA, oB, tau)
        assert pl.stats()["survivors"] == int(surv.sum())
        ref = S.multiply_with_skipset(a, b, leaf, surv)
        assert np.linalg.norm(host(C) - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,leaf,mode", [(203, 128, OP.BF16), (131, 64, OP.FP16_SPLIT),
                                         (97, 64, OP.TF32X3)])
def test_tensor_ragged_unaligned(n, leaf, mode):
    """n not a multiple of 4 (no 16-byte rows): scalar paths of rounding and epilogue."""
    a = synth.exp_decay_normal(n, 0.05, n)
    b = synth.exp_decay_normal(n, 0.05, n + 1)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    pl = P.Plan(n, leaf, mode)
    C = torch.full_like(A, float("nan"))
    pl.plan_multiply(nA, nB, 0.0, A, B, C, 1e-7)
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    surv, flags = plan_mask(pl)
    got = host(C).astype(np.float64)
    emu = OP.emulated_multiply(a, b, leaf, surv, mode, flags)
    bound = OP.accumulation_bound(S.normmap(a, leaf), S.normmap(b, leaf), surv, mode, leaf)
    assert np.isfinite(got).all()
    assert np.linalg.norm(got - emu) <= bound


def test_bounded_wait_gives_up_and_reports():
    """Failure detection without a fault: the multiply's and the norm map's wait routines on
    a phase nothing completes give up after their limit, and the status word reports
    SPAMM_ERR_TIMEOUT."""
    assert P.spamm_last_device_status() in (0, 5)  # clear
    elapsed = P.spamm_selftest_bounded_wait(20_000_000)
    assert 20_000_000 <= elapsed < 2_000_000_000
    assert P.spamm_last_device_status() == 5       # SPAMM_ERR_TIMEOUT, then cleared
    assert P.spamm_last_device_status() == 0
    # the context is still usable
    x = torch.ones(64, 64, device="cuda")
    assert host(P.spamm_normmap(x, 32))[0, 0] == 32.0
