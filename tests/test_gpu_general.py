"""The general form of Section 2 and chained products, through the C ABI, against the oracle
(oracle.general): C = alpha * SpAMM(A, B) + beta * C with A m x k, B k x n (rectangular,
ragged, strided views), and matrix powers X_{t+1} = SpAMM(X_t, X_t) or SpAMM(X_t, A) planned
from the norm map that the multiply's epilogue writes.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2103_13042_gb300 as P
import synth
from oracle import general as G
from oracle import precision as OP
from oracle import spamm as S
from tests.gpu_helpers import band_ok, dev, host

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _rect(m, k, seed, kind="exp", rate=0.02):
    if kind == "sparse":
        return synth.rect_near_sparse(m, k, seed)
    return synth.rect_decay_normal(m, k, rate, seed)


def _gpu_surv(plan):
    tp, kk = plan.export()
    surv = np.zeros((plan.bm, plan.bk, plan.bn), dtype=bool)
    for t in range(plan.bm * plan.bn):
        i, j = divmod(t, plan.bn)
        ks = (kk[tp[t]:tp[t + 1]] & 0x3FF).astype(np.int64)
        assert np.all(np.diff(ks) > 0)
        surv[i, ks, j] = True
    return surv


def _check_general(a, b, c_in, leaf, tau, alpha, beta, mode, oracle_norms=False):
    m, k = a.shape
    n = b.shape[1]
    ref = G.spamm_general(a, b, leaf, tau, alpha, beta, c_in if beta != 0.0 else None)
    A, B = dev(a), dev(b)
    C = dev(c_in.copy())
    if oracle_norms:
        nA, nB = dev(ref["nA"]), dev(ref["nB"])
    else:
        nA, nB = P.spamm_normmap_rect(A, leaf), P.spamm_normmap_rect(B, leaf)
        g = host(nA)
        assert np.all(np.abs(g - ref["nA"]) <= 3e-13 * ref["nA"])
    plan = P.GeneralPlan(m, k, n, leaf, mode)
    plan.plan_multiply(nA, nB, tau, A, B, C, 1e-6, alpha, beta)
    torch.cuda.synchronize()
    assert P.spamm_last_device_status() == 0
    surv = _gpu_surv(plan)
    p = ref["nA"][:, :, None] * ref["nB"][None, :, :]
    if oracle_norms:
        assert np.array_equal(surv, ref["surv"])
    else:
        assert band_ok(surv, ref["surv"], p, tau)
    st = plan.stats()
    assert st["survivors"] == int(surv.sum())
    assert st["valid_ratio"] == pytest.approx(surv.sum() / surv.size, rel=1e-15)
    got = host(C).astype(np.float64)
    want = alpha * G.product_rect(a, b, leaf, surv)
    if beta != 0.0:
        want = want + beta * c_in.astype(np.float64)
    if mode == OP.FP32:
        t = OP.accumulation_tile_bounds(ref["nA"], ref["nB"], surv, mode, leaf)
    else:
        t = OP.apriori_tile_bounds(ref["nA"], ref["nB"], surv, mode, leaf)
    # the epilogue adds one rounding of alpha * acc and one of the FMA with beta * C
    scale = OP.tile_errors(np.abs(want), np.zeros_like(want), leaf)
    if beta != 0.0:                                 # beta = 0 never reads C (it may hold NaN)
        scale = scale + OP.tile_errors(np.abs(beta * c_in.astype(np.float64)),
                                       np.zeros_like(want), leaf)
    bound = abs(alpha) * t + 3 * U32 * scale
    err = OP.tile_errors(got, want, leaf)
    assert np.all(err <= bound + 1e-30), (err - bound).max()
    return got, surv, plan


@pytest.mark.parametrize("m,k,n,leaf,kind", [(300, 577, 190, 64, "exp"), (128, 576, 1000, 32, "exp"),
                                             (97, 130, 260, 32, "sparse"), (256, 1152, 640, 128, "sparse")])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.75, 1.0), (2.0, 0.5)])
def test_general_fp32_against_oracle(m, k, n, leaf, kind, alpha, beta):
    a = _rect(m, k, 11 + m, kind)
    b = _rect(k, n, 12 + n, kind)
    c_in = _rect(m, n, 13, "exp", 0.5)
    nA, nB = G.normmap_rect(a, leaf), G.normmap_rect(b, leaf)
    p = (nA[:, :, None] * nB[None, :, :]).ravel()
    tau = float(np.quantile(p[p > 0], 0.4))
    got, surv, _ = _check_general(a, b, c_in, leaf, tau, alpha, beta, OP.FP32)
    empty = ~surv.any(axis=1)
    for i, j in zip(*np.nonzero(empty)):   # tiles without survivors: beta * C exactly
        blk = (slice(i * leaf, min(m, (i + 1) * leaf)), slice(j * leaf, min(n, (j + 1) * leaf)))
        assert np.array_equal(got[blk], (np.float32(beta) * c_in[blk]).astype(np.float64))


@pytest.mark.parametrize("name,mode", [("bf16", OP.BF16), ("fp16_split", OP.FP16_SPLIT),
                                       ("tf32x3", OP.TF32X3)])
@pytest.mark.parametrize("m,k,n,leaf", [(300, 577, 190, 64), (200, 1000, 333, 128)])
def test_general_tensor_modes_against_oracle(name, mode, m, k, n, leaf):
    a = _rect(m, k, 21, "exp")
    b = _rect(k, n, 22, "exp")
    c_in = _rect(m, n, 23, "exp", 0.5)
    nA, nB = G.normmap_rect(a, leaf), G.normmap_rect(b, leaf)
    p = (nA[:, :, None] * nB[None, :, :]).ravel()
    tau = float(np.quantile(p[p > 0], 0.3))
    _check_general(a, b, c_in, leaf, tau, 1.0, 0.0, mode, oracle_norms=True)
    _check_general(a, b, c_in, leaf, tau, -1.5, 0.5, mode, oracle_norms=True)


def test_vgg13_conv_shapes_bf16():
    """The im2col shapes of the paper's VGG13 layers (Section 4.3.2): conv21 128 x 576 x 25600
    and conv31 256 x 1152 x 6400, near-sparse activations, BF16 at leaf 64."""
    for (m, k, n), seed in (((128, 576, 25600), 5), ((256, 1152, 6400), 6)):
        a = _rect(m, k, seed, "exp", 0.05)           # weights: smooth in the channel index
        b = _rect(k, n, seed + 1, "sparse")          # ReLU activations
        nA, nB = G.normmap_rect(a, 64), G.normmap_rect(b, 64)
        p = (nA[:, :, None] * nB[None, :, :]).ravel()
        tau = float(np.quantile(p[p > 0], 0.5))
        _check_general(a, b, np.zeros((m, n), np.float32), 64, tau, 1.0, 0.0, OP.BF16)


def test_beta_zero_ignores_nan_in_c():
    m, k, n, leaf = 130, 200, 97, 64
    a, b = _rect(m, k, 31), _rect(k, n, 32)
    c_in = np.full((m, n), np.nan, np.float32)
    got, _, _ = _check_general(a, b, c_in, leaf, 0.0, 1.0, 0.0, OP.FP32)
    assert np.isfinite(got).all()


def test_strided_views_equal_contiguous_operands():
    """Row-major views with leading dimensions larger than their widths (a block of a wider
    matrix) give the same bits as contiguous copies, and only C's own columns are written."""
    m, k, n, leaf = 200, 300, 150, 64
    a, b = _rect(m, k, 41), _rect(k, n, 42)
    wideA = torch.zeros((m, k + 37), device="cuda")   # views start on 16-byte boundaries
    wideA[:, 8:8 + k] = dev(a)
    wideB = torch.zeros((k, n + 64), device="cuda")
    wideB[:, 64:] = dev(b)
    wideC = torch.full((m, n + 20), 7.0, device="cuda")
    Av, Bv, Cv = wideA[:, 8:8 + k], wideB[:, 64:], wideC[:, 4:4 + n]
    assert Av.stride(0) == k + 37
    nA, nB = P.spamm_normmap_rect(Av, leaf), P.spamm_normmap_rect(Bv, leaf)
    nAc, nBc = P.spamm_normmap_rect(dev(a), leaf), P.spamm_normmap_rect(dev(b), leaf)
    # rows 16-byte aligned or not take different read paths (same exact-square sums, other
    # order): equal to the norm map's accuracy, not bit for bit
    assert torch.allclose(nA, nAc, rtol=1e-13, atol=0) and torch.allclose(nB, nBc, rtol=1e-13, atol=0)
    tau = float(torch.quantile(host_t(nAc).flatten(), 0.5)) * float(host_t(nBc).max())
    pl = P.GeneralPlan(m, k, n, leaf, P.FP32)
    pl.plan_multiply(nAc, nBc, tau, Av, Bv, Cv)   # the same plan input: the same bits
    ref = torch.empty((m, n), device="cuda")
    P.GeneralPlan(m, k, n, leaf, P.FP32).plan_multiply(nAc, nBc, tau, dev(a), dev(b), ref)
    torch.cuda.synchronize()
    assert torch.equal(Cv, ref)
    assert bool((wideC[:, :4] == 7.0).all()) and bool((wideC[:, 4 + n:] == 7.0).all())


def host_t(t):
    torch.cuda.synchronize()
    return t.detach().cpu()


def test_rect_normmap_against_oracle():
    for rows, cols, ld, leaf in ((333, 517, 517, 64), (130, 1000, 1003, 32), (1, 5, 5, 32),
                                 (257, 129, 160, 128), (100, 1026, 1028, 64), (64, 33, 36, 32)):
        g = np.random.Generator(np.random.PCG64(rows + cols))
        x = (g.standard_normal((rows, ld)) * np.exp2(g.integers(-40, 40, (rows, ld)))).astype(np.float32)
        X = dev(x)[:, :cols]
        got = host(P.spamm_normmap_rect(X, leaf))
        want = G.normmap_rect(x[:, :cols], leaf)
        nz = want > 0
        assert np.array_equal(got == 0, want == 0)
        assert np.all(np.abs(got[nz] - want[nz]) <= 3e-13 * want[nz])


@pytest.mark.parametrize("name,mode,leaf", [("fp32", OP.FP32, 32), ("fp32", OP.FP32, 64),
                                            ("bf16_split", OP.BF16_SPLIT, 64),
                                            ("tf32x3", OP.TF32X3, 128)])
def test_output_norm_map_equals_norm_of_stored_c(name, mode, leaf):
    """normC written by the multiply's epilogue equals the exactly rounded norms of the C it
    stored (to the norm map's 3e-13), at ragged n, beta = 0 and beta != 0 (empty tiles
    too), and agrees with a separate norm pass over C."""
    n = 777
    a = synth.exp_decay_normal(n, 0.05, 51)
    b = synth.exp_decay_normal(n, 0.05, 52)
    A, B = dev(a), dev(b)
    nA, nB = P.spamm_normmap(A, leaf), P.spamm_normmap(B, leaf)
    p = S.triple_products(S.normmap(a, leaf), S.normmap(b, leaf))
    tau = float(np.quantile(p[p > 0], 0.8))
    pl = P.GeneralPlan(n, n, n, leaf, mode)
    for alpha, beta in ((1.0, 0.0), (0.5, -1.0)):
        C = dev(synth.exp_decay_normal(n, 1.0, 53))
        bd = P.num_blocks(n, leaf)
        nC = torch.full((bd, bd), float("nan"), dtype=torch.float64, device="cuda")
        pl.plan_multiply(nA, nB, tau, A, B, C, 1e-6, alpha, beta, normC=nC)
        got = host(nC)
        c = host(C)
        want = S.normmap(c, leaf)
        nz = want > 0
        assert np.array_equal(got == 0, want == 0)
        assert np.all(np.abs(got[nz] - want[nz]) <= 3e-13 * want[nz])
        sep = host(P.spamm_normmap(C, leaf))
        assert np.all(np.abs(got - sep) <= 1e-12 * np.maximum(sep, 1e-300))


@pytest.mark.parametrize("squaring", [True, False])
@pytest.mark.parametrize("name,mode", [("fp32", OP.FP32), ("tf32x3", OP.TF32X3)])
def test_power_chain_against_oracle(squaring, name, mode):
    """Matrix powers of an exponential-decay matrix at a ragged size (the ergo-shaped stand-in
    of Section 4.3, scaled down): each step plans from the norm map the previous multiply
    wrote (no norm pass over X_t) and stays within the oracle's chain at every step."""
    n, leaf, steps = 1000, 64, 3
    a = (0.5 * synth.exp_decay_normal(n, 0.5, 61)).astype(np.float32)
    tau = 1e-6
    chain = G.power_chain(a, leaf, tau, steps, squaring)
    X = dev(a)
    A = dev(a)
    bd = P.num_blocks(n, leaf)
    nX = P.spamm_normmap(X, leaf)
    nA = nX.clone()
    pl = P.GeneralPlan(n, n, n, leaf, mode)
    for t, ref in enumerate(chain):
        Y = torch.empty_like(X)
        nY = torch.empty((bd, bd), dtype=torch.float64, device="cuda")
        pl.plan_multiply(nX, nX if squaring else nA, tau, X, X if squaring else A, Y, 1e-6,
                         normC=nY)
        torch.cuda.synchronize()
        assert P.spamm_last_device_status() == 0
        got = host(Y).astype(np.float64)
        want = ref["X"].astype(np.float64)
        rel = S.frobenius(got - want) / S.frobenius(want)
        assert rel <= 1e-5 * (t + 1), (t, rel)
        # the planned norms equal the oracle's norm map of its own X_t up to the chain's drift
        assert np.allclose(host(nX), ref["norms"], rtol=1e-5 * (t + 1), atol=0.0)
        X, nX = Y, nY


@pytest.mark.parametrize("m,k,n,leaf", [(1, 1, 1, 32), (1, 300, 5, 64), (257, 1, 129, 32),
                                        (64, 64, 64, 64), (3, 2000, 2, 128)])
def test_general_degenerate_shapes(m, k, n, leaf):
    """Single rows, columns and inner dimensions, one block per grid and long thin products."""
    a = _rect(m, k, 91 + m + k, "exp", 0.01)
    b = _rect(k, n, 92 + n, "exp", 0.01)
    c_in = _rect(m, n, 93, "exp", 0.5)
    mode = OP.FP32 if leaf == 32 else OP.TF32X3
    _check_general(a, b, c_in, leaf, 0.0, 1.0, 0.0, mode)
    nA, nB = G.normmap_rect(a, leaf), G.normmap_rect(b, leaf)
    p = (nA[:, :, None] * nB[None, :, :]).ravel()
    _check_general(a, b, c_in, leaf, float(np.median(p)), -1.0, 2.0, mode)


def test_general_argument_errors_enqueue_nothing():
    m, k, n, leaf = 100, 200, 60, 64
    pl = P.GeneralPlan(m, k, n, leaf, P.FP32)
    A, B = dev(_rect(m, k, 95)), dev(_rect(k, n, 96))
    C = torch.full((m, n), 5.0, device="cuda")
    nA, nB = P.spamm_normmap_rect(A, leaf), P.spamm_normmap_rect(B, leaf)
    lib = P.lib()
    s = torch.cuda.current_stream().cuda_stream
    args = lambda lda, cptr: (pl.handle, ctypes.c_void_p(A.data_ptr()), lda,
                              ctypes.c_void_p(B.data_ptr()), n, cptr, n, 1.0, 0.0, None,
                              ctypes.c_void_p(s))
    assert lib.spamm_multiply_general(*args(k - 1, ctypes.c_void_p(C.data_ptr()))) == 1  # lda < k
    assert lib.spamm_multiply_general(*args(k, ctypes.c_void_p(A.data_ptr()))) == 1      # C aliases A
    assert lib.spamm_multiply_general(pl.handle, ctypes.c_void_p(A.data_ptr()), k,
                                      ctypes.c_void_p(B.data_ptr()), n,
                                      ctypes.c_void_p(C.data_ptr()), n, float("nan"), 0.0, None,
                                      ctypes.c_void_p(s)) == 1                         # alpha NaN
    torch.cuda.synchronize()
    assert bool((C == 5.0).all())
    pl.plan_multiply(nA, nB, 0.0, A, B, C)
    torch.cuda.synchronize()
    assert not bool((C == 5.0).all())
