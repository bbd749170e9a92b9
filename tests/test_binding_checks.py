"""The Python binding's tensor checks, on the CPU: a recording stand-in replaces the library,
CPU tensors stand in for device tensors, and every entry point is called once with valid
operands (each call reaches the library with its declared number of arguments) and with each
kind of invalid operand (the call raises SPAMM_ERR_INVALID_ARG before reaching the library)."""
import ctypes

import pytest
import torch

import paper_2103_13042_gb300 as P


class _Recorder:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if name not in P._SIGS:
            raise AttributeError(name)

        def fn(*args):
            assert len(args) == len(P._SIGS[name]), (name, len(args))
            self.calls.append(name)
            return 0
        return fn


@pytest.fixture()
def rec(monkeypatch):
    r = _Recorder()
    monkeypatch.setattr(P, "_lib", r)
    monkeypatch.setattr(P, "_DEVICE_TYPE", "cpu")
    monkeypatch.setattr(P, "_PARAMS", 8449)
    monkeypatch.setattr(P, "_stream", lambda stream: 0)
    monkeypatch.setattr(P, "_current_index", lambda: 0)
    return r


def _m(n, dtype=torch.float32):
    return torch.zeros(n, n, dtype=dtype)


def _plan(n=100, leaf=32):
    return P.Plan(n, leaf, P.FP32)


def _invalid(fn, *args, **kw):
    with pytest.raises(P.SpammError) as e:
        fn(*args, **kw)
    assert e.value.code == 1
    return str(e.value)


def test_valid_calls_reach_the_library(rec):
    n, leaf = 100, 32
    bd = P.num_blocks(n, leaf)
    A, B, C = _m(n), _m(n), _m(n)
    nA = P.spamm_normmap(A, leaf)
    assert nA.shape == (bd, bd) and nA.dtype == torch.float64
    nB = torch.zeros(bd * bd, dtype=torch.float64)              # flat is accepted
    pl = _plan(n, leaf)
    pl.plan(nA, nB, 0.1)
    pl.multiply(A, B, C)
    pl.plan_multiply(nA, nB, 0.1, A, B, C)
    pl.band(nA, nB, 0.0, 0.1)
    pl.tau_for_valid_ratio(nA, nB, 0.5)
    pl.histogram(nA, nB)
    W = torch.zeros(8449)
    pl.tau_predict(nA, nB, 1e-5, W)
    P.spamm_frobenius_diff(torch.zeros(7), torch.zeros(7))
    P.spamm_frobenius_diff(torch.zeros(7))
    P.spamm_multiply_fp32_noalloc(A, B, C, leaf, 0.1)
    X = torch.zeros(5, 65)
    P.spamm_mlp_forward(W, X)
    P.spamm_mlp_grad(W, X, torch.zeros(5), 0.5)
    P.spamm_mlp_adam(W, torch.zeros(8449), torch.zeros(8449), torch.zeros(8449), 1, 1e-3)
    P.spamm_mlp_train(W, torch.zeros(8449), torch.zeros(8449), 0, X, torch.zeros(5),
                      torch.zeros(6, dtype=torch.int32), 2, 3, 1e-3, 0.5)
    ns = [64, 100]
    As, Bs, Cs = [_m(k) for k in ns], [_m(k) for k in ns], [_m(k) for k in ns]
    b = P.Batch(ns, 32, P.FP32, graph=False)
    b.run(As, Bs, Cs, [0.1, 0.2])
    b.tau_predict(As, Bs, [1e-5, 1e-6], W)
    P.spamm_multiply_batched(As, Bs, Cs, [0.1, 0.2], 32)
    P.spamm_batch_autotune(As, Bs, Cs, [0.1, 0.2])
    for name in ("spamm_normmap", "spamm_plan", "spamm_multiply", "spamm_plan_multiply",
                 "spamm_plan_band", "spamm_tau_for_valid_ratio", "spamm_norm_histogram",
                 "spamm_tau_predict", "spamm_frobenius_diff", "spamm_multiply_fp32_noalloc",
                 "spamm_mlp_forward", "spamm_mlp_grad", "spamm_mlp_adam", "spamm_mlp_train",
                 "spamm_batch_run", "spamm_batch_tau_predict", "spamm_multiply_batched",
                 "spamm_batch_autotune"):
        assert name in rec.calls, name


def test_matrix_operands_are_checked(rec):
    n = 100
    A, B, C = _m(n), _m(n), _m(n)
    pl = _plan(n)
    rec.calls.clear()
    assert "on meta" in _invalid(pl.multiply, torch.empty(n, n, device="meta"), B, C)
    assert "float64" in _invalid(pl.multiply, _m(n, torch.float64), B, C)
    assert "contiguous" in _invalid(pl.multiply, A, _m(n).t(), C)   # a transposed view
    assert "contiguous" in _invalid(pl.multiply, A, torch.zeros(n, 2 * n)[:, :n], C)
    assert "shape" in _invalid(pl.multiply, A, B, _m(n + 1))
    assert "shape" in _invalid(pl.multiply, A, B, torch.zeros(n * n))
    assert "not a tensor" in _invalid(pl.multiply, A, B, [[0.0]])
    assert "2-D" in _invalid(P.spamm_normmap, torch.zeros(n * n), 32)
    assert "shape" in _invalid(P.spamm_normmap, torch.zeros(n, n + 4), 32)
    assert "shape" in _invalid(P.spamm_multiply_fp32_noalloc, A, B, _m(n - 1), 32, 0.1)
    assert rec.calls == []


def test_norm_maps_weights_and_features_are_checked(rec):
    n, leaf = 100, 32
    bd = P.num_blocks(n, leaf)
    good = torch.zeros(bd, bd, dtype=torch.float64)
    pl = _plan(n, leaf)
    rec.calls.clear()
    assert "float32" in _invalid(pl.plan, good.float(), good, 0.1)
    assert "elements" in _invalid(pl.plan, good, torch.zeros(bd + 1, bd, dtype=torch.float64), 0.1)
    assert "elements" in _invalid(P.spamm_normmap, _m(n), leaf, out=torch.zeros(bd, bd - 1,
                                                                               dtype=torch.float64))
    assert "elements" in _invalid(pl.tau_predict, good, good, 1e-5, torch.zeros(8448))
    assert "[count, 65]" in _invalid(P.spamm_mlp_forward, torch.zeros(8449), torch.zeros(5, 64))
    assert "elements" in _invalid(P.spamm_mlp_grad, torch.zeros(8449), torch.zeros(5, 65),
                                  torch.zeros(4), 0.5)
    assert "at least" in _invalid(P.spamm_mlp_train, torch.zeros(8449), torch.zeros(8449),
                                  torch.zeros(8449), 0, torch.zeros(5, 65), torch.zeros(5),
                                  torch.zeros(5, dtype=torch.int32), 2, 3, 1e-3, 0.5)
    assert "int32" in _invalid(P.spamm_mlp_train, torch.zeros(8449), torch.zeros(8449),
                               torch.zeros(8449), 0, torch.zeros(5, 65), torch.zeros(5),
                               torch.zeros(6, dtype=torch.int64), 2, 3, 1e-3, 0.5)
    assert rec.calls == []


def test_batch_tables_are_checked(rec):
    ns = [64, 100]
    As, Bs, Cs = [_m(k) for k in ns], [_m(k) for k in ns], [_m(k) for k in ns]
    b = P.Batch(ns, 32, P.FP32, graph=False)
    rec.calls.clear()
    assert "Cs[1]" in _invalid(b.run, As, Bs, [Cs[0], _m(101)], [0.1, 0.2])
    assert "Bs[0]" in _invalid(b.run, As, [_m(64, torch.float16), Bs[1]], Cs, [0.1, 0.2])
    assert "length" in _invalid(b.run, As, Bs, Cs, [0.1])
    assert "batch of 2" in _invalid(b.run, As + As, Bs + Bs, Cs + Cs, [0.1] * 4)
    assert "targets" in _invalid(b.tau_predict, As, Bs, [1e-5], torch.zeros(8449))
    assert "As[1]" in _invalid(P.spamm_multiply_batched, [As[0], As[1].t()], Bs, Cs,
                               [0.1, 0.2], 32)
    assert rec.calls == []


def test_tensors_on_another_device_are_rejected(rec, monkeypatch):
    """Every operand must live on the current device, where the library launches: with the
    current device mocked as 1, tensors of device 0 are refused before any pointer reaches the
    library, by the general check and by the batch's fast path alike."""
    n, leaf = 100, 32
    bd = P.num_blocks(n, leaf)
    A, B, C = _m(n), _m(n), _m(n)
    nA = torch.zeros(bd, bd, dtype=torch.float64)
    pl = _plan(n, leaf)
    ns = [64, 100]
    As, Bs, Cs = [_m(k) for k in ns], [_m(k) for k in ns], [_m(k) for k in ns]
    b = P.Batch(ns, 32, P.FP32, graph=False)
    rec.calls.clear()
    monkeypatch.setattr(P, "_current_index", lambda: 1)
    assert "current device is 1" in _invalid(pl.multiply, A, B, C)
    assert "current device is 1" in _invalid(pl.plan, nA, nA, 0.1)
    assert "current device is 1" in _invalid(P.spamm_normmap, A, leaf)
    assert "current device is 1" in _invalid(P.spamm_frobenius_diff, torch.zeros(7))
    assert "current device is 1" in _invalid(P.spamm_multiply_fp32_noalloc, A, B, C, leaf, 0.1)
    assert "current device is 1" in _invalid(b.run, As, Bs, Cs, [0.1, 0.2])
    assert "current device is 1" in _invalid(P.spamm_multiply_batched, As, Bs, Cs, [0.1, 0.2], 32)
    assert rec.calls == []
    monkeypatch.setattr(P, "_current_index", lambda: 0)
    pl.multiply(A, B, C)
    b.run(As, Bs, Cs, [0.1, 0.2])
    assert rec.calls == ["spamm_multiply", "spamm_batch_run"]


def test_general_plan_operands_are_checked(rec):
    """GeneralPlan takes row-major views (contiguous rows, any leading dimension) of the
    declared shapes and refuses the rest before reaching the library."""
    m, k, n, leaf = 70, 130, 50, 32
    pl = P.GeneralPlan(m, k, n, leaf, P.FP32)
    assert (pl.bm, pl.bk, pl.bn) == (3, 5, 2)
    A, B, C = torch.zeros(m, k), torch.zeros(k, n), torch.zeros(m, n)
    nA = torch.zeros(pl.bm, pl.bk, dtype=torch.float64)
    nB = torch.zeros(pl.bk, pl.bn, dtype=torch.float64)
    rec.calls.clear()
    wide = torch.zeros(m, k + 9)
    pl.plan_multiply(nA, nB, 0.1, wide[:, 3:3 + k], B, C, alpha=2.0, beta=0.5)  # a view: ok
    pl.multiply(A, B, C, normC=torch.zeros(pl.bm, pl.bn, dtype=torch.float64))
    P.spamm_normmap_rect(wide[:, :k], leaf)
    assert rec.calls == ["spamm_plan_multiply_general", "spamm_multiply_general",
                         "spamm_normmap_rect"]
    rec.calls.clear()
    assert "shape" in _invalid(pl.multiply, A.t().contiguous(), B, C)           # k x m, not m x k
    assert "rows are not contiguous" in _invalid(pl.multiply, torch.zeros(k, m).t(), B, C)
    assert "elements" in _invalid(pl.plan, nB, nB, 0.1)                          # normA of B's grid
    assert "elements" in _invalid(pl.multiply, A, B, C, normC=torch.zeros(4, dtype=torch.float64))
    assert "float32" in _invalid(pl.multiply, A.double(), B, C)
    assert rec.calls == []
