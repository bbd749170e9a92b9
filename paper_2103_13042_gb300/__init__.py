"""Python binding of the GB300 SpAMM library (ctypes over ``lib/libspamm.so``).

Argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are passed as raw device pointers (``data_ptr()``), streams as
``torch.cuda.current_stream().cuda_stream``.  The names follow the C ABI in
``include/spamm.h``.  There is no CPU fallback: if the library is missing,
loading it raises.
"""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libspamm.so")

FP32, TF32X3, BF16, FP16, BF16_SPLIT, FP16_SPLIT = range(6)
PRECISIONS = {"fp32": FP32, "tf32x3": TF32X3, "bf16": BF16, "fp16": FP16,
              "bf16_split": BF16_SPLIT, "fp16_split": FP16_SPLIT}

STATUS = {0: "SPAMM_OK", 1: "SPAMM_ERR_INVALID_ARG", 2: "SPAMM_ERR_UNSUPPORTED",
          3: "SPAMM_ERR_CUDA", 4: "SPAMM_ERR_NO_MEMORY", 5: "SPAMM_ERR_TIMEOUT",
          6: "SPAMM_ERR_DEVICE_FAULT"}


class SpammError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("survivors", ctypes.c_int64), ("nonempty_tiles", ctypes.c_int64),
                ("flagged", ctypes.c_int64), ("valid_ratio", ctypes.c_double),
                ("skipped_bound1", ctypes.c_double), ("skipped_bound2", ctypes.c_double),
                ("norm_a", ctypes.c_double), ("norm_b", ctypes.c_double),
                ("leaf", ctypes.c_int32), ("bd", ctypes.c_int32),
                ("max_tile_survivors", ctypes.c_int32), ("flag_exponent", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Problem(ctypes.Structure):
    """One instance of a batch (spamm_problem_t)."""
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("tau", ctypes.c_double)]


BATCH_GRAPH, BATCH_DYNAMIC, BATCH_TIMING = 1, 2, 4


class Tune(ctypes.Structure):
    """One autotuner candidate (spamm_tune_t)."""
    _fields_ = [("leaf", ctypes.c_int32), ("flags", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"leaf": self.leaf, "schedule": "dynamic" if self.flags & BATCH_DYNAMIC else "static",
                "flags": self.flags, "ms": self.ms}

_lib = None

_VP, _I64, _I32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_SIGS = {
    "spamm_normmap": [_VP, _I64, _I32, _VP, _VP],
    "spamm_plan_workspace_size": [_I64, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)],
    "spamm_plan_create": [ctypes.POINTER(_VP), _I64, _I32, _I32, _VP, ctypes.c_size_t],
    "spamm_plan_destroy": [_VP],
    "spamm_plan": [_VP, _VP, _VP, _D, _D, _VP],
    "spamm_plan_stats": [_VP, ctypes.POINTER(Stats), _VP],
    "spamm_plan_export": [_VP, _VP, _VP, _I64, _VP],
    "spamm_multiply": [_VP, _VP, _VP, _VP, _VP],
    "spamm_plan_multiply": [_VP, _VP, _VP, _D, _D, _VP, _VP, _VP, _VP],
    "spamm_frobenius_diff": [_VP, _VP, _I64, ctypes.POINTER(_D), _VP],
    "spamm_last_device_status": [_VP, ctypes.POINTER(_I32)],
    "spamm_multiply_fp32_noalloc": [_VP, _VP, _VP, _I64, _I32, _D, _VP],
    "spamm_selftest_bounded_wait": [_I64, ctypes.POINTER(_I64), _VP],
    "spamm_batch_workspace_size": [_VP, _I32, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)],
    "spamm_batch_create": [ctypes.POINTER(_VP), _VP, _I32, _I32, _I32, _I32, _VP,
                           ctypes.c_size_t],
    "spamm_batch_run": [_VP, _VP, _D, _VP],
    "spamm_batch_stats": [_VP, _VP, _VP],
    "spamm_batch_export": [_VP, _I32, _VP, _VP, _VP, _VP, _I64, _VP],
    "spamm_multiply_batched": [_VP, _I32, _I32, _I32, _D, _VP, _VP],
    "spamm_batch_destroy": [_VP],
    "spamm_batch_timings": [_VP, _VP],
    "spamm_plan_band": [_VP, _VP, _VP, _D, _D, _VP],
    "spamm_tau_for_valid_ratio": [_VP, _VP, _VP, _D, _D, _I32, ctypes.POINTER(_D),
                                  ctypes.POINTER(_D), ctypes.POINTER(_I32), _VP],
    "spamm_norm_histogram": [_VP, _VP, _VP, _VP, _VP],
    "spamm_tau_predict": [_VP, _VP, _VP, _D, _VP, ctypes.POINTER(_D), _VP],
    "spamm_batch_tau_predict": [_VP, _VP, _VP, _VP, _VP, _VP],
    "spamm_mlp_param_count": [ctypes.POINTER(_I32)],
    "spamm_mlp_forward": [_VP, _VP, _I32, _VP, _VP],
    "spamm_mlp_grad": [_VP, _VP, _VP, _I32, ctypes.c_float, _VP, _VP, _VP],
    "spamm_mlp_adam": [_VP, _VP, _VP, _VP, _I32, ctypes.c_float, _VP],
    "spamm_mlp_train": [_VP, _VP, _VP, _I32, _VP, _VP, _VP, _I32, _I32, ctypes.c_float,
                        ctypes.c_float, _VP, _VP],
    "spamm_batch_autotune": [_VP, _I32, _I32, _D, _I32, _VP, ctypes.POINTER(Tune), _VP,
                             ctypes.POINTER(_I32)],
}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libspamm.so not built ({LIB_PATH}); run "
                               "`python -m paper_2103_13042_gb300.build`")
        l = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        l.spamm_status_string.argtypes = [ctypes.c_int]
        l.spamm_status_string.restype = ctypes.c_char_p
        _lib = l
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise SpammError(code, where)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def num_blocks(n: int, leaf: int) -> int:
    return -(-n // leaf)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def spamm_normmap(X, leaf: int, out=None, stream=None):
    """Leaf Frobenius norms of the n x n FP32 device tensor X -> FP64 [bd, bd] tensor."""
    import torch
    n = X.shape[0]
    bd = num_blocks(n, leaf)
    if out is None:
        out = torch.empty((bd, bd), dtype=torch.float64, device=X.device)
    _check(lib().spamm_normmap(_ptr(X), n, leaf, _ptr(out), _stream(stream)), "spamm_normmap")
    return out


class Plan:
    """Owns a spamm_plan_t (work queues for one (n, leaf, precision))."""

    def __init__(self, n: int, leaf: int, precision: int = FP32, workspace=None):
        self.n, self.leaf, self.precision = n, leaf, precision
        self.bd = num_blocks(n, leaf)
        h = ctypes.c_void_p()
        ws_ptr, ws_bytes = (None, 0) if workspace is None else (_ptr(workspace),
                                                                 workspace.numel() * workspace.element_size())
        _check(lib().spamm_plan_create(ctypes.byref(h), n, leaf, precision, ws_ptr, ws_bytes),
               "spamm_plan_create")
        self.handle = h
        self._workspace = workspace

    @staticmethod
    def workspace_size(n: int, leaf: int, precision: int = FP32) -> int:
        b = ctypes.c_size_t()
        _check(lib().spamm_plan_workspace_size(n, leaf, precision, ctypes.byref(b)),
               "spamm_plan_workspace_size")
        return b.value

    def close(self):
        if self.handle:
            lib().spamm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, normA, normB, tau: float, target_rel_err: float = 1e-5, stream=None):
        _check(lib().spamm_plan(self.handle, _ptr(normA), _ptr(normB), float(tau),
                                float(target_rel_err), _stream(stream)), "spamm_plan")
        return self

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(lib().spamm_plan_stats(self.handle, ctypes.byref(s), _stream(stream)),
               "spamm_plan_stats")
        return s.as_dict()

    def export(self, stream=None):
        """(tile_ptr int32[bd*bd+1], k_idx uint16[S]) as numpy arrays."""
        import numpy as np
        st = self.stats(stream)
        tp = np.zeros(self.bd * self.bd + 1, dtype=np.int32)
        kk = np.zeros(max(1, st["survivors"]), dtype=np.uint16)
        _check(lib().spamm_plan_export(self.handle, tp.ctypes.data_as(ctypes.c_void_p),
                                       kk.ctypes.data_as(ctypes.c_void_p), kk.size,
                                       _stream(stream)), "spamm_plan_export")
        return tp, kk[:st["survivors"]]

    def multiply(self, A, B, C, stream=None):
        _check(lib().spamm_multiply(self.handle, _ptr(A), _ptr(B), _ptr(C), _stream(stream)),
               "spamm_multiply")
        return C

    def plan_multiply(self, normA, normB, tau: float, A, B, C, target_rel_err: float = 1e-5,
                      stream=None):
        """plan() then multiply() in one call (zero-fill of empty tiles overlapped)."""
        _check(lib().spamm_plan_multiply(self.handle, _ptr(normA), _ptr(normB), float(tau),
                                         float(target_rel_err), _ptr(A), _ptr(B), _ptr(C),
                                         _stream(stream)), "spamm_plan_multiply")
        return C

    def band(self, normA, normB, tau_lo: float, tau_hi: float, stream=None):
        """Plan the triples with tau_lo <= p < tau_hi (error measurement)."""
        _check(lib().spamm_plan_band(self.handle, _ptr(normA), _ptr(normB), float(tau_lo),
                                     float(tau_hi), _stream(stream)), "spamm_plan_band")
        return self

    def tau_for_valid_ratio(self, normA, normB, target: float, tol: float = 0.01,
                            max_probes: int = 20, stream=None):
        """(tau, valid ratio, probes) of the valid-ratio search (Section 3.5.2)."""
        t, r, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        _check(lib().spamm_tau_for_valid_ratio(self.handle, _ptr(normA), _ptr(normB),
                                               float(target), float(tol), int(max_probes),
                                               ctypes.byref(t), ctypes.byref(r), ctypes.byref(k),
                                               _stream(stream)), "spamm_tau_for_valid_ratio")
        return t.value, r.value, k.value

    def histogram(self, normA, normB, stream=None):
        """Raw counts of the 64-bin log2 histogram of relative norm products."""
        import numpy as np
        out = np.zeros(64, dtype=np.int64)
        _check(lib().spamm_norm_histogram(self.handle, _ptr(normA), _ptr(normB),
                                          out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
               "spamm_norm_histogram")
        return out

    def tau_predict(self, normA, normB, target_rel_err: float, weights, stream=None) -> float:
        """The network's tau for this plan's shape (weights: device float32 [8449])."""
        t = ctypes.c_double()
        _check(lib().spamm_tau_predict(self.handle, _ptr(normA), _ptr(normB),
                                       float(target_rel_err), _ptr(weights), ctypes.byref(t),
                                       _stream(stream)), "spamm_tau_predict")
        return t.value


def spamm_plan(normA, normB, n: int, leaf: int, tau: float, precision: int = FP32,
               target_rel_err: float = 1e-5, stream=None) -> Plan:
    return Plan(n, leaf, precision).plan(normA, normB, tau, target_rel_err, stream)


def spamm_multiply(plan: Plan, A, B, C=None, stream=None):
    import torch
    if C is None:
        C = torch.empty_like(A)
    return plan.multiply(A, B, C, stream)


def spamm_frobenius_diff(X, Y=None, stream=None) -> float:
    out = ctypes.c_double()
    _check(lib().spamm_frobenius_diff(_ptr(X), _ptr(Y), X.numel(), ctypes.byref(out),
                                      _stream(stream)), "spamm_frobenius_diff")
    return out.value


def spamm_multiply_fp32_noalloc(A, B, C, leaf: int, tau: float, stream=None):
    """FP32 SpAMM with no device allocation (static library scratch; ceil(n/leaf) <= 64)."""
    _check(lib().spamm_multiply_fp32_noalloc(_ptr(A), _ptr(B), _ptr(C), A.shape[0], leaf,
                                             float(tau), _stream(stream)),
           "spamm_multiply_fp32_noalloc")
    return C


def _problems(As, Bs, Cs, taus):
    arr = (Problem * len(As))()
    for i, (A, B, C, t) in enumerate(zip(As, Bs, Cs, taus)):
        arr[i] = Problem(A.data_ptr(), B.data_ptr(), C.data_ptr(), A.shape[0], float(t))
    return arr


class Batch:
    """Owns a spamm_batch_t: many independent products of fixed shapes."""

    def __init__(self, ns, leaf: int, precision: int = FP32, graph: bool = True,
                 workspace=None, dynamic: bool = False, timing: bool = False):
        self.ns = [int(n) for n in ns]
        self.leaf, self.precision = leaf, precision
        self.count = len(self.ns)
        n_arr = (ctypes.c_int64 * self.count)(*self.ns)
        ws_ptr, ws_bytes = (None, 0) if workspace is None else (
            _ptr(workspace), workspace.numel() * workspace.element_size())
        h = ctypes.c_void_p()
        flags = ((BATCH_GRAPH if graph else 0) | (BATCH_DYNAMIC if dynamic else 0) |
                 (BATCH_TIMING if timing else 0))
        _check(lib().spamm_batch_create(ctypes.byref(h), ctypes.cast(n_arr, ctypes.c_void_p),
                                        self.count, leaf, precision, flags, ws_ptr, ws_bytes),
               "spamm_batch_create")
        self.handle = h
        self._workspace = workspace
        self._keep = None

    @staticmethod
    def workspace_size(ns, leaf: int, precision: int = FP32) -> int:
        n_arr = (ctypes.c_int64 * len(ns))(*[int(n) for n in ns])
        b = ctypes.c_size_t()
        _check(lib().spamm_batch_workspace_size(ctypes.cast(n_arr, ctypes.c_void_p), len(ns),
                                                leaf, precision, ctypes.byref(b)),
               "spamm_batch_workspace_size")
        return b.value

    def run(self, As, Bs, Cs, taus, target_rel_err: float = 1e-5, stream=None):
        probs = _problems(As, Bs, Cs, taus)
        self._keep = probs
        _check(lib().spamm_batch_run(self.handle, ctypes.cast(probs, ctypes.c_void_p),
                                     float(target_rel_err), _stream(stream)), "spamm_batch_run")
        return Cs

    def stats(self, stream=None):
        arr = (Stats * self.count)()
        _check(lib().spamm_batch_stats(self.handle, ctypes.cast(arr, ctypes.c_void_p),
                                       _stream(stream)), "spamm_batch_stats")
        return [a.as_dict() for a in arr]

    def export(self, index: int, stream=None):
        """(normA, normB [bd, bd] float64, tile_ptr int32[bd*bd+1], k_idx uint16[S]) of one instance."""
        import numpy as np
        bd = num_blocks(self.ns[index], self.leaf)
        nA = np.zeros((bd, bd)); nB = np.zeros((bd, bd))
        tp = np.zeros(bd * bd + 1, dtype=np.int32)
        _check(lib().spamm_batch_export(self.handle, index, nA.ctypes.data_as(ctypes.c_void_p),
                                        nB.ctypes.data_as(ctypes.c_void_p),
                                        tp.ctypes.data_as(ctypes.c_void_p), None, 0,
                                        _stream(stream)), "spamm_batch_export")
        kk = np.zeros(max(1, int(tp[-1])), dtype=np.uint16)
        _check(lib().spamm_batch_export(self.handle, index, None, None, None,
                                        kk.ctypes.data_as(ctypes.c_void_p), kk.size,
                                        _stream(stream)), "spamm_batch_export")
        return nA, nB, tp, kk[:int(tp[-1])]

    def tau_predict(self, As, Bs, targets, weights, stream=None):
        """Predicted tau per instance (the norm maps of As / Bs are computed on the way)."""
        import numpy as np
        probs = (Problem * len(As))()
        for i, (A, B) in enumerate(zip(As, Bs)):   # no output: C stays NULL
            probs[i] = Problem(A.data_ptr(), B.data_ptr(), None, A.shape[0], 0.0)
        tg = np.ascontiguousarray(targets, dtype=np.float64)
        out = np.zeros(self.count, dtype=np.float64)
        _check(lib().spamm_batch_tau_predict(self.handle, ctypes.cast(probs, ctypes.c_void_p),
                                             tg.ctypes.data_as(ctypes.c_void_p), _ptr(weights),
                                             out.ctypes.data_as(ctypes.c_void_p),
                                             _stream(stream)), "spamm_batch_tau_predict")
        return out

    def timings(self):
        """{"normmap", "plan", "round", "multiply"} device ms of the last run (timing batches only)."""
        ms = (ctypes.c_float * 4)()
        _check(lib().spamm_batch_timings(self.handle, ctypes.cast(ms, ctypes.c_void_p)),
               "spamm_batch_timings")
        return {"normmap": ms[0], "plan": ms[1], "round": ms[2], "multiply": ms[3]}

    def close(self):
        if self.handle:
            lib().spamm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spamm_batch_autotune(As, Bs, Cs, taus, precision: int = FP32, target_rel_err: float = 1e-5,
                         reps: int = 3, stream=None):
    """Times every (leaf, schedule) candidate on these problems: (best, all) as dicts."""
    probs = _problems(As, Bs, Cs, taus)
    best = Tune()
    res = (Tune * 8)()
    nres = ctypes.c_int32(8)
    _check(lib().spamm_batch_autotune(ctypes.cast(probs, ctypes.c_void_p), len(As), precision,
                                      float(target_rel_err), reps, _stream(stream),
                                      ctypes.byref(best), ctypes.cast(res, ctypes.c_void_p),
                                      ctypes.byref(nres)), "spamm_batch_autotune")
    return best.as_dict(), [res[i].as_dict() for i in range(min(nres.value, 8))]


def spamm_multiply_batched(As, Bs, Cs, taus, leaf: int, precision: int = FP32,
                           target_rel_err: float = 1e-5, stream=None):
    """One-off batch (allocates and blocks). Returns the per-instance statistics."""
    probs = _problems(As, Bs, Cs, taus)
    arr = (Stats * len(As))()
    _check(lib().spamm_multiply_batched(ctypes.cast(probs, ctypes.c_void_p), len(As), leaf,
                                        precision, float(target_rel_err),
                                        ctypes.cast(arr, ctypes.c_void_p), _stream(stream)),
           "spamm_multiply_batched")
    return [a.as_dict() for a in arr]


# ---------------------------------------------------------------------------
# Learned-tau network (device float32 tensors)
# ---------------------------------------------------------------------------

def spamm_mlp_param_count() -> int:
    c = ctypes.c_int32()
    _check(lib().spamm_mlp_param_count(ctypes.byref(c)), "spamm_mlp_param_count")
    return c.value


def spamm_mlp_forward(weights, X, stream=None):
    import torch
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(lib().spamm_mlp_forward(_ptr(weights), _ptr(X), X.shape[0], _ptr(y), _stream(stream)),
           "spamm_mlp_forward")
    return y


def spamm_mlp_grad(weights, X, y_true, quantile: float, stream=None):
    """(gradient [8449], loss tensor [1]) of the mean pinball loss."""
    import torch
    g = torch.empty_like(weights)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(lib().spamm_mlp_grad(_ptr(weights), _ptr(X), _ptr(y_true), X.shape[0],
                                float(quantile), _ptr(g), _ptr(loss), _stream(stream)),
           "spamm_mlp_grad")
    return g, loss


def spamm_mlp_adam(weights, grad, m, v, t: int, lr: float, stream=None):
    _check(lib().spamm_mlp_adam(_ptr(weights), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr),
                                _stream(stream)), "spamm_mlp_adam")


def spamm_mlp_train(weights, m, v, t0: int, X, y_true, idx, steps: int, batch: int, lr: float,
                    quantile: float, stream=None):
    """Runs `steps` Adam steps in one launch; returns the per-step losses (device tensor)."""
    import torch
    hist = torch.empty(max(1, steps), dtype=torch.float32, device=X.device)
    _check(lib().spamm_mlp_train(_ptr(weights), _ptr(m), _ptr(v), int(t0), _ptr(X), _ptr(y_true),
                                 _ptr(idx), int(steps), int(batch), float(lr), float(quantile),
                                 _ptr(hist), _stream(stream)), "spamm_mlp_train")
    return hist[:steps]


TAU_WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                                "tau_mlp_leaf64.f32")


def load_tau_weights(device=None, path: str = TAU_WEIGHTS_PATH):
    """The trained learned-tau network (leaf 64) as a device float32 tensor [8449]."""
    import numpy as np
    import torch
    w = np.fromfile(path, dtype=np.float32)
    if w.size != spamm_mlp_param_count():
        raise RuntimeError(f"{path}: {w.size} values, expected {spamm_mlp_param_count()}")
    return torch.from_numpy(w).to(device or torch.device("cuda"))


def spamm_selftest_bounded_wait(limit_ns: int = 20_000_000, stream=None) -> int:
    """Bounded-wait self-test; returns the nanoseconds the wait took before giving up."""
    e = ctypes.c_int64()
    _check(lib().spamm_selftest_bounded_wait(int(limit_ns), ctypes.byref(e), _stream(stream)),
           "spamm_selftest_bounded_wait")
    return e.value


def spamm_last_device_status(stream=None) -> int:
    c = ctypes.c_int32()
    _check(lib().spamm_last_device_status(_stream(stream), ctypes.byref(c)),
           "spamm_last_device_status")
    return c.value


def spamm(A, B, leaf: int, tau: float, precision: int = FP32, target_rel_err: float = 1e-5,
          stream=None):
    """One SpAMM call through the library: norm maps, plan, multiply. Returns (C, plan)."""
    nA = spamm_normmap(A, leaf, stream=stream)
    nB = spamm_normmap(B, leaf, stream=stream)
    plan = spamm_plan(nA, nB, A.shape[0], leaf, tau, precision, target_rel_err, stream)
    C = spamm_multiply(plan, A, B, stream=stream)
    return C, plan
