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


BATCH_GRAPH, BATCH_DYNAMIC, BATCH_TIMING, BATCH_GROUPS = 1, 2, 4, 8


class Tune(ctypes.Structure):
    """One autotuner candidate (spamm_tune_t)."""
    _fields_ = [("leaf", ctypes.c_int32), ("flags", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        sched = ("dynamic" if self.flags & BATCH_DYNAMIC else
                 "groups" if self.flags & BATCH_GROUPS else "static")
        return {"leaf": self.leaf, "schedule": sched, "flags": self.flags, "ms": self.ms}

_lib = None

_VP, _I64, _I32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_SIGS = {
    "spamm_normmap": [_VP, _I64, _I32, _VP, _VP],
    "spamm_plan_workspace_size": [_I64, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)],
    "spamm_plan_create": [ctypes.POINTER(_VP), _I64, _I32, _I32, _VP, ctypes.c_size_t],
    "spamm_plan_destroy": [_VP],
    "spamm_plan_set_schedule": [_VP, _I32],
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
    "spamm_normmap_rect": [_VP, _I64, _I64, _I64, _I32, _VP, _VP],
    "spamm_normmap_pair": [_VP, _VP, _I64, _I32, _VP, _VP, _VP],
    "spamm_plan_workspace_size_general": [_I64, _I64, _I64, _I32, _I32,
                                          ctypes.POINTER(ctypes.c_size_t)],
    "spamm_plan_create_general": [ctypes.POINTER(_VP), _I64, _I64, _I64, _I32, _I32, _VP,
                                  ctypes.c_size_t],
    "spamm_multiply_general": [_VP, _VP, _I64, _VP, _I64, _VP, _I64, ctypes.c_float,
                               ctypes.c_float, _VP, _VP],
    "spamm_plan_multiply_general": [_VP, _VP, _VP, _D, _D, _VP, _I64, _VP, _I64, _VP, _I64,
                                    ctypes.c_float, ctypes.c_float, _VP, _VP],
    "spamm_peak_rates": [_VP, _VP],
    "spamm_tau_certify": [_VP, _VP, _VP, _D, ctypes.POINTER(_D), ctypes.POINTER(_D), _VP],
    "spamm_tau_error": [_VP, _VP, _VP, _VP, _VP, _D, _D, _VP, ctypes.POINTER(_D), _VP],
    "spamm_tau_select": [_VP, _VP, _VP, _VP, _VP, _D, _VP, _VP, ctypes.POINTER(_D),
                         ctypes.POINTER(_I32), ctypes.POINTER(_D), _VP],
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


# Tensor checks.  The C ABI sees bare pointers, so it cannot tell a CPU tensor, a wrong dtype,
# a strided view or a short buffer from a valid operand; those are caught here, before any
# pointer reaches a kernel, and reported as SPAMM_ERR_INVALID_ARG like the library's own
# argument errors.  Alignment, aliasing and value checks stay in the library.

_DEVICE_TYPE = "cuda"
MLP_INPUTS = 65


def _bad(where: str, what: str):
    raise SpammError(1, f"{where}: {what}")


def _current_index() -> int:
    """Index of the current CUDA device: the library launches every kernel there, so every
    tensor of a call must live on it (a tensor on another GPU would be read through an
    address that GPU 0 cannot reach)."""
    import torch
    return torch.cuda.current_device()


def _index_of(t) -> int:
    return t.device.index if t.device.index is not None else 0


def _tensor(t, where: str, name: str, dtype, numel=None, square=None, min_numel=None):
    """Pointer of ``t`` after checking device, dtype, contiguity and size.

    ``numel``: the exact element count; ``min_numel``: the least one; ``square``: the side n
    of an n x n matrix."""
    import torch
    if not isinstance(t, torch.Tensor):
        _bad(where, f"{name} is not a tensor")
    if t.device.type != _DEVICE_TYPE:
        _bad(where, f"{name} is on {t.device}, not on the GPU")
    cur = _current_index()
    if _index_of(t) != cur:
        _bad(where, f"{name} is on {t.device}, but the current device is {cur}")
    if t.dtype != dtype:
        _bad(where, f"{name} is {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        _bad(where, f"{name} is not contiguous")
    if square is not None and (t.dim() != 2 or t.shape[0] != square or t.shape[1] != square):
        _bad(where, f"{name} has shape {tuple(t.shape)}, expected ({square}, {square})")
    if numel is not None and t.numel() != numel:
        _bad(where, f"{name} has {t.numel()} elements, expected {numel}")
    if min_numel is not None and t.numel() < min_numel:
        _bad(where, f"{name} has {t.numel()} elements, expected at least {min_numel}")
    return ctypes.c_void_p(t.data_ptr())


_F32 = None


def _mat_ptr(t, where: str, name, n: int, dev=None) -> int:
    """Address of an n x n contiguous FP32 tensor on the current GPU (fast path; _tensor names
    the fault).  ``dev``: the current device index, when the caller already has it."""
    global _F32
    if _F32 is None:
        import torch
        _F32 = torch.float32
    if dev is None:
        dev = _current_index()
    try:
        ok = (t.dtype is _F32 and t.shape == (n, n) and t.is_contiguous() and
              (t.is_cuda and t.get_device() == dev if _DEVICE_TYPE == "cuda" else
               t.device.type == _DEVICE_TYPE and _index_of(t) == dev))
    except AttributeError:
        ok = False
    if not ok:
        if not isinstance(name, str):             # ("As", i): formatted only on failure
            name = "%s[%d]" % name
        return _tensor(t, where, name, _F32, square=n).value
    return t.data_ptr()


def _mat(t, where: str, name: str, n: int):
    return ctypes.c_void_p(_mat_ptr(t, where, name, n))


def _rowmajor(t, where: str, name: str, rows: int, cols: int):
    """(pointer, leading dimension) of a rows x cols FP32 GPU tensor whose rows are contiguous
    (a row-major matrix or a view of one: stride(1) == 1, stride(0) >= cols)."""
    import torch
    if not isinstance(t, torch.Tensor):
        _bad(where, f"{name} is not a tensor")
    if t.device.type != _DEVICE_TYPE:
        _bad(where, f"{name} is on {t.device}, not on the GPU")
    cur = _current_index()
    if _index_of(t) != cur:
        _bad(where, f"{name} is on {t.device}, but the current device is {cur}")
    if t.dtype != torch.float32:
        _bad(where, f"{name} is {t.dtype}, expected torch.float32")
    if t.dim() != 2 or t.shape[0] != rows or t.shape[1] != cols:
        _bad(where, f"{name} has shape {tuple(t.shape)}, expected ({rows}, {cols})")
    ld = t.stride(0) if rows > 1 else max(cols, t.stride(0))
    if (t.stride(1) != 1 and cols > 1) or ld < cols:
        _bad(where, f"{name} rows are not contiguous (strides {tuple(t.stride())})")
    return ctypes.c_void_p(t.data_ptr()), ld


def _side(t, where: str, name: str) -> int:
    """n of an n x n operand (checked to be 2-D and square by the caller's _mat)."""
    if getattr(t, "dim", lambda: 0)() != 2:
        _bad(where, f"{name} must be a 2-D n x n tensor")
    return int(t.shape[0])


def _norms(t, where: str, name: str, bd: int):
    import torch
    return _tensor(t, where, name, torch.float64, numel=bd * bd)


_PARAMS = None


def _weights(t, where: str, name: str = "weights"):
    import torch
    global _PARAMS
    if _PARAMS is None:
        _PARAMS = spamm_mlp_param_count()
    return _tensor(t, where, name, torch.float32, numel=_PARAMS)


def _features_arg(X, where: str):
    import torch
    if getattr(X, "dim", lambda: 0)() != 2 or X.shape[1] != MLP_INPUTS:
        _bad(where, f"X must be [count, {MLP_INPUTS}]")
    return _tensor(X, where, "X", torch.float32)


def num_blocks(n: int, leaf: int) -> int:
    return -(-n // leaf)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def spamm_normmap(X, leaf: int, out=None, stream=None):
    """Leaf Frobenius norms of the n x n FP32 device tensor X -> FP64 [bd, bd] tensor."""
    import torch
    n = _side(X, "spamm_normmap", "X")
    x = _mat(X, "spamm_normmap", "X", n)
    bd = num_blocks(n, leaf) if leaf > 0 else 0
    if out is None:
        out = torch.empty((bd, bd), dtype=torch.float64, device=X.device)
    o = _norms(out, "spamm_normmap", "out", bd)
    _check(lib().spamm_normmap(x, n, leaf, o, _stream(stream)), "spamm_normmap")
    return out


def spamm_normmap_pair(A, B, leaf: int, outA=None, outB=None, stream=None):
    """Norm maps of both n x n operands of a product in one launch -> (normA, normB)."""
    import torch
    w = "spamm_normmap_pair"
    n = _side(A, w, "A")
    a, b = _mat(A, w, "A", n), _mat(B, w, "B", n)
    bd = num_blocks(n, leaf) if leaf > 0 else 0
    if outA is None:
        outA = torch.empty((bd, bd), dtype=torch.float64, device=A.device)
    if outB is None:
        outB = torch.empty((bd, bd), dtype=torch.float64, device=A.device)
    _check(lib().spamm_normmap_pair(a, b, n, leaf, _norms(outA, w, "normA", bd),
                                    _norms(outB, w, "normB", bd), _stream(stream)), w)
    return outA, outB


class Plan:
    """Owns a spamm_plan_t (work queues for one (n, leaf, precision))."""

    def __init__(self, n: int, leaf: int, precision: int = FP32, workspace=None):
        self.n, self.leaf, self.precision = n, leaf, precision
        self.bd = num_blocks(n, leaf) if leaf > 0 else 0
        self.m, self.k = n, n
        self.bm = self.bk = self.bn = self.bd
        h = ctypes.c_void_p()
        ws_ptr, ws_bytes = (None, 0) if workspace is None else (
            _tensor(workspace, "spamm_plan_create", "workspace", workspace.dtype),
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

    def set_schedule(self, schedule: str = "static"):
        """Tile order of later multiplies: "static", "dynamic" or "groups" (same bits)."""
        flags = {"static": 0, "dynamic": BATCH_DYNAMIC, "groups": BATCH_GROUPS}
        if schedule not in flags:
            raise SpammError(1, "spamm_plan_set_schedule")
        _check(lib().spamm_plan_set_schedule(self.handle, flags[schedule]), "spamm_plan_set_schedule")
        return self

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
        w = "spamm_plan"
        _check(lib().spamm_plan(self.handle, self._na(normA, w), self._nb(normB, w), float(tau),
                                float(target_rel_err), _stream(stream)), w)
        return self

    def _na(self, t, w):
        import torch
        return _tensor(t, w, "normA", torch.float64, numel=self.bm * self.bk)

    def _nb(self, t, w):
        import torch
        return _tensor(t, w, "normB", torch.float64, numel=self.bk * self.bn)

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(lib().spamm_plan_stats(self.handle, ctypes.byref(s), _stream(stream)),
               "spamm_plan_stats")
        return s.as_dict()

    def export(self, stream=None):
        """(tile_ptr int32[bd*bd+1], k_idx uint16[S]) as numpy arrays."""
        import numpy as np
        st = self.stats(stream)
        tp = np.zeros(self.bm * self.bn + 1, dtype=np.int32)
        kk = np.zeros(max(1, st["survivors"]), dtype=np.uint16)
        _check(lib().spamm_plan_export(self.handle, tp.ctypes.data_as(ctypes.c_void_p),
                                       kk.ctypes.data_as(ctypes.c_void_p), kk.size,
                                       _stream(stream)), "spamm_plan_export")
        return tp, kk[:st["survivors"]]

    def multiply(self, A, B, C, stream=None):
        w, n = "spamm_multiply", self.n
        _check(lib().spamm_multiply(self.handle, _mat(A, w, "A", n), _mat(B, w, "B", n),
                                    _mat(C, w, "C", n), _stream(stream)), w)
        return C

    def plan_multiply(self, normA, normB, tau: float, A, B, C, target_rel_err: float = 1e-5,
                      stream=None):
        """plan() then multiply() in one call (zero-fill of empty tiles overlapped)."""
        w, n = "spamm_plan_multiply", self.n
        _check(lib().spamm_plan_multiply(self.handle, self._na(normA, w), self._nb(normB, w),
                                         float(tau),
                                         float(target_rel_err), _mat(A, w, "A", n),
                                         _mat(B, w, "B", n), _mat(C, w, "C", n),
                                         _stream(stream)), w)
        return C

    def band(self, normA, normB, tau_lo: float, tau_hi: float, stream=None):
        """Plan the triples with tau_lo <= p < tau_hi (error measurement)."""
        w = "spamm_plan_band"
        _check(lib().spamm_plan_band(self.handle, self._na(normA, w), self._nb(normB, w),
                                     float(tau_lo),
                                     float(tau_hi), _stream(stream)), w)
        return self

    def tau_for_valid_ratio(self, normA, normB, target: float, tol: float = 0.01,
                            max_probes: int = 20, stream=None):
        """(tau, valid ratio, probes) of the valid-ratio search (Section 3.5.2)."""
        t, r, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        w = "spamm_tau_for_valid_ratio"
        _check(lib().spamm_tau_for_valid_ratio(self.handle, self._na(normA, w),
                                               self._nb(normB, w),
                                               float(target), float(tol), int(max_probes),
                                               ctypes.byref(t), ctypes.byref(r), ctypes.byref(k),
                                               _stream(stream)), "spamm_tau_for_valid_ratio")
        return t.value, r.value, k.value

    def histogram(self, normA, normB, stream=None):
        """Raw counts of the 64-bin log2 histogram of relative norm products."""
        import numpy as np
        out = np.zeros(64, dtype=np.int64)
        w = "spamm_norm_histogram"
        _check(lib().spamm_norm_histogram(self.handle, self._na(normA, w), self._nb(normB, w),
                                          out.ctypes.data_as(ctypes.c_void_p), _stream(stream)), w)
        return out

    def tau_certify(self, normA, normB, ref_rel: float = 1e-11, stream=None):
        """(tau_ref, ||A||_F ||B||_F): the largest tau on the certification grid whose skipped
        bound2 is <= ref_rel ||A|| ||B||."""
        t, ab = ctypes.c_double(), ctypes.c_double()
        w = "spamm_tau_certify"
        _check(lib().spamm_tau_certify(self.handle, _norms(normA, w, "normA", self.bd),
                                       _norms(normB, w, "normB", self.bd), float(ref_rel),
                                       ctypes.byref(t), ctypes.byref(ab), _stream(stream)), w)
        return t.value, ab.value

    def tau_error(self, normA, normB, A, B, tau: float, tau_ref: float, scratch,
                  stream=None) -> float:
        """e(tau) = ||AB - SpAMM(tau)||_F / (||A|| ||B||) up to the certified tau_ref's bound."""
        out = ctypes.c_double()
        w, n, bd = "spamm_tau_error", self.n, self.bd
        _check(lib().spamm_tau_error(self.handle, _norms(normA, w, "normA", bd),
                                     _norms(normB, w, "normB", bd), _mat(A, w, "A", n),
                                     _mat(B, w, "B", n), float(tau), float(tau_ref),
                                     _mat(scratch, w, "scratch", n), ctypes.byref(out),
                                     _stream(stream)), w)
        return out.value

    def tau_select(self, normA, normB, A, B, target_rel_err: float, weights=None, scratch=None,
                   stream=None):
        """(tau, evaluations of e, e(tau)): the network's tau checked once, bisection on the
        error on a miss (or without weights)."""
        import torch
        w, n, bd = "spamm_tau_select", self.n, self.bd
        if scratch is None:
            scratch = torch.empty_like(A)
        t, k, e = ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().spamm_tau_select(self.handle, _norms(normA, w, "normA", bd),
                                      _norms(normB, w, "normB", bd), _mat(A, w, "A", n),
                                      _mat(B, w, "B", n), float(target_rel_err),
                                      None if weights is None else _weights(weights, w),
                                      _mat(scratch, w, "scratch", n), ctypes.byref(t),
                                      ctypes.byref(k), ctypes.byref(e), _stream(stream)), w)
        return t.value, k.value, e.value

    def tau_predict(self, normA, normB, target_rel_err: float, weights, stream=None) -> float:
        """The network's tau for this plan's shape (weights: device float32 [8449])."""
        t = ctypes.c_double()
        w = "spamm_tau_predict"
        _check(lib().spamm_tau_predict(self.handle, self._na(normA, w), self._nb(normB, w),
                                       float(target_rel_err), _weights(weights, w),
                                       ctypes.byref(t), _stream(stream)), w)
        return t.value


class GeneralPlan(Plan):
    """A plan of the general form C = alpha * SpAMM(A, B) + beta * C with A m x k and B k x n
    (spamm_plan_create_general).  Norm maps are [bm, bk] (A) and [bk, bn] (B)."""

    def __init__(self, m: int, k: int, n: int, leaf: int, precision: int = FP32,
                 workspace=None):
        self.m, self.k, self.n, self.leaf, self.precision = m, k, n, leaf, precision
        self.bm, self.bk, self.bn = (num_blocks(x, leaf) if leaf > 0 else 0 for x in (m, k, n))
        self.bd = self.bm
        h = ctypes.c_void_p()
        ws_ptr, ws_bytes = (None, 0) if workspace is None else (
            _tensor(workspace, "spamm_plan_create_general", "workspace", workspace.dtype),
            workspace.numel() * workspace.element_size())
        _check(lib().spamm_plan_create_general(ctypes.byref(h), m, k, n, leaf, precision, ws_ptr,
                                               ws_bytes), "spamm_plan_create_general")
        self.handle = h
        self._workspace = workspace

    @staticmethod
    def workspace_size(m: int, k: int, n: int, leaf: int, precision: int = FP32) -> int:
        b = ctypes.c_size_t()
        _check(lib().spamm_plan_workspace_size_general(m, k, n, leaf, precision, ctypes.byref(b)),
               "spamm_plan_workspace_size_general")
        return b.value

    def _nc(self, t, w):
        import torch
        return None if t is None else _tensor(t, w, "normC", torch.float64,
                                               numel=self.bm * self.bn)

    def multiply(self, A, B, C, alpha: float = 1.0, beta: float = 0.0, normC=None, stream=None):
        """C = alpha * (pruned A B) + beta * C; A, B, C may be row-major views (contiguous rows).
        normC (float64 [bm, bn], optional) receives C's norm map as stored."""
        w = "spamm_multiply_general"
        a, lda = _rowmajor(A, w, "A", self.m, self.k)
        b, ldb = _rowmajor(B, w, "B", self.k, self.n)
        c, ldc = _rowmajor(C, w, "C", self.m, self.n)
        _check(lib().spamm_multiply_general(self.handle, a, lda, b, ldb, c, ldc, float(alpha),
                                            float(beta), self._nc(normC, w), _stream(stream)), w)
        return C

    def plan_multiply(self, normA, normB, tau: float, A, B, C, target_rel_err: float = 1e-5,
                      alpha: float = 1.0, beta: float = 0.0, normC=None, stream=None):
        w = "spamm_plan_multiply_general"
        a, lda = _rowmajor(A, w, "A", self.m, self.k)
        b, ldb = _rowmajor(B, w, "B", self.k, self.n)
        c, ldc = _rowmajor(C, w, "C", self.m, self.n)
        _check(lib().spamm_plan_multiply_general(self.handle, self._na(normA, w),
                                                 self._nb(normB, w), float(tau),
                                                 float(target_rel_err), a, lda, b, ldb, c, ldc,
                                                 float(alpha), float(beta), self._nc(normC, w),
                                                 _stream(stream)), w)
        return C


def spamm_normmap_rect(X, leaf: int, out=None, stream=None):
    """Leaf Frobenius norms of a rows x cols FP32 device matrix (contiguous rows, any leading
    dimension) -> FP64 [ceil(rows/leaf), ceil(cols/leaf)] tensor."""
    import torch
    w = "spamm_normmap_rect"
    if getattr(X, "dim", lambda: 0)() != 2:
        _bad(w, "X must be a 2-D tensor")
    rows, cols = int(X.shape[0]), int(X.shape[1])
    x, ld = _rowmajor(X, w, "X", rows, cols)
    br, bc = (num_blocks(rows, leaf), num_blocks(cols, leaf)) if leaf > 0 else (0, 0)
    if out is None:
        out = torch.empty((br, bc), dtype=torch.float64, device=X.device)
    o = _tensor(out, w, "out", torch.float64, numel=br * bc)
    _check(lib().spamm_normmap_rect(x, rows, cols, ld, leaf, o, _stream(stream)), w)
    return out


def spamm_general(A, B, leaf: int, tau: float, C=None, alpha: float = 1.0, beta: float = 0.0,
                  precision: int = FP32, target_rel_err: float = 1e-5, normC=None, stream=None):
    """One general-form call: norm maps of A (m x k) and B (k x n), plan, multiply into C
    (m x n, created when None; beta must be 0 then).  Returns (C, plan)."""
    import torch
    m, k = int(A.shape[0]), int(A.shape[1])
    n = int(B.shape[1])
    nA = spamm_normmap_rect(A, leaf, stream=stream)
    nB = spamm_normmap_rect(B, leaf, stream=stream)
    plan = GeneralPlan(m, k, n, leaf, precision)
    if C is None:
        if beta != 0.0:
            _bad("spamm_general", "beta != 0 needs C")
        C = torch.empty((m, n), dtype=torch.float32, device=A.device)
    plan.plan_multiply(nA, nB, tau, A, B, C, target_rel_err, alpha, beta, normC, stream)
    return C, plan


def spamm_plan(normA, normB, n: int, leaf: int, tau: float, precision: int = FP32,
               target_rel_err: float = 1e-5, stream=None) -> Plan:
    return Plan(n, leaf, precision).plan(normA, normB, tau, target_rel_err, stream)


def spamm_multiply(plan: Plan, A, B, C=None, stream=None):
    import torch
    if C is None:
        C = torch.empty_like(A)
    return plan.multiply(A, B, C, stream)


def spamm_frobenius_diff(X, Y=None, stream=None) -> float:
    import torch
    w = "spamm_frobenius_diff"
    x = _tensor(X, w, "X", torch.float32)
    y = None if Y is None else _tensor(Y, w, "Y", torch.float32, numel=X.numel())
    out = ctypes.c_double()
    _check(lib().spamm_frobenius_diff(x, y, X.numel(), ctypes.byref(out), _stream(stream)), w)
    return out.value


def spamm_multiply_fp32_noalloc(A, B, C, leaf: int, tau: float, stream=None):
    """FP32 SpAMM with no device allocation (static library scratch; ceil(n/leaf) <= 64)."""
    w = "spamm_multiply_fp32_noalloc"
    n = _side(A, w, "A")
    _check(lib().spamm_multiply_fp32_noalloc(_mat(A, w, "A", n), _mat(B, w, "B", n),
                                             _mat(C, w, "C", n), n, leaf, float(tau),
                                             _stream(stream)), w)
    return C


def _problems(As, Bs, Cs, taus, where: str, ns=None):
    """The problem table; every operand checked (n x n FP32 on the GPU, n = ns[i] if given).
    Cs may be None (no outputs: C stays NULL)."""
    count = len(As)
    if len(Bs) != count or (Cs is not None and len(Cs) != count) or len(taus) != count:
        _bad(where, "As, Bs, Cs and taus differ in length")
    if ns is not None and count != len(ns):
        _bad(where, f"{count} problems for a batch of {len(ns)}")
    arr = (Problem * count)()
    dev = _current_index()
    for i in range(count):
        A = As[i]
        n = _side(A, where, f"As[{i}]") if ns is None else ns[i]
        arr[i] = Problem(_mat_ptr(A, where, ("As", i), n, dev),
                         _mat_ptr(Bs[i], where, ("Bs", i), n, dev),
                         None if Cs is None else _mat_ptr(Cs[i], where, ("Cs", i), n, dev),
                         n, float(taus[i]))
    return arr


class Batch:
    """Owns a spamm_batch_t: many independent products of fixed shapes."""

    def __init__(self, ns, leaf: int, precision: int = FP32, graph: bool = True,
                 workspace=None, dynamic: bool = False, timing: bool = False,
                 groups: bool = False):
        self.ns = [int(n) for n in ns]
        self.leaf, self.precision = leaf, precision
        self.count = len(self.ns)
        n_arr = (ctypes.c_int64 * self.count)(*self.ns)
        ws_ptr, ws_bytes = (None, 0) if workspace is None else (
            _tensor(workspace, "spamm_batch_create", "workspace", workspace.dtype),
            workspace.numel() * workspace.element_size())
        h = ctypes.c_void_p()
        flags = ((BATCH_GRAPH if graph else 0) | (BATCH_DYNAMIC if dynamic else 0) |
                 (BATCH_TIMING if timing else 0) | (BATCH_GROUPS if groups else 0))
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
        probs = _problems(As, Bs, Cs, taus, "spamm_batch_run", self.ns)
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
        w = "spamm_batch_tau_predict"
        probs = _problems(As, Bs, None, [0.0] * len(As), w, self.ns)
        tg = np.ascontiguousarray(targets, dtype=np.float64)
        if tg.shape != (self.count,):
            _bad(w, f"{tg.size} targets for a batch of {self.count}")
        out = np.zeros(self.count, dtype=np.float64)
        _check(lib().spamm_batch_tau_predict(self.handle, ctypes.cast(probs, ctypes.c_void_p),
                                             tg.ctypes.data_as(ctypes.c_void_p),
                                             _weights(weights, w),
                                             out.ctypes.data_as(ctypes.c_void_p),
                                             _stream(stream)), w)
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
    probs = _problems(As, Bs, Cs, taus, "spamm_batch_autotune")
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
    probs = _problems(As, Bs, Cs, taus, "spamm_multiply_batched")
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
    w = "spamm_mlp_forward"
    x = _features_arg(X, w)
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(lib().spamm_mlp_forward(_weights(weights, w), x, X.shape[0], _ptr(y),
                                   _stream(stream)), w)
    return y


def spamm_mlp_grad(weights, X, y_true, quantile: float, stream=None):
    """(gradient [8449], loss tensor [1]) of the mean pinball loss."""
    import torch
    w = "spamm_mlp_grad"
    wp, x = _weights(weights, w), _features_arg(X, w)
    y = _tensor(y_true, w, "y_true", torch.float32, numel=X.shape[0])
    g = torch.empty_like(weights)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(lib().spamm_mlp_grad(wp, x, y, X.shape[0], float(quantile), _ptr(g), _ptr(loss),
                                _stream(stream)), w)
    return g, loss


def spamm_mlp_adam(weights, grad, m, v, t: int, lr: float, stream=None):
    w = "spamm_mlp_adam"
    _check(lib().spamm_mlp_adam(_weights(weights, w), _weights(grad, w, "grad"),
                                _weights(m, w, "m"), _weights(v, w, "v"), int(t), float(lr),
                                _stream(stream)), w)


def spamm_mlp_train(weights, m, v, t0: int, X, y_true, idx, steps: int, batch: int, lr: float,
                    quantile: float, stream=None):
    """Runs `steps` Adam steps in one launch; returns the per-step losses (device tensor).

    idx holds steps * batch sample indices (int32), each in [0, rows of X)."""
    import torch
    w = "spamm_mlp_train"
    args = (_weights(weights, w), _weights(m, w, "m"), _weights(v, w, "v"), int(t0),
            _features_arg(X, w), _tensor(y_true, w, "y_true", torch.float32, numel=X.shape[0]),
            _tensor(idx, w, "idx", torch.int32, min_numel=max(0, int(steps)) * max(0, int(batch))))
    hist = torch.empty(max(1, steps), dtype=torch.float32, device=X.device)
    _check(lib().spamm_mlp_train(*args, int(steps), int(batch), float(lr), float(quantile),
                                 _ptr(hist), _stream(stream)), w)
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


def spamm_peak_rates(stream=None) -> dict:
    """Measured peak rates of the current GPU (TFLOP/s): FP32 FFMA, FP64 DFMA and dense
    tcgen05 BF16, FP16 and TF32 MMA."""
    out = (ctypes.c_double * 5)()
    _check(lib().spamm_peak_rates(ctypes.cast(out, ctypes.c_void_p), _stream(stream)),
           "spamm_peak_rates")
    return dict(zip(("ffma_fp32", "dfma_fp64", "mma_bf16", "mma_fp16", "mma_tf32"), out))


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
