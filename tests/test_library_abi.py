"""The C-ABI library loads on a CPU-only machine and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spamm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|spamm_status_t)\s+(spamm_\w+)\s*\(",
                                 src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_2103_13042_gb300 as P
    if not os.path.exists(P.LIB_PATH):
        from paper_2103_13042_gb300 import build
        build.build()
    return P.lib()


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for core in ("spamm_normmap", "spamm_plan", "spamm_multiply"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for code in range(7):
        assert lib.spamm_status_string(code)


def test_argument_validation_without_gpu(lib):
    """Host-side checks run before any CUDA call, so they work with no GPU."""
    b = ctypes.c_size_t()
    assert lib.spamm_plan_workspace_size(0, 64, 0, ctypes.byref(b)) == 1        # n < 1
    assert lib.spamm_plan_workspace_size(1024, 48, 0, ctypes.byref(b)) == 2     # leaf
    assert lib.spamm_plan_workspace_size(1024, 64, 9, ctypes.byref(b)) == 1     # precision
    assert lib.spamm_plan_workspace_size(1024, 64, 0, ctypes.byref(b)) == 0
    assert b.value > 1024 // 64 * 1024 // 64 * 1024 // 64 * 2                   # holds k_idx
    assert lib.spamm_normmap(None, 1024, 64, None, None) == 1
    assert lib.spamm_normmap(ctypes.c_void_p(16), 1024, 40, ctypes.c_void_p(16), None) == 2
    assert lib.spamm_normmap(ctypes.c_void_p(18), 1024, 64, ctypes.c_void_p(16), None) == 1
    assert lib.spamm_plan(None, None, None, 0.0, 0.0, None) == 1
    assert lib.spamm_plan_set_schedule(None, 0) == 1


def test_batch_validation_without_gpu(lib):
    """Batch shape checks run on the host before any CUDA call."""
    b = ctypes.c_size_t()
    ns = (ctypes.c_int64 * 3)(256, 1000, 4096)
    assert lib.spamm_batch_workspace_size(ns, 3, 64, 2, ctypes.byref(b)) == 0
    one = ctypes.c_size_t()
    ns1 = (ctypes.c_int64 * 1)(4096)
    assert lib.spamm_batch_workspace_size(ns1, 1, 64, 2, ctypes.byref(one)) == 0
    assert b.value > one.value
    assert lib.spamm_batch_workspace_size(ns, 0, 64, 2, ctypes.byref(b)) == 1     # count < 1
    assert lib.spamm_batch_workspace_size(ns, 3, 32, 2, ctypes.byref(b)) == 2     # tensor at 32
    assert lib.spamm_batch_workspace_size(ns, 3, 96, 0, ctypes.byref(b)) == 2     # leaf
    bad = (ctypes.c_int64 * 2)(256, 0)
    assert lib.spamm_batch_workspace_size(bad, 2, 64, 0, ctypes.byref(b)) == 1    # n < 1
    h = ctypes.c_void_p()
    assert lib.spamm_batch_create(ctypes.byref(h), ns, 3, 64, 0, 16, None, 0) == 1  # flags
    assert lib.spamm_batch_create(ctypes.byref(h), ns, 3, 64, 0, 2 | 8, None, 0) == 1  # dynamic + groups
    assert lib.spamm_batch_run(None, None, 0.0, None) == 1
    assert lib.spamm_batch_destroy(None) == 1


def test_shape_limits_without_gpu(lib):
    """The block grid is capped at 1024 leaf blocks a side: the largest n for each leaf is
    accepted, one more element is UNSUPPORTED (2), and n < 1 is INVALID_ARG (1)."""
    b = ctypes.c_size_t()
    for leaf in (32, 64, 128):
        n_max = 1024 * leaf
        assert lib.spamm_plan_workspace_size(n_max, leaf, 0, ctypes.byref(b)) == 0
        assert lib.spamm_plan_workspace_size(n_max + 1, leaf, 0, ctypes.byref(b)) == 2
        assert lib.spamm_normmap(ctypes.c_void_p(16), n_max + 1, leaf,
                                 ctypes.c_void_p(16), None) == 2
        assert lib.spamm_plan_workspace_size(-5, leaf, 0, ctypes.byref(b)) == 1
    assert lib.spamm_plan_workspace_size(1024, 64, 0, None) == 1              # null out
    assert lib.spamm_plan_workspace_size(1024, 32, 2, ctypes.byref(b)) == 2   # BF16 at leaf 32
    for prec in (1, 2, 3, 4, 5):                                              # tensor modes
        assert lib.spamm_plan_workspace_size(1024, 64, prec, ctypes.byref(b)) == 0
    assert lib.spamm_plan_workspace_size(1024, 64, -1, ctypes.byref(b)) == 1


def test_workspace_grows_with_n(lib):
    """The plan workspace holds the per-triple index lists, so it grows with the block count."""
    sizes = []
    for n in (256, 1024, 4096, 16384):
        b = ctypes.c_size_t()
        assert lib.spamm_plan_workspace_size(n, 64, 4, ctypes.byref(b)) == 0
        sizes.append(b.value)
    assert sizes == sorted(sizes) and len(set(sizes)) == len(sizes)
    bd = 16384 // 64
    assert sizes[-1] >= bd ** 3 * 2                                            # k_idx, 2 B each


def test_unknown_status_string(lib):
    lib.spamm_status_string.restype = ctypes.c_char_p
    assert lib.spamm_status_string(0) == b"ok"
    assert lib.spamm_status_string(5) == b"a bounded device wait timed out"
    assert lib.spamm_status_string(99) == b"unknown status"


def test_batch_index_range_limit_without_gpu(lib):
    """Tile ids and k slots of a batch are 32-bit on the device: one instance at the largest
    block grid (1024^3 slots) fits, two of them (2^31 slots) are UNSUPPORTED."""
    b = ctypes.c_size_t()
    one = (ctypes.c_int64 * 1)(65536)
    two = (ctypes.c_int64 * 2)(65536, 65536)
    assert lib.spamm_batch_workspace_size(one, 1, 64, 0, ctypes.byref(b)) == 0
    assert lib.spamm_batch_workspace_size(two, 2, 64, 0, ctypes.byref(b)) == 2
    big = (ctypes.c_int64 * 1)((1 << 20) + 1)
    assert lib.spamm_batch_workspace_size(big, 1, 128, 0, ctypes.byref(b)) == 2


def test_batch_of_one_holds_a_plan_and_its_norm_maps(lib):
    """A batch of one instance provisions the plan's workspace plus both norm maps."""
    for n, leaf, prec in ((1000, 64, 4), (4096, 128, 1), (777, 32, 0)):
        pw, bw = ctypes.c_size_t(), ctypes.c_size_t()
        assert lib.spamm_plan_workspace_size(n, leaf, prec, ctypes.byref(pw)) == 0
        ns = (ctypes.c_int64 * 1)(n)
        assert lib.spamm_batch_workspace_size(ns, 1, leaf, prec, ctypes.byref(bw)) == 0
        bd = -(-n // leaf)
        assert bw.value >= pw.value + 2 * 8 * bd * bd


def test_general_shape_validation_without_gpu(lib):
    """The general form's shape checks run on the host before any CUDA call."""
    b = ctypes.c_size_t()
    f = lib.spamm_plan_workspace_size_general
    f.argtypes = [ctypes.c_int64] * 3 + [ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_size_t)]
    assert f(0, 100, 100, 64, 0, ctypes.byref(b)) == 1                 # m < 1
    assert f(100, 100, 100, 48, 0, ctypes.byref(b)) == 2               # leaf
    assert f(100, 64 * 1025, 100, 64, 0, ctypes.byref(b)) == 2         # bk > 1024
    assert f(1 << 25, 100, 100, 64, 0, ctypes.byref(b)) == 2           # a dimension > 2^24
    assert f(64 * 4096, 64, 64 * 1025, 64, 0, ctypes.byref(b)) == 2    # bm * bn > 2^22
    assert f(100, 100, 100, 32, 2, ctypes.byref(b)) == 2               # tensor mode at leaf 32
    assert f(128, 576, 25600, 64, 2, ctypes.byref(b)) == 0             # the VGG13 conv21 shape
    small = b.value
    assert f(128, 576, 25600 * 2, 64, 2, ctypes.byref(b)) == 0 and b.value > small
    g = lib.spamm_multiply_general
    g.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                  ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
    assert g(None, None, 1, None, 1, None, 1, 1.0, 0.0, None, None) == 1
