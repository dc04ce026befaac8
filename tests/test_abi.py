"""The C-ABI library loads and exports every function include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(vrprpd_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2602_23685_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2602_23685_gb300 as vrp
    import numpy as np
    with pytest.raises(RuntimeError):
        vrp.Instance(2, 4, 4, np.array([1, 2], np.int32), coords=np.zeros((3, 2), np.int32))


def test_oracle_not_imported_by_product():
    pkg = os.path.join(ROOT, "paper_2602_23685_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text and "oracle/" not in text, path


def test_noalloc_launch_shape_stays_inside_the_scratch():
    """The allocation-free entry point's launch shape (a host function, no
    GPU): blocks x threads never exceeds the threads the fixed 4 Mi-word
    scratch holds, blocks shrink below 128 threads when fewer fit, and an
    instance that leaves room for fewer than 32 threads is refused."""
    from paper_2602_23685_gb300.build import build
    lib = ctypes.CDLL(build())
    fn = lib.vrprpd_evaluate_plain_noalloc_shape
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                   ctypes.POINTER(ctypes.c_int32)]
    fn.restype = ctypes.c_int
    scratch = 4 << 20

    def words(n, m):
        return (n + 1) + 3 * m + (2 * n + 2 + 31) // 32

    def shape(n, m, num):
        b, t = ctypes.c_int32(), ctypes.c_int32()
        rc = fn(n, m, num, ctypes.byref(b), ctypes.byref(t))
        return rc, b.value, t.value

    # n where room for 32..127 threads remains (the range a fixed 128-thread
    # block overran), then around both thresholds
    cases = [(100, 4), (1000, 20), (20000, 4096), (31000, 2), (40000, 2), (60000, 1), (100000, 3)]
    for n in range(1, 130000, 997):
        cases.append((n, 1 + n % 40))
    for n, m in cases:
        w = words(n, m)
        cap = scratch // w
        for num in (1, 33, 127, 128, 129, 10**6, 10**9):
            rc, b, t = shape(n, m, num)
            if cap < 32:
                assert rc != 0, (n, m)
                continue
            assert rc == 0, (n, m, num)
            assert t % 32 == 0 and 32 <= t <= 128 and b >= 1
            assert b * t <= cap, (n, m, num, b, t, cap)
            assert t == min(128, cap // 32 * 32)
            assert b == min(max(1, -(-num // t)), cap // t)
    # the exact boundary: the largest n (m = 1) that still fits 32 threads
    n = max(n for n in range(120000, 126000) if scratch // words(n, 1) >= 32)
    assert shape(n, 1, 1000)[0] == 0 and shape(n + 1, 1, 1000)[0] != 0
    assert shape(0, 1, 10)[0] != 0 and shape(10, 0, 10)[0] != 0 and shape(10, 1, -1)[0] != 0
