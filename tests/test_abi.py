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
