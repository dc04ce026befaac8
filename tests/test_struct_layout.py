"""The binding's ctypes mirrors of the C-ABI structs have the header's layout.

ctypes cannot read a C header, so the binding restates each struct of
include/vrprpd.h field by field; a field missing, reordered or of the wrong
width would shift every later field and the library would read garbage
without any error.  This test compiles a small C program against the header
(gcc, no GPU) that prints sizeof of each struct and offsetof of each field the
mirror names, and compares them with the mirror's own layout.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def mirrors():
    import paper_2602_23685_gb300 as vrp
    from paper_2602_23685_gb300 import _search_sig as sig
    return {
        "vrprpd_batch": vrp.Batch,
        "vrprpd_batch16": vrp.Batch,            # the same layout, 16-bit element pointers
        "vrprpd_eval_config": vrp.EvalConfig,
        "vrprpd_solution": sig.Solution,
        "vrprpd_alns_params": sig.AlnsParams,
        "vrprpd_alns_stats": sig.AlnsStats,
        "vrprpd_brkga_params": sig.BrkgaParams,
        "vrprpd_request": sig.Request,
        "vrprpd_result": sig.Result,
        "vrprpd_server_stats": sig.ServerStats,
    }


def c_layout(structs, tmp_path):
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "vrprpd.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_mirrors_match_the_header(tmp_path):
    structs = mirrors()
    got = c_layout(structs, tmp_path)
    bad = []
    for cname, cls in structs.items():
        if got[(cname, "sizeof")] != ctypes.sizeof(cls):
            bad.append((cname, "sizeof", got[(cname, "sizeof")], ctypes.sizeof(cls)))
        for f in cls._fields_:
            if got[(cname, f[0])] != getattr(cls, f[0]).offset:
                bad.append((cname, f[0], got[(cname, f[0])], getattr(cls, f[0]).offset))
    assert not bad, bad


def header_defines():
    import re
    text = open(os.path.join(ROOT, "include", "vrprpd.h")).read()
    out = {}
    for m in re.finditer(r"^#define\s+(VRPRPD_\w+)\s+\(?(-?\d+)u?\)?", text, re.M):
        out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_the_header():
    """The binding's names for the header's distance modes, walks and
    chromosome layouts carry the header's values."""
    import paper_2602_23685_gb300 as vrp
    d = header_defines()
    for name, v in vrp.DIST_MODES.items():
        assert d["VRPRPD_DIST_" + name.upper()] == v, name
    for name, v in vrp.WALKS.items():
        assert d["VRPRPD_WALK_" + name.upper()] == v, name
    assert d["VRPRPD_LAYOUT_VKEYS"] == vrp.LAYOUT_VKEYS and d["VRPRPD_LAYOUT_HINTS"] == vrp.LAYOUT_HINTS
    # the error codes and status bits the tests name
    assert d["VRPRPD_ETIMEOUT"] == -4 and d["VRPRPD_EINVAL"] == -1
    assert (d["VRPRPD_CYCLE"], d["VRPRPD_VEH_CAP"], d["VRPRPD_POOL"], d["VRPRPD_MALFORMED"]) == (1, 2, 4, 8)
