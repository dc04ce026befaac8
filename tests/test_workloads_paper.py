"""The paper's own instance rules (Section 5.1) in the input generator: the
fleet by instance size, and the processing-time variants drawn between the
instance's extreme edge weights (checked against the oracle's EUC_2D matrix,
computed independently of the generator)."""
import numpy as np
import pytest

import oracle
import workloads


def test_fleet_rule():
    assert workloads.paper_fleet(23) == (3, 5, 15)
    assert workloads.paper_fleet(24) == (6, 4, 24)
    assert workloads.paper_fleet(1000)[:2] == (6, 4)


@pytest.mark.parametrize("layout", ["uniform", "clustered"])
@pytest.mark.parametrize("n", [5, 23, 24, 150])
def test_variants(layout, n):
    ws = {v: workloads.make_paper_instance(n, v, layout, seed=n) for v in ("base", "2x", "5x", "1R10", "1R20")}
    d = oracle.euc2d(ws["base"].coords).astype(np.int64)
    off_diag = d[~np.eye(n + 1, dtype=bool)]
    base = ws["base"].p.astype(np.int64)
    assert base.min() >= off_diag.min() and base.max() <= off_diag.max()
    assert np.array_equal(ws["2x"].p, 2 * base) and np.array_equal(ws["5x"].p, 5 * base)
    for v, hi in (("1R10", 10), ("1R20", 20)):
        p = ws[v].p.astype(np.int64)
        nz = base > 0
        assert (p[~nz] == 0).all()
        k = p[nz] // base[nz]
        assert np.array_equal(k * base[nz], p[nz]) and k.min() >= 1 and k.max() <= hi
    for w in ws.values():
        assert (w.m, w.Q, w.R) == workloads.paper_fleet(n)
        assert np.array_equal(w.coords, ws["base"].coords)
