"""The oracle's row-band runner (used by the all-core CPU baseline): bands
partition the interior rows with odd first rows, and V(2,1) cycles and
residuals run over bands on several threads give the one-thread oracle's
values bit for bit (within one colour the points are decoupled)."""
import numpy as np
import pytest

import workloads as w
from oracle import boxmg as bx


@pytest.mark.parametrize("n,threads", [(255, 4), (511, 3), (1023, 16), (15, 8)])
def test_bands_partition_the_rows(n, threads):
    B = bx.RowBands(threads, min_rows=16)
    rows = []
    for b in B.slices(n):
        j0, j1 = b.start + 1, b.stop - 2
        assert j0 % 2 == 1 and 1 <= j0 <= j1 <= n
        rows.extend(range(j0, j1 + 1))
    assert rows == list(range(1, n + 1))
    B.close()


@pytest.mark.parametrize("case", ["poisson", "binary", "lognormal"])
@pytest.mark.parametrize("arith", ["rounded", "fused"])
def test_banded_cycles_equal_one_thread(case, arith):
    n = 255
    if case == "poisson":
        kind, planes, f = w.poisson_problem(n, 1)
    elif case == "binary":
        kind, planes, f = w.binary_contrast_problem(n, 16, seed_k=2, seed_f=3)
    else:
        kind, planes, f = w.lognormal_problem(n, 2.0, 8.0, seed_k=4, seed_f=7)
    levels = bx.setup(kind, planes, arith=arith)
    B = bx.RowBands(4, min_rows=16)
    x1, x2 = np.zeros_like(f), np.zeros_like(f)
    for _ in range(3):
        bx.vcycle(levels, 0, x1, f)
        bx.vcycle(levels, 0, x2, f, bands=B)
        assert np.array_equal(x1, x2)
    fu = arith == "fused"
    assert np.array_equal(bx.residual(levels[0].planes, x1, f, fu), bx.residual(levels[0].planes, x2, f, fu, B))
    B.close()
