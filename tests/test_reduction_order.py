"""The device summation order (tests/reduction_order.py), written out point by
point: the helper the GPU tests use to check the norm kernels bit for bit is
the order it states, and it is the sum to within rounding."""
import math

import numpy as np
import pytest

import workloads as w
from reduction_order import device_norm, device_order_sum
from test_oracle_fused import fma_exact64


def _tree(s):
    s = list(s)
    h = len(s) // 2
    while h >= 1:
        for t in range(h):
            s[t] = s[t] + s[t + h]
        h //= 2
    return s[0]


def _stated_order(v, u=None):
    rows, cols = v.shape
    G, T = min(rows, 1024), 256
    acc = [[0.0] * T for _ in range(G)]
    for b in range(G):
        for j in range(b, rows, G):
            for i in range(cols):
                if u is None:
                    acc[b][i % T] = acc[b][i % T] + float(v[j, i])
                else:
                    acc[b][i % T] = fma_exact64(v[j, i], u[j, i], acc[b][i % T])
    parts = [_tree(a) for a in acc]
    parts += [0.0] * (-len(parts) % T)
    fin = [0.0] * T
    for m in range(len(parts) // T):
        for t in range(T):
            fin[t] = fin[t] + parts[m * T + t]
    return _tree(fin)


@pytest.mark.parametrize("shape", [(3, 600), (1100, 3), (17, 300)])
def test_device_order_is_the_stated_order(shape):
    rng = np.random.default_rng(4)
    v = rng.standard_normal(shape)
    u = rng.standard_normal(shape)
    assert device_order_sum(v) == _stated_order(v)
    assert device_order_sum(v, u) == _stated_order(v, u)


@pytest.mark.parametrize("n", [3, 7, 255, 1023, 1500])
def test_device_order_is_the_sum(n):
    v = w.normal(900 + n, n * n).reshape(n, n)
    exact = math.fsum(v.reshape(-1))
    assert abs(device_order_sum(v) - exact) <= 4 * n * n * 2.3e-16 * np.abs(v).sum()
    ints = np.round(v * 1000)
    assert device_order_sum(ints) == math.fsum(ints.reshape(-1))
    r = np.pad(v, 1)
    assert device_norm(r) == pytest.approx(math.sqrt(math.fsum((v * v).reshape(-1))), rel=1e-14)


@pytest.mark.parametrize("case,n,prec", [("binary", 127, "fp64"), ("binary", 127, "fp32"), ("lognormal", 63, "bf16"),
                                         ("poisson", 63, "fp64"), ("contrast1e6", 127, "fp64")])
def test_fcg_reading_holds_between_summation_orders(case, n, prec):
    """Flexible CG feeds its inner products back into the iterates, so the
    oracle run with the plain sum and the one with the device's summation order
    take different iterates at rounding level, amplified by the conditioning
    and, with an FP32/BF16 preconditioner, by the FP32 rounding of z.  The
    stated reading for FCG holds between them: identical iteration counts,
    entries above 1e-3 ||r_0|| within 1e-6 relative, the others within
    1e-9 ||r_0||."""
    from oracle import boxmg as bx
    from oracle import mixed as mx
    from reduction_order import device_inner
    from test_gpu_parity import problem
    tol = 1e-10
    if case == "contrast1e6":
        kind, planes, f = w.binary_contrast_problem(n, 8, 1.0, 1e6, seed_k=6, seed_f=7)
        tol = 1e-8
    else:
        kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes)
    if prec == "fp64":
        run = lambda inner=None: bx.solve_fcg(levels, f, tol=tol, maxit=300, inner=inner)
    else:
        l32 = mx.lower(levels, 0 if prec == "fp32" else 2)
        run = lambda inner=None: mx.solve_fcg_ir(levels, l32, f, tol=tol, maxit=300, inner=inner)
    (xa, ha), (xb, hb) = run(), run(device_inner())
    assert len(ha) == len(hb)
    for g, t in zip(hb, ha):
        assert abs(g - t) <= (1e-6 * t if t >= 1e-3 * ha[0] else 1e-9 * ha[0])
