"""The summation order the CUDA library's norm and inner-product kernels
promise (k_residual / k_dot partial sums, then k_norm_finalize), written out in
numpy so that tests can check that the device reduction follows it bit for bit.

This is a convention checker for the kernels, not part of the oracle: the
oracle defines the norm as the plain sum of squares (numpy's sum), which has no
block or thread structure, and the solve histories are compared with it at the
stated tolerance (every entry within 1e-12 ||r_0||, 1e-12 relative while above
1e-3 ||r_0||, identical iteration counts).

The order, FP64, one rounding per addition:
  1. for b < G = min(n_rows, 1024) and t < 256, a running sum over the rows
     j = b, b+G, ... (outer) and the columns i = t, t+256, ... (inner);
  2. per b, a halving tree over t: s[t] += s[t + h] for h = 128, 64, ..., 1;
  3. over the G block sums: running sums over b = t, t+256, ... per t < 256,
     then the same halving tree.
In the fused arithmetic mode the products of step 1 are fused into the
running sums (acc = fma(v, w, acc)); steps 2 and 3 are unchanged.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.fused import fma

BLOCKS = 1024
THREADS = 256


def device_order_sum(v: np.ndarray, w: np.ndarray | None = None) -> float:
    """Sum of an (n_rows, n_cols) array in the device's order; with w given,
    the sum of the products v w with each product fused into step 1."""
    v = np.asarray(v, dtype=np.float64)
    if w is not None:
        w = np.asarray(w, dtype=np.float64)
    n_rows, n_cols = v.shape
    G = min(n_rows, BLOCKS)
    T = THREADS
    acc = np.zeros((G, T))
    for k in range(0, (n_rows + G - 1) // G):
        rows = v[k * G:(k + 1) * G]
        for m in range(0, (n_cols + T - 1) // T):
            blk = rows[:, m * T:(m + 1) * T]
            a = acc[:blk.shape[0], :blk.shape[1]]
            if w is None:
                a[...] = a + blk
            else:
                a[...] = fma(blk, w[k * G:(k + 1) * G, m * T:(m + 1) * T], a)
    acc = _halving_tree(acc)
    parts = np.zeros(((G + T - 1) // T) * T)
    parts[:G] = acc
    fin = np.zeros((1, T))
    for m in range(0, len(parts) // T):
        fin[0] = fin[0] + parts[m * T:(m + 1) * T]
    return float(_halving_tree(fin)[0])


def _halving_tree(a: np.ndarray) -> np.ndarray:
    a = a.copy()
    h = a.shape[1] // 2
    while h >= 1:
        a[:, :h] = a[:, :h] + a[:, h:2 * h]
        h //= 2
    return a[:, 0]


def device_norm(r: np.ndarray, fused: bool = False) -> float:
    """||r|| over the interior of an (n+2)^2 array in the device's order."""
    v = np.asarray(r, dtype=np.float64)[1:-1, 1:-1]
    return math.sqrt(device_order_sum(v, v) if fused else device_order_sum(v * v))


def device_inner(fused: bool = False):
    """inner(a, b) over the interior of two (n+2)^2 arrays in the device's
    order, for the oracle solves' `inner` argument: the sum of the rounded
    products, or (fused arithmetic mode) of the products fused into step 1."""
    def inner(a, b):
        a = np.asarray(a, dtype=np.float64)[1:-1, 1:-1]
        b = np.asarray(b, dtype=np.float64)[1:-1, 1:-1]
        return device_order_sum(a, b) if fused else device_order_sum(a * b)
    return inner
