"""Mixed-precision BoxMG oracle: FP32 (or BF16-stencil) V(2,1) cycles inside
FP64 iterative refinement.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's solver is FP64 throughout; this extension follows the stated
reading:

* outer loop in FP64: r = f - A x, rho = ||r||; scale s = 2^e with
  rho = m 2^e, 1/2 <= m < 1; r32 = fl32(r / s) (the division by a power of two
  is exact); e32 = V32(r32) from a zero guess; x = x + s * fl64(e32);
* the inner cycle runs the FP64 hierarchy rounded to FP32 (round to nearest
  even, numpy's cast), every operation in FP32 with one rounding each, the
  same expression orders as the FP64 oracle;
* BF16-stencil levels store W, S, SW, NW as bf16(fl32(a)) (round to nearest
  even on the float32 bit pattern), and recompute the diagonal in FP32 so that
  row sums stay what they were: O32 = fl32(sum_NBR a) - W_b - E_b - S_b - N_b
  - SW_b - NE_b - NW_b - SE_b, d32 = 1 / O32;
* the coarsest solve stays FP64: fl32(L^-T L^-1 fl64(f32));
* a hierarchy set up with arith="fused" fuses the multiply-adds of both the
  FP64 outer loop and the FP32 cycle (fmaf for FP32 operands); x + s e32 is
  the same either way (s e32 is exact).
"""
from __future__ import annotations

import math

import numpy as np

from . import boxmg as bx

F32 = np.float32


def bf16_round(a) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even) and
    return them as float32 with the low 16 bits zero.  Finite inputs only."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))
    u = ((u + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return u.view(np.float32).reshape(a.shape)


class Level32:
    def __init__(self, n, kind, planes, dinv, ci, L):
        self.n, self.kind, self.planes, self.dinv, self.ci, self.L = n, kind, planes, dinv, ci, L


def lower(levels, bf16_levels: int = 0) -> list[Level32]:
    """FP32 copy of an FP64 hierarchy; the first `bf16_levels` levels get
    BF16-stored off-diagonals and the recomputed FP32 diagonal."""
    out = []
    for li, lev in enumerate(levels):
        planes = lev.planes.astype(F32)
        dinv = lev.dinv.astype(F32)
        if li < bf16_levels:
            planes[1:] = bf16_round(planes[1:])
            p64 = lev.planes
            rs = bx.coupling(p64, 0, 0).copy()
            for d in bx.NBR[1:]:
                rs = rs + bx.coupling(p64, *d)
            o32 = rs.astype(F32)
            for d in bx.NBR[1:]:
                o32 = o32 - bx.coupling(planes, *d)
            bx.at(planes[0], 0, 0)[...] = o32
            dinv = np.zeros_like(planes[0])
            bx.at(dinv, 0, 0)[...] = F32(1) / o32
        ci = None if lev.ci is None else lev.ci.astype(F32)
        out.append(Level32(lev.n, lev.kind, planes, dinv, ci, lev.L))
        out[-1].smoother = getattr(lev, "smoother", "point")
        out[-1].fused = getattr(lev, "fused", False)
    return out


def scale_of(rho: float) -> float:
    """The power of two 2^e with rho = m 2^e, 1/2 <= m < 1 (1 for rho = 0)."""
    if rho == 0.0 or not math.isfinite(rho):
        return 1.0
    return math.ldexp(1.0, math.frexp(rho)[1])


def inner_cycle(levels32, r32, cycles: int = 1, nu1=2, nu2=1) -> np.ndarray:
    """e32 = `cycles` FP32 V-cycles on A e = r32 from e = 0."""
    e = np.zeros_like(r32)
    for _ in range(cycles):
        bx.vcycle(levels32, 0, e, r32, nu1, nu2)
    return e


def solve_ir(levels, levels32, f, x0=None, tol=1e-10, maxit=100, cycles=1, nu1=2, nu2=1, inner=None):
    """FP64 iterative refinement around FP32 V-cycles.  Returns (x, history),
    history[k] = ||f - A x_k|| in FP64.  inner: as in boxmg.solve (the norm's
    summation order; the power-of-two scale drawn from it changes no bit of
    the iterates)."""
    p64 = levels[0].planes
    fu = levels[0].fused
    nrm = bx._norm_of(inner)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    r = bx.residual(p64, x, f, fu)
    hist = [nrm(r)]
    if hist[0] == 0.0:
        return x, hist
    it = 0
    while it < maxit and hist[-1] / hist[0] > tol:
        s = scale_of(hist[-1])
        r32 = (r * (1.0 / s)).astype(F32)
        e32 = inner_cycle(levels32, r32, cycles, nu1, nu2)
        x = x + s * e32.astype(np.float64)
        r = bx.residual(p64, x, f, fu)
        hist.append(nrm(r))
        it += 1
    return x, hist


def solve_fcg_ir(levels, levels32, f, x0=None, tol=1e-10, maxit=100, cycles=1, nu1=2, nu2=1, inner=None):
    """Flexible CG in FP64 whose preconditioner is the FP32 cycle:
    z = s fl64(V32(fl32(r / s))) with s = 2^e the power of two of ||r||
    (any power of two gives the same z bit for bit)."""
    def precond(r):
        s = scale_of(bx.norm(r))
        r32 = (r * (1.0 / s)).astype(F32)
        return s * inner_cycle(levels32, r32, cycles, nu1, nu2).astype(np.float64)
    return bx._fcg(levels[0].planes, precond, f, x0, tol, maxit, levels[0].fused, inner)
