"""BoxMG oracle: plain, vectorised numpy, FP64 (or FP32 when handed float32
arrays -- every operation keeps the dtype of its inputs).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Method.  BoxMG as the paper uses it (Nytko et al., Sec. 2 and Fig. 1): Gauss-
Seidel relaxation, residual, restriction, interpolation and a Cholesky coarse
solve in a V-cycle, with a setup that builds coarse operators "through local
stencil operations" and defers the formulas to Dendy's black-box multigrid.
The formulas below are that published method:

* operator-dependent (Dendy) interpolation, classic collapsed-stencil form;
* restriction R = P^T, exactly the loop of Fig. 2 (coincident weight 1);
* Galerkin coarse operator A_c = P^T A P.

Layout and conventions (shared with the CUDA path as a written convention,
never as code):

* A level with n = 2^m - 1 interior points per side is an (n+2) x (n+2) array
  indexed [j, i] with a zero Dirichlet ghost ring.  Coarse point (ic, jc) sits
  on fine point (2ic, 2jc); n_c = (n - 1) / 2.
* A stencil is five planes [O, W, S, SW, NW]; E, N, NE, SE follow by symmetry.
* Every sum over a row of A runs over the neighbours in the order
  NBR = O, W, E, S, N, SW, NE, NW, SE, left to right, one rounding per
  operation (no fused multiply-add).
* Fused arithmetic mode (setup(..., arith="fused")): the same expressions in
  the same order, but each product that is added to or subtracted from a
  running sum is one fused multiply-add, fma(a, b, s) = a b + s rounded once
  (oracle/fused.py): the row sums of residual, Gauss-Seidel and A p, the
  weighted terms of restriction and interpolation and the flexible-CG
  vector updates.  Norms and inner products are plain sums (numpy) in both
  modes: their definition has no arithmetic mode.  Products
  that stand alone (the first term of a sum, s * d) and the coincident
  restriction term keep their single rounding; setup, line relaxation and the
  coarsest solve are the same in both modes.
* Interpolation weights are eight planes of shape (n_c+2, n_c+2), indexed by
  the coarse cell (ic, jc) whose north-east corner is coarse point (ic, jc),
  with the labels of Fig. 2:
    centre fine point (2ic-1, 2jc-1): LSW, LSE, LNW, LNE -> weights toward
        coarse points (ic-1, jc-1), (ic, jc-1), (ic-1, jc), (ic, jc);
    x-edge fine point (2ic-1, 2jc):   LL, LR -> toward (ic-1, jc), (ic, jc);
    y-edge fine point (2ic, 2jc-1):   LB, LA -> toward (ic, jc-1), (ic, jc).
  Weights toward ghost coarse points come out zero because couplings to ghost
  points are zero.
"""
from __future__ import annotations

import math

import numpy as np

from .fused import fma

NBR = ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, 1), (-1, 1), (1, -1))
LSW, LSE, LNW, LNE, LL, LR, LB, LA = range(8)
# Four-colour order for 9-point stencils, as (i parity, j parity):
# (odd, odd), (even, odd), (odd, even), (even, even).
COLOURS9 = ((1, 1), (0, 1), (1, 0), (0, 0))
# Red-black for 5-point stencils: red = i + j even, then black.
COLOURS5 = (((1, 1), (0, 0)), ((0, 1), (1, 0)))


class SingularError(ArithmeticError):
    """A non-positive pivot in the coarsest Cholesky factorisation."""


# ---------------------------------------------------------------------------
# Grid helpers
# ---------------------------------------------------------------------------

def size_of(a: np.ndarray) -> int:
    return a.shape[-1] - 2


def at(a: np.ndarray, di: int, dj: int) -> np.ndarray:
    """View of a(i+di, j+dj) over all interior (i, j): shape (n, n) for a
    level array; a band of rows (a view of rows j0-1 .. j1+1 of a level
    array) gives its rows j0 .. j1."""
    return a[1 + dj:a.shape[-2] - 1 + dj, 1 + di:a.shape[-1] - 1 + di]


def coupling(planes: np.ndarray, di: int, dj: int) -> np.ndarray:
    """a(p, p + (di, dj)) over all interior p, using the symmetry of A."""
    O, W, S, SW, NW = planes
    table = {(0, 0): (O, 0, 0), (-1, 0): (W, 0, 0), (1, 0): (W, 1, 0),
             (0, -1): (S, 0, 0), (0, 1): (S, 0, 1), (-1, -1): (SW, 0, 0),
             (1, 1): (SW, 1, 1), (-1, 1): (NW, 0, 0), (1, -1): (NW, 1, -1)}
    a, oi, oj = table[(di, dj)]
    return at(a, oi, oj)


def colour(pi: int, pj: int):
    """Index of the interior points with i % 2 == pi and j % 2 == pj, in an
    (n, n) interior array."""
    return (slice(1 - pj, None, 2), slice(1 - pi, None, 2))


def drop_ghost_couplings(planes: np.ndarray) -> np.ndarray:
    """Zero the ghost ring and every coupling from an interior point to a ghost
    point (Dirichlet rows hold no such entries).  In place; planes may be
    rectangular, (ny+2) x (nx+2)."""
    ny, nx = planes.shape[-2] - 2, planes.shape[-1] - 2
    for a in planes:
        a[0, :] = 0
        a[ny + 1, :] = 0
        a[:, 0] = 0
        a[:, nx + 1] = 0
    planes[1][:, 1] = 0     # W  of i = 1
    planes[2][1, :] = 0     # S  of j = 1
    planes[3][:, 1] = 0     # SW of i = 1
    planes[3][1, :] = 0     # SW of j = 1
    planes[4][:, 1] = 0     # NW of i = 1
    planes[4][ny, :] = 0    # NW of j = ny
    return planes


# ---------------------------------------------------------------------------
# General grid sizes: embedding into the next 2^m - 1 square
# ---------------------------------------------------------------------------

def embed_size(nx: int, ny: int) -> int:
    """The smallest n = 2^m - 1 >= max(nx, ny, 3)."""
    n = 3
    while n < max(nx, ny):
        n = 2 * n + 1
    return n


def embed(planes: np.ndarray, f: np.ndarray):
    """A problem on an nx x ny interior grid of any size, as one on the n x n
    grid, n = embed_size(nx, ny) (reading; the paper states only 2^m - 1
    sizes).  The caller's points keep their indices (i, j) in [1, nx] x
    [1, ny] and their equations, with the couplings across the caller's
    Dirichlet boundary dropped; every other interior point of the n x n grid
    gets the identity row (a_O = 1, no couplings, f = 0).  The extra unknowns
    are decoupled from the caller's and are zero in the solution, so the
    caller's unknowns solve the caller's system.  planes: (5, ny+2, nx+2);
    f: (ny+2, nx+2).  Returns (planes_n, f_n), both on the (n+2)^2 grid."""
    planes = drop_ghost_couplings(np.array(planes, dtype=np.float64))
    ny, nx = planes.shape[-2] - 2, planes.shape[-1] - 2
    n = embed_size(nx, ny)
    pn = np.zeros((5, n + 2, n + 2))
    pn[:, 1:ny + 1, 1:nx + 1] = planes[:, 1:ny + 1, 1:nx + 1]
    pad = np.zeros((n + 2, n + 2), dtype=bool)
    pad[1:n + 1, 1:n + 1] = True
    pad[1:ny + 1, 1:nx + 1] = False
    pn[0][pad] = 1.0
    fn = np.zeros((n + 2, n + 2))
    fn[1:ny + 1, 1:nx + 1] = np.asarray(f, dtype=np.float64)[1:ny + 1, 1:nx + 1]
    return pn, fn


def extract(x_n: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """The caller's (ny+2) x (nx+2) grid of an embedded solution (ghost ring 0)."""
    x = np.zeros((ny + 2, nx + 2))
    x[1:ny + 1, 1:nx + 1] = x_n[1:ny + 1, 1:nx + 1]
    return x


def level_sizes(n: int, coarsest: int = 3) -> list[int]:
    """n, (n-1)/2, ... down to the coarsest size (inclusive)."""
    if n < 3 or (n + 1) & n:
        raise ValueError(f"n = {n} is not 2^m - 1 >= 3")
    if coarsest < 3 or (coarsest + 1) & coarsest:
        raise ValueError(f"coarsest = {coarsest} is not 2^m - 1 >= 3")
    out = [n]
    while out[-1] > coarsest:
        out.append((out[-1] - 1) // 2)
    return out


class RowBands:
    """Runs a function of a band of rows on every band of a level, the bands
    in a thread pool (numpy releases the interpreter lock inside its array
    loops), and waits for all of them.  A band b = slice(j0 - 1, j1 + 2) of a
    level array holds its interior rows j0 .. j1 (j0 odd, so colours keep their
    parity) and one neighbour row on each side.  Used only where the rows of
    one call are independent: one Gauss-Seidel colour, the residual.  Levels
    smaller than min_rows run as one band in the calling thread."""

    def __init__(self, threads: int, min_rows: int = 256):
        from concurrent.futures import ThreadPoolExecutor
        self.threads = max(1, int(threads))
        self.min_rows = min_rows
        self.pool = ThreadPoolExecutor(self.threads) if self.threads > 1 else None

    def slices(self, n: int):
        if self.pool is None or n < self.min_rows:
            return [slice(0, n + 2)]
        step = 2 * max(1, -(-n // (2 * self.threads)))          # even band height: every j0 odd
        return [slice(j0 - 1, min(j0 + step - 1, n) + 2) for j0 in range(1, n + 1, step)]

    def run(self, n: int, fn) -> None:
        bands = self.slices(n)
        if len(bands) == 1:
            fn(bands[0])
            return
        for fut in [self.pool.submit(fn, b) for b in bands]:
            fut.result()

    def close(self) -> None:
        if self.pool is not None:
            self.pool.shutdown()


# ---------------------------------------------------------------------------
# Operator apply and residual (A5/A6/A9 building blocks)
# ---------------------------------------------------------------------------

def madd(s, a, b, fused: bool = False):
    """s + a b: rounded product then rounded sum, or one fused multiply-add."""
    return fma(a, b, s) if fused else s + a * b


def msub(s, a, b, fused: bool = False):
    """s - a b: rounded product then rounded difference, or fma(-a, b, s)
    (negation is exact, so this is s - a b rounded once)."""
    return fma(-a, b, s) if fused else s - a * b


def apply(planes: np.ndarray, x: np.ndarray, fused: bool = False) -> np.ndarray:
    """y = A x over the interior (ghost ring of y zero); the row sum runs in
    NBR order."""
    y = np.zeros_like(x)
    acc = coupling(planes, 0, 0) * at(x, 0, 0)
    for d in NBR[1:]:
        acc = madd(acc, coupling(planes, *d), at(x, *d), fused)
    at(y, 0, 0)[...] = acc
    return y


def residual(planes: np.ndarray, x: np.ndarray, f: np.ndarray, fused: bool = False, bands=None) -> np.ndarray:
    """r = f - A x, evaluated as f - a_O x_p - a_W x_W - ... (NBR order).
    bands: a RowBands runner (the rows are independent), or None."""
    r = np.zeros_like(x)
    if bands is None:
        residual_into(planes, x, f, r, fused)
    else:
        bands.run(size_of(x), lambda b: residual_into(planes[:, b], x[b], f[b], r[b], fused))
    return r


def residual_into(planes, x, f, r, fused: bool = False) -> None:
    """The interior of r = f - A x, written into r (rows of a band or of a level)."""
    acc = at(f, 0, 0).copy()
    for d in NBR:
        acc = msub(acc, coupling(planes, *d), at(x, *d), fused)
    at(r, 0, 0)[...] = acc


def norm(r: np.ndarray) -> float:
    """Euclidean norm over the interior points (Sec. 4: the solver takes the
    l2 norm of the residual, there through cuBLAS): the square root of the sum of the
    squares, summed by numpy (pairwise).  The definition is the same in both
    arithmetic modes; any summation order gives it to within a few rounding
    errors of the exact value."""
    v = at(r, 0, 0).astype(np.float64)
    return math.sqrt(float(np.sum(v * v)))


def dot(a: np.ndarray, b: np.ndarray) -> float:
    """Interior inner product: the sum of the products, summed by numpy."""
    a = at(a, 0, 0).astype(np.float64)
    b = at(b, 0, 0).astype(np.float64)
    return float(np.sum(a * b))


# ---------------------------------------------------------------------------
# Gauss-Seidel (A5; Fig. 1 "Gauss Seidel", the highlighted smoother)
# ---------------------------------------------------------------------------

def gs_colour(planes, dinv, x, f, pi, pj, fused: bool = False) -> None:
    """Update every point of one colour: x_p = (f_p - sum_{q != p} a_pq x_q) * d_p
    with d_p = 1 / a_pp.  Points of one colour share no coupling, so they are
    updated together from the same neighbour values."""
    c = colour(pi, pj)
    s = at(f, 0, 0)[c].copy()
    for d in NBR[1:]:
        s = msub(s, coupling(planes, *d)[c], at(x, *d)[c], fused)
    at(x, 0, 0)[c] = s * at(dinv, 0, 0)[c]


def gs_sweep(kind: int, planes, dinv, x, f, fused: bool = False, bands=None) -> None:
    """One Gauss-Seidel sweep: red-black for a 5-point stencil, four colours
    (i, j parities (odd,odd), (even,odd), (odd,even), (even,even)) for a
    9-point stencil.  bands: a RowBands runner, or None; within one colour the
    points are decoupled, so bands of rows update together and give the same
    values."""
    order = [c for group in COLOURS5 for c in group] if kind == 5 else COLOURS9
    for pi, pj in order:
        if bands is None:
            gs_colour(planes, dinv, x, f, pi, pj, fused)
        else:
            bands.run(size_of(x), lambda b: gs_colour(planes[:, b], dinv[b], x[b], f[b], pi, pj, fused))


# Line relaxation (Fig. 1 "Line" relaxation; the smoother BoxMG offers for
# anisotropic operators)
def line_sweep(kind: int, planes, x, f) -> None:
    """One zebra x-line Gauss-Seidel sweep: the odd rows, then the even rows.
    Each row j is solved exactly along x with the other rows held fixed: the
    row's equations form a tridiagonal system with diagonal a_O, sub-diagonal
    a_W and super-diagonal a_E, whose right-hand side is f minus the couplings
    to rows j - 1 and j + 1 in the canonical order S, N, SW, NE, NW, SE.  The
    system is solved by the Thomas algorithm (forward elimination
    m_i = a_O - a_W c_{i-1}, c_i = a_E / m_i, d_i = (g_i - a_W d_{i-1}) / m_i,
    then x_n = d_n, x_i = d_i - c_i x_{i+1}), one rounding per operation.
    Rows of one parity share no coupling, so they are solved together."""
    del kind   # the 5-point planes SW, NW are zero: their terms subtract exact zeros
    n = size_of(x)
    for first in (1, 2):                                 # odd rows, then even rows
        rows = slice(first - 1, n, 2)                    # interior row index j - 1
        g = at(f, 0, 0)[rows].copy()
        for di, dj in NBR[3:]:                           # S, N, SW, NE, NW, SE
            g = g - coupling(planes, di, dj)[rows] * at(x, di, dj)[rows]
        aO = coupling(planes, 0, 0)[rows]
        aW = coupling(planes, -1, 0)[rows]
        aE = coupling(planes, 1, 0)[rows]
        c = np.empty_like(g)
        d = np.empty_like(g)
        c[:, 0] = aE[:, 0] / aO[:, 0]
        d[:, 0] = g[:, 0] / aO[:, 0]
        for i in range(1, n):
            m = aO[:, i] - aW[:, i] * c[:, i - 1]
            c[:, i] = aE[:, i] / m
            d[:, i] = (g[:, i] - aW[:, i] * d[:, i - 1]) / m
        xr = at(x, 0, 0)[rows]                           # a view: written in place
        xr[:, n - 1] = d[:, n - 1]
        for i in range(n - 2, -1, -1):
            xr[:, i] = d[:, i] - c[:, i] * xr[:, i + 1]


def line_sweep_y(kind: int, planes, x, f) -> None:
    """One zebra y-line Gauss-Seidel sweep: the odd columns, then the even
    columns.  Each column i is solved exactly along y with the other columns
    held fixed: the column's equations form a tridiagonal system with diagonal
    a_O, sub-diagonal a_S and super-diagonal a_N, whose right-hand side is f
    minus the couplings to columns i - 1 and i + 1 in the order W, E, SW, NE,
    SE, NW (the x-line order S, N, SW, NE, NW, SE with the two axes exchanged).
    The system is solved by the Thomas algorithm from j = 1 upward
    (m_j = a_O - a_S c_{j-1}, c_j = a_N / m_j, d_j = (g_j - a_S d_{j-1}) / m_j,
    then x_n = d_n, x_j = d_j - c_j x_{j+1}), one rounding per operation.
    Columns of one parity share no coupling, so they are solved together."""
    del kind   # the 5-point planes SW, NW are zero: their terms subtract exact zeros
    n = size_of(x)
    for first in (1, 2):                                 # odd columns, then even columns
        cols = slice(first - 1, n, 2)                    # interior column index i - 1
        g = at(f, 0, 0)[:, cols].copy()
        for di, dj in ((-1, 0), (1, 0), (-1, -1), (1, 1), (1, -1), (-1, 1)):   # W, E, SW, NE, SE, NW
            g = g - coupling(planes, di, dj)[:, cols] * at(x, di, dj)[:, cols]
        aO = coupling(planes, 0, 0)[:, cols]
        aS = coupling(planes, 0, -1)[:, cols]
        aN = coupling(planes, 0, 1)[:, cols]
        c = np.empty_like(g)
        d = np.empty_like(g)
        c[0] = aN[0] / aO[0]
        d[0] = g[0] / aO[0]
        for j in range(1, n):
            m = aO[j] - aS[j] * c[j - 1]
            c[j] = aN[j] / m
            d[j] = (g[j] - aS[j] * d[j - 1]) / m
        xc = at(x, 0, 0)[:, cols]                        # a view: written in place
        xc[n - 1] = d[n - 1]
        for j in range(n - 2, -1, -1):
            xc[j] = d[j] - c[j] * xc[j + 1]


LINE_SMOOTHERS = ("line", "yline", "xyline")


def relax(lev, x, f, bands=None) -> None:
    """One sweep of the level's smoother: point Gauss-Seidel (default), zebra
    x-line ("line") or y-line ("yline") Gauss-Seidel, or alternating lines
    ("xyline": an x-line sweep, then a y-line sweep)."""
    sm = getattr(lev, "smoother", "point")
    if sm in ("line", "xyline"):
        line_sweep(lev.kind, lev.planes, x, f)
    if sm in ("yline", "xyline"):
        line_sweep_y(lev.kind, lev.planes, x, f)
    if sm not in LINE_SMOOTHERS:
        gs_sweep(lev.kind, lev.planes, lev.dinv, x, f, getattr(lev, "fused", False), bands)


# ---------------------------------------------------------------------------
# Dendy interpolation (A2)
# ---------------------------------------------------------------------------

def dendy_interp(planes: np.ndarray) -> np.ndarray:
    """Operator-dependent interpolation weights (Dendy, classic form).

    x-edge point (between coarse W and E): collapse the stencil in y,
        D = (a_S + a_O) + a_N,
        LL = -((a_SW + a_W) + a_NW) / D,  LR = -((a_SE + a_E) + a_NE) / D.
    y-edge point (between coarse S and N): collapse in x,
        D = (a_W + a_O) + a_E,
        LB = -((a_SW + a_S) + a_SE) / D,  LA = -((a_NW + a_N) + a_NE) / D.
    centre point: the row of A at p is solved for u_p with the four edge
    neighbours already interpolated, giving for the south-west corner
        LSW = -((a_SW + a_W * LB_west) + a_S * LL_south) / a_O
    and likewise for SE, NW, NE.
    """
    n = size_of(planes)
    nc = (n - 1) // 2
    dt = planes.dtype
    ci = np.zeros((8, nc + 2, nc + 2), dtype=dt)
    a = {d: coupling(planes, *d) for d in NBR}
    aO, aW, aE, aS, aN = a[(0, 0)], a[(-1, 0)], a[(1, 0)], a[(0, -1)], a[(0, 1)]
    aSW, aNE, aNW, aSE = a[(-1, -1)], a[(1, 1)], a[(-1, 1)], a[(1, -1)]

    # x-edge points i = 2ic-1 (ic = 1..nc+1), j = 2jc (jc = 1..nc)
    X = (slice(1, n - 1, 2), slice(0, n, 2))
    D = (aS[X] + aO[X]) + aN[X]
    ci[LL, 1:nc + 1, 1:nc + 2] = -(((aSW[X] + aW[X]) + aNW[X]) / D)
    ci[LR, 1:nc + 1, 1:nc + 2] = -(((aSE[X] + aE[X]) + aNE[X]) / D)

    # y-edge points i = 2ic (ic = 1..nc), j = 2jc-1 (jc = 1..nc+1)
    Y = (slice(0, n, 2), slice(1, n - 1, 2))
    D = (aW[Y] + aO[Y]) + aE[Y]
    ci[LB, 1:nc + 2, 1:nc + 1] = -(((aSW[Y] + aS[Y]) + aSE[Y]) / D)
    ci[LA, 1:nc + 2, 1:nc + 1] = -(((aNW[Y] + aN[Y]) + aNE[Y]) / D)

    # centre points i = 2ic-1, j = 2jc-1 (ic, jc = 1..nc+1)
    C = (slice(0, n, 2), slice(0, n, 2))
    lb_w = ci[LB, 1:nc + 2, 0:nc + 1]     # LB(ic-1, jc): west neighbour
    la_w = ci[LA, 1:nc + 2, 0:nc + 1]
    lb_e = ci[LB, 1:nc + 2, 1:nc + 2]     # LB(ic, jc): east neighbour
    la_e = ci[LA, 1:nc + 2, 1:nc + 2]
    ll_s = ci[LL, 0:nc + 1, 1:nc + 2]     # LL(ic, jc-1): south neighbour
    lr_s = ci[LR, 0:nc + 1, 1:nc + 2]
    ll_n = ci[LL, 1:nc + 2, 1:nc + 2]     # LL(ic, jc): north neighbour
    lr_n = ci[LR, 1:nc + 2, 1:nc + 2]
    o = aO[C]
    sw = -(((aSW[C] + aW[C] * lb_w) + aS[C] * ll_s) / o)
    se = -(((aSE[C] + aE[C] * lb_e) + aS[C] * lr_s) / o)
    nw = -(((aNW[C] + aW[C] * la_w) + aN[C] * ll_n) / o)
    ne = -(((aNE[C] + aE[C] * la_e) + aN[C] * lr_n) / o)
    ci[LSW, 1:nc + 2, 1:nc + 2] = sw
    ci[LSE, 1:nc + 2, 1:nc + 2] = se
    ci[LNW, 1:nc + 2, 1:nc + 2] = nw
    ci[LNE, 1:nc + 2, 1:nc + 2] = ne
    return ci


def basis(ci: np.ndarray) -> np.ndarray:
    """phi[dy+1, dx+1, jc, ic] = weight of fine point (2ic+dx, 2jc+dy) toward
    coarse point (ic, jc), the 3x3 footprint of column (ic, jc) of P; zero for
    ghost coarse points."""
    nc = ci.shape[-1] - 2
    phi = np.zeros((3, 3, nc + 2, nc + 2), dtype=ci.dtype)
    I = (slice(1, nc + 1), slice(1, nc + 1))

    def w(k, dic, djc):
        return ci[k, 1 + djc:nc + 1 + djc, 1 + dic:nc + 1 + dic]

    phi[1, 1][I] = 1
    phi[1, 0][I] = w(LR, 0, 0)
    phi[1, 2][I] = w(LL, 1, 0)
    phi[0, 1][I] = w(LA, 0, 0)
    phi[2, 1][I] = w(LB, 0, 1)
    phi[0, 0][I] = w(LNE, 0, 0)
    phi[0, 2][I] = w(LNW, 1, 0)
    phi[2, 0][I] = w(LSE, 0, 1)
    phi[2, 2][I] = w(LSW, 1, 1)
    return phi


# ---------------------------------------------------------------------------
# Restriction (A6; Fig. 2) and interpolation + correction (A8)
# ---------------------------------------------------------------------------

def restrict(ci: np.ndarray, r: np.ndarray, fused: bool = False) -> np.ndarray:
    """f_c = P^T r, term by term in the order of the Fig. 2 loop:
    QC = LNE Q(i-1,j-1) + LA Q(i,j-1) + LNW' Q(i+1,j-1) + LR Q(i-1,j) + Q(i,j)
         + LL' Q(i+1,j) + LSE' Q(i-1,j+1) + LB' Q(i,j+1) + LSW' Q(i+1,j+1)
    where a primed weight is read at the neighbouring coarse cell."""
    nc = ci.shape[-1] - 2
    fc = np.zeros((nc + 2, nc + 2), dtype=r.dtype)

    def q(di, dj):
        return r[2 + dj:2 * nc + 1 + dj:2, 2 + di:2 * nc + 1 + di:2]

    def w(k, dic, djc):
        return ci[k, 1 + djc:nc + 1 + djc, 1 + dic:nc + 1 + dic]

    t = w(LNE, 0, 0) * q(-1, -1)
    t = madd(t, w(LA, 0, 0), q(0, -1), fused)
    t = madd(t, w(LNW, 1, 0), q(1, -1), fused)
    t = madd(t, w(LR, 0, 0), q(-1, 0), fused)
    t = t + q(0, 0)
    t = madd(t, w(LL, 1, 0), q(1, 0), fused)
    t = madd(t, w(LSE, 0, 1), q(-1, 1), fused)
    t = madd(t, w(LB, 0, 1), q(0, 1), fused)
    t = madd(t, w(LSW, 1, 1), q(1, 1), fused)
    fc[1:nc + 1, 1:nc + 1] = t
    return fc


def interp_correct(ci: np.ndarray, ec: np.ndarray, x: np.ndarray, fused: bool = False) -> None:
    """x += P e_c (in place).  The interpolated value is formed first, then
    added: coincident x + e; x-edge x + (LL e_W + LR e_E); y-edge
    x + (LB e_S + LA e_N); centre x + (((LSW e_SW + LSE e_SE) + LNW e_NW) + LNE e_NE)."""
    nc = ci.shape[-1] - 2
    A = slice(1, nc + 1)      # coarse 1..nc
    B = slice(1, nc + 2)      # coarse 1..nc+1
    Bm = slice(0, nc + 1)     # coarse 0..nc (the "minus one" neighbour)
    even = slice(2, 2 * nc + 1, 2)
    odd = slice(1, 2 * nc + 2, 2)
    x[even, even] = x[even, even] + ec[A, A]
    t = ci[LL, A, B] * ec[A, Bm]
    t = madd(t, ci[LR, A, B], ec[A, B], fused)
    x[even, odd] = x[even, odd] + t
    t = ci[LB, B, A] * ec[Bm, A]
    t = madd(t, ci[LA, B, A], ec[B, A], fused)
    x[odd, even] = x[odd, even] + t
    t = ci[LSW, B, B] * ec[Bm, Bm]
    t = madd(t, ci[LSE, B, B], ec[Bm, B], fused)
    t = madd(t, ci[LNW, B, B], ec[B, Bm], fused)
    t = madd(t, ci[LNE, B, B], ec[B, B], fused)
    x[odd, odd] = x[odd, odd] + t


# ---------------------------------------------------------------------------
# Galerkin coarse operator (A3)
# ---------------------------------------------------------------------------

RAP_TARGETS = ((0, 0), (-1, 0), (0, -1), (-1, -1), (-1, 1))   # O, W, S, SW, NW
BLOCK = tuple((dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1))


def rap(planes: np.ndarray, ci: np.ndarray) -> np.ndarray:
    """A_c = P^T A P, entry by entry:
        A_c(c, c') = sum_{p} P(p, c) * ( sum_{q} a(p, q) P(q, c') ),
    p over the 3x3 fine block of c (dy outer, dx inner, -1..1), q over the row
    of A at p in NBR order.  A term whose P(q, c') lies outside the footprint of
    c' is a structural zero and is left out.  Returns the five coarse planes
    with the ghost ring and ghost couplings zero."""
    n = size_of(planes)
    nc = (n - 1) // 2
    phi = basis(ci)
    A = {d: coupling(planes, *d) for d in NBR}
    out = np.zeros((5, nc + 2, nc + 2), dtype=planes.dtype)
    for t_idx, (tx, ty) in enumerate(RAP_TARGETS):
        acc = None
        for (ux, uy) in BLOCK:
            prow = slice(1 + uy, 2 * nc + uy, 2)      # interior index of j = 2jc + uy
            pcol = slice(1 + ux, 2 * nc + ux, 2)
            inner = None
            for (vx, vy) in NBR:
                ox, oy = ux + vx - 2 * tx, uy + vy - 2 * ty
                if abs(ox) > 1 or abs(oy) > 1:
                    continue
                term = A[(vx, vy)][prow, pcol] * phi[oy + 1, ox + 1, 1 + ty:nc + 1 + ty, 1 + tx:nc + 1 + tx]
                inner = term if inner is None else inner + term
            if inner is None:
                continue
            term = phi[uy + 1, ux + 1, 1:nc + 1, 1:nc + 1] * inner
            acc = term if acc is None else acc + term
        out[t_idx, 1:nc + 1, 1:nc + 1] = acc
    return drop_ghost_couplings(out)


# ---------------------------------------------------------------------------
# Dense and sparse forms (coarsest solve; also used by the pins)
# ---------------------------------------------------------------------------

def dense_matrix(planes: np.ndarray) -> np.ndarray:
    """A over the interior unknowns, lexicographic (j outer, i inner)."""
    n = size_of(planes)
    m = n * n
    A = np.zeros((m, m), dtype=np.float64)
    C = {d: coupling(planes, *d) for d in NBR}
    for j in range(1, n + 1):
        for i in range(1, n + 1):
            p = (j - 1) * n + (i - 1)
            for (di, dj) in NBR:
                ii, jj = i + di, j + dj
                if 1 <= ii <= n and 1 <= jj <= n:
                    A[p, (jj - 1) * n + (ii - 1)] = C[(di, dj)][j - 1, i - 1]
    return A


def cholesky(A: np.ndarray) -> np.ndarray:
    """Textbook right-looking Cholesky A = L L^T, FP64, in this order: pivot
    column k (sqrt, divide), then the trailing update a_ij -= l_ik l_jk for
    j = k+1.., i = j.."""
    m = A.shape[0]
    a = np.array(A, dtype=np.float64)
    L = np.zeros_like(a)
    for k in range(m):
        if not a[k, k] > 0.0:
            raise SingularError(f"pivot {k} = {a[k, k]!r}")
        lkk = math.sqrt(a[k, k])
        L[k, k] = lkk
        for i in range(k + 1, m):
            L[i, k] = a[i, k] / lkk
        for j in range(k + 1, m):
            for i in range(j, m):
                a[i, j] = a[i, j] - L[i, k] * L[j, k]
    return L


def chol_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve L L^T x = b: forward then backward substitution, inner sums in
    increasing index order, FP64."""
    m = L.shape[0]
    y = [0.0] * m
    for i in range(m):
        s = float(b[i])
        for k in range(i):
            s = s - float(L[i, k]) * y[k]
        y[i] = s / float(L[i, i])
    x = [0.0] * m
    for i in range(m - 1, -1, -1):
        s = y[i]
        for k in range(i + 1, m):
            s = s - float(L[k, i]) * x[k]
        x[i] = s / float(L[i, i])
    return np.array(x, dtype=np.float64)


# ---------------------------------------------------------------------------
# Hierarchy (A2-A4), V(2,1) (A5-A8) and the solve loop (A9)
# ---------------------------------------------------------------------------

class Level:
    def __init__(self, n, kind, planes):
        self.n = n
        self.kind = kind
        self.planes = planes
        self.dinv = np.zeros_like(planes[0])
        at(self.dinv, 0, 0)[...] = planes.dtype.type(1) / at(planes[0], 0, 0)
        self.ci = None
        self.L = None
        self.smoother = "point"
        self.fused = False


def setup(kind: int, planes: np.ndarray, coarsest: int = 3, smoother: str = "point",
          arith: str = "rounded") -> list[Level]:
    """Build the hierarchy: Dendy P and Galerkin A_c level by level, then the
    Cholesky factor of the coarsest operator.  smoother: "point" (Gauss-Seidel
    by colours), "line" (zebra x-line Gauss-Seidel), "yline" (zebra y-lines) or
    "xyline" (an x-line then a y-line sweep per sweep) on every level.  arith:
    "rounded" (one rounding per operation) or "fused" (the cycle's
    multiply-adds fused, see the module notes); the setup itself is the same."""
    if smoother not in ("point",) + LINE_SMOOTHERS:
        raise ValueError("smoother must be 'point', 'line', 'yline' or 'xyline'")
    if arith not in ("rounded", "fused"):
        raise ValueError("arith must be 'rounded' or 'fused'")
    planes = np.array(planes, dtype=np.float64)
    n = size_of(planes)
    sizes = level_sizes(n, coarsest)
    if kind == 5:
        planes[3:] = 0
    elif kind != 9:
        raise ValueError("kind must be 5 or 9")
    drop_ghost_couplings(planes)
    levels = []
    for li, nl in enumerate(sizes):
        lev = Level(nl, kind, planes)
        lev.smoother = smoother
        lev.fused = arith == "fused"
        if li == len(sizes) - 1:
            lev.L = cholesky(dense_matrix(planes))
        else:
            lev.ci = dendy_interp(planes)
            planes = rap(planes, lev.ci)
            kind = 9
        levels.append(lev)
    return levels


def coarse_solve(lev: Level, x: np.ndarray, f: np.ndarray) -> None:
    """x = A^{-1} f on the coarsest level (FP64 Cholesky solve); the result is
    rounded to the dtype of x."""
    n = lev.n
    sol = chol_solve(lev.L, at(f, 0, 0).astype(np.float64).reshape(-1))
    at(x, 0, 0)[...] = sol.reshape(n, n).astype(x.dtype)


def vcycle(levels, l, x, f, nu1=2, nu2=1, bands=None) -> None:
    """V(nu1, nu2) on level l (Fig. 1): relax, restrict the residual, recurse
    with a zero initial guess (or solve directly on the coarsest level),
    interpolate and correct, relax.  bands: a RowBands runner for the
    colour passes and residuals (same values as without), or None."""
    lev = levels[l]
    if lev.L is not None:
        coarse_solve(lev, x, f)
        return
    fu = lev.fused
    for _ in range(nu1):
        relax(lev, x, f, bands)
    r = residual(lev.planes, x, f, fu, bands)
    fc = restrict(lev.ci, r, fu)
    xc = np.zeros_like(fc)
    vcycle(levels, l + 1, xc, fc, nu1, nu2, bands)
    interp_correct(lev.ci, xc, x, fu)
    for _ in range(nu2):
        relax(lev, x, f, bands)


def solve(levels, f, x0=None, tol=1e-10, maxit=100, nu1=2, nu2=1, inner=None):
    """V(nu1, nu2) iterations until ||r_k|| / ||r_0|| <= tol or maxit cycles.
    Returns (x, history) with history = [||r_0||, ||r_1||, ...].  inner(a, b):
    the interior inner product the history's norms take (default dot); the
    norms do not feed back into the iterates."""
    lev = levels[0]
    fu = lev.fused
    nrm = _norm_of(inner)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    hist = [nrm(residual(lev.planes, x, f, fu))]
    if hist[0] == 0.0:
        return x, hist
    it = 0
    while it < maxit and hist[-1] / hist[0] > tol:
        vcycle(levels, 0, x, f, nu1, nu2)
        hist.append(nrm(residual(lev.planes, x, f, fu)))
        it += 1
    return x, hist


def _norm_of(inner):
    if inner is None:
        return norm
    return lambda r: math.sqrt(inner(r, r))


def solve_fcg(levels, f, x0=None, tol=1e-10, maxit=100, nu1=2, nu2=1, inner=None):
    """Flexible conjugate gradients (one-term recurrence, Notay's FCG(1)) with
    one V(nu1, nu2) cycle from a zero guess as the preconditioner.  Per step:
      z = V(r); p = z if first else z + beta p with beta = -(z.q)/(p.q) of the
      previous step; q = A p; alpha = (p.r)/(p.q); x += alpha p; r -= alpha q.
    The test uses the recursively updated residual.  inner(a, b): the interior
    inner product (default dot); here it feeds back into the iterates through
    alpha and beta, so another summation order of the same sum gives other
    iterates at rounding level.  Returns (x, history)."""
    return _fcg(levels[0].planes, lambda r: _precondition64(levels, r, nu1, nu2), f, x0, tol, maxit,
                levels[0].fused, inner)


def _precondition64(levels, r, nu1, nu2):
    z = np.zeros_like(r)
    vcycle(levels, 0, z, r, nu1, nu2)
    return z


def _fcg(planes, precond, f, x0, tol, maxit, fused: bool = False, inner=None, ops=None):
    """The FCG(1) recurrence of solve_fcg.  ops: the operator's (residual(x, f),
    apply(p)) pair, by default those of the Dirichlet planes (the periodic
    oracle passes its wrap-around ones)."""
    fu = fused
    ip = dot if inner is None else inner
    nrm = _norm_of(inner)
    res, app = ops if ops is not None else (lambda x_, f_: residual(planes, x_, f_, fu),
                                            lambda p_: apply(planes, p_, fu))
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    r = res(x, f)
    hist = [nrm(r)]
    if hist[0] == 0.0:
        return x, hist
    p = q = None
    pq = 0.0
    it = 0
    while it < maxit and hist[-1] / hist[0] > tol:
        z = precond(r)
        if p is None:
            p = z
        else:
            beta = -(ip(z, q) / pq)
            p = madd(z, beta, p, fu)
        q = app(p)
        pq = ip(p, q)
        alpha = ip(p, r) / pq
        x = madd(x, alpha, p, fu)
        r = msub(r, alpha, q, fu)
        hist.append(nrm(r))
        it += 1
    return x, hist
