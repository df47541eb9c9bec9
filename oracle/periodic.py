"""Periodic boundaries for the BoxMG oracle: plain numpy, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper states BoxMG on Dirichlet grids only (Sec. 2, Fig. 1); periodic
sides are a capability of the black-box method it defers to, added here as
the reading below.  Every formula is the Dirichlet oracle's (oracle/boxmg.py):
the same Dendy weights, Fig. 2 restriction, Galerkin product, Gauss-Seidel
colours and term orders, taken over a grid that wraps around.

Reading (periodic sides).
* An axis is Dirichlet (N = 2^m - 1 points, zero ghost values) or periodic
  (N = 2^m points, point N + 1 is point 1 and point 0 is point N).  Both axes
  share m, so both reach their coarsest size together: 3 points on a
  Dirichlet axis, 4 on a periodic one (coarsest = 12 or 16 unknowns).
* Coarse point c of an axis sits on fine point 2c, on a periodic axis too:
  N_c = N / 2 there, and its coarse grid is periodic with period N_c.  N is
  even, so the (i, j)-parity colours and the red-black colours stay
  consistent across the seam.
* Couplings across a periodic side are entries of A: W at i = 1 couples to
  i = N, and so on.  Couplings toward a Dirichlet ghost are dropped.
* A periodic grid is stored like a Dirichlet one, as (N_y + 2) x (N_x + 2)
  arrays, and its ghost lines hold copies of the opposite interior lines
  (wrap()): ghost column 0 = column N_x, ghost column N_x + 1 = column 1,
  then the same for rows (corners included).  With the copies current, every
  neighbour read of the Dirichlet formulas is the wrapped neighbour.  The
  oracle refreshes the copies of the iterate after every colour of a
  Gauss-Seidel sweep, of residuals and coarse corrections before they are read.
* Interpolation weights keep the Fig. 2 layout per coarse cell (ic, jc).  A
  periodic axis has N_c cells (ic = 1..N_c, the cell of fine odd point
  2ic - 1), against N_c + 1 on a Dirichlet axis, and its cell 0 / N_c + 1 are
  copies of cells N_c / 1.
* With both axes periodic, a diffusion operator annihilates constants and is
  singular; such problems need a positive term on the diagonal (the coarsest
  Cholesky reports the singular case).
"""
from __future__ import annotations

import numpy as np

from . import boxmg as bx
from .boxmg import (COLOURS5, COLOURS9, LA, LB, LL, LNE, LNW, LR, LSE, LSW, NBR, RAP_TARGETS, BLOCK, at,
                    coupling, madd)


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------

def axis_m(n: int, periodic: bool) -> int:
    """m of an axis with n points: n = 2^m (periodic) or 2^m - 1 (Dirichlet),
    m >= 2; ValueError otherwise."""
    v = n if periodic else n + 1
    if v < 4 or v & (v - 1):
        raise ValueError(f"{n} points is not {'2^m' if periodic else '2^m - 1'} with m >= 2")
    return v.bit_length() - 1


def coarse_count(n: int, periodic: bool) -> int:
    """Coarse points of an axis: N / 2 (periodic) or (N - 1) / 2."""
    return n // 2 if periodic else (n - 1) // 2


def cell_count(n: int, periodic: bool) -> int:
    """Interpolation cells of an axis (one per fine odd point): N_c or N_c + 1."""
    return (n + 1) // 2


def level_shapes(nx: int, ny: int, px: bool, py: bool, coarsest_m: int = 2) -> list[tuple[int, int]]:
    """(nx, ny) of every level down to the coarsest, both axes sharing m."""
    mx, my = axis_m(nx, px), axis_m(ny, py)
    if mx != my:
        raise ValueError(f"axes of {nx} and {ny} points do not coarsen together")
    if coarsest_m < 2 or coarsest_m > mx:
        raise ValueError("coarsest_m out of range")
    out = [(nx, ny)]
    while axis_m(out[-1][0], px) > coarsest_m:
        x, y = out[-1]
        out.append((coarse_count(x, px), coarse_count(y, py)))
    return out


def wrap(a: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """Refresh the ghost copies of a (..., N_y + 2, N_x + 2) array in place on
    its periodic axes: columns first, then rows (so corners wrap both ways).
    Dirichlet axes are left alone."""
    ny, nx = a.shape[-2] - 2, a.shape[-1] - 2
    if px:
        a[..., :, 0] = a[..., :, nx]
        a[..., :, nx + 1] = a[..., :, 1]
    if py:
        a[..., 0, :] = a[..., ny, :]
        a[..., ny + 1, :] = a[..., 1, :]
    return a


def prepare(kind: int, planes: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """The level-0 stencil: FP64 copy, SW and NW zero for a 5-point stencil,
    the ghost lines and every coupling toward a Dirichlet ghost zero, then the
    periodic ghost copies."""
    p = np.array(planes, dtype=np.float64)
    if kind == 5:
        p[3:] = 0
    elif kind != 9:
        raise ValueError("kind must be 5 or 9")
    drop_dirichlet_couplings(p, px, py)
    return wrap(p, px, py)


def drop_dirichlet_couplings(planes: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """boxmg.drop_ghost_couplings restricted to the Dirichlet axes: zero the
    ghost lines, then the couplings of the first / last interior lines toward
    them; a periodic axis keeps its wrap-around couplings."""
    ny, nx = planes.shape[-2] - 2, planes.shape[-1] - 2
    for a in planes:
        a[0, :] = 0
        a[ny + 1, :] = 0
        a[:, 0] = 0
        a[:, nx + 1] = 0
    if not px:
        planes[1][:, 1] = 0     # W  of i = 1
        planes[3][:, 1] = 0     # SW of i = 1
        planes[4][:, 1] = 0     # NW of i = 1
    if not py:
        planes[2][1, :] = 0     # S  of j = 1
        planes[3][1, :] = 0     # SW of j = 1
        planes[4][ny, :] = 0    # NW of j = ny
    return planes


# ---------------------------------------------------------------------------
# Residual, Gauss-Seidel (the Dirichlet formulas over wrapped arrays)
# ---------------------------------------------------------------------------

def apply(planes, x, px, py, fused: bool = False) -> np.ndarray:
    """y = A x (interior), the row sum in NBR order; y's ghost copies refreshed."""
    wrap(x, px, py)
    return wrap(bx.apply(planes, x, fused), px, py)


def residual(planes, x, f, px, py, fused: bool = False) -> np.ndarray:
    """r = f - A x in the order of boxmg.residual, over the wrapped grid."""
    wrap(x, px, py)
    r = np.zeros_like(x)
    bx.residual_into(planes, x, f, r, fused)
    return wrap(r, px, py)


def gs_sweep(kind, planes, dinv, x, f, px, py, fused: bool = False) -> None:
    """One Gauss-Seidel sweep in the colour order of boxmg.gs_sweep; the ghost
    copies of x are refreshed before every colour, so a colour reads the
    wrapped neighbours' current values."""
    order = [c for group in COLOURS5 for c in group] if kind == 5 else COLOURS9
    for pi, pj in order:
        wrap(x, px, py)
        bx.gs_colour(planes, dinv, x, f, pi, pj, fused)
    wrap(x, px, py)


# ---------------------------------------------------------------------------
# Dendy interpolation, restriction, interpolation + correction
# ---------------------------------------------------------------------------

def dendy_interp(planes: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """Dendy's weights (the formulas of boxmg.dendy_interp) on a grid with
    periodic axes.  Returns (8, N_cy + 2, N_cx + 2) in the Fig. 2 layout with
    the cell ghost copies refreshed."""
    ny, nx = planes.shape[-2] - 2, planes.shape[-1] - 2
    ncx, ncy = coarse_count(nx, px), coarse_count(ny, py)
    kx, ky = cell_count(nx, px), cell_count(ny, py)
    ci = np.zeros((8, ncy + 2, ncx + 2), dtype=planes.dtype)
    a = {d: coupling(planes, *d) for d in NBR}
    aO, aW, aE, aS, aN = a[(0, 0)], a[(-1, 0)], a[(1, 0)], a[(0, -1)], a[(0, 1)]
    aSW, aNE, aNW, aSE = a[(-1, -1)], a[(1, 1)], a[(-1, 1)], a[(1, -1)]

    # x-edge points i = 2ic - 1, j = 2jc
    X = (slice(1, ny, 2), slice(0, nx, 2))
    D = (aS[X] + aO[X]) + aN[X]
    ci[LL, 1:ncy + 1, 1:kx + 1] = -(((aSW[X] + aW[X]) + aNW[X]) / D)
    ci[LR, 1:ncy + 1, 1:kx + 1] = -(((aSE[X] + aE[X]) + aNE[X]) / D)
    # y-edge points i = 2ic, j = 2jc - 1
    Y = (slice(0, ny, 2), slice(1, nx, 2))
    D = (aW[Y] + aO[Y]) + aE[Y]
    ci[LB, 1:ky + 1, 1:ncx + 1] = -(((aSW[Y] + aS[Y]) + aSE[Y]) / D)
    ci[LA, 1:ky + 1, 1:ncx + 1] = -(((aNW[Y] + aN[Y]) + aNE[Y]) / D)
    wrap(ci, px, py)          # the centre formula reads the edge weights of wrapped cells

    # centre points i = 2ic - 1, j = 2jc - 1
    C = (slice(0, ny, 2), slice(0, nx, 2))
    lb_w = ci[LB, 1:ky + 1, 0:kx]
    la_w = ci[LA, 1:ky + 1, 0:kx]
    lb_e = ci[LB, 1:ky + 1, 1:kx + 1]
    la_e = ci[LA, 1:ky + 1, 1:kx + 1]
    ll_s = ci[LL, 0:ky, 1:kx + 1]
    lr_s = ci[LR, 0:ky, 1:kx + 1]
    ll_n = ci[LL, 1:ky + 1, 1:kx + 1]
    lr_n = ci[LR, 1:ky + 1, 1:kx + 1]
    o = aO[C]
    sw = -(((aSW[C] + aW[C] * lb_w) + aS[C] * ll_s) / o)
    se = -(((aSE[C] + aE[C] * lb_e) + aS[C] * lr_s) / o)
    nw = -(((aNW[C] + aW[C] * la_w) + aN[C] * ll_n) / o)
    ne = -(((aNE[C] + aE[C] * la_e) + aN[C] * lr_n) / o)
    ci[LSW, 1:ky + 1, 1:kx + 1] = sw
    ci[LSE, 1:ky + 1, 1:kx + 1] = se
    ci[LNW, 1:ky + 1, 1:kx + 1] = nw
    ci[LNE, 1:ky + 1, 1:kx + 1] = ne
    return wrap(ci, px, py)


def basis(ci: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """phi[dy+1, dx+1, jc, ic] = weight of fine point (2ic+dx, 2jc+dy) toward
    coarse point (ic, jc) (boxmg.basis over wrapped cells), ghost copies
    refreshed."""
    ncy, ncx = ci.shape[-2] - 2, ci.shape[-1] - 2
    phi = np.zeros((3, 3, ncy + 2, ncx + 2), dtype=ci.dtype)
    I = (slice(1, ncy + 1), slice(1, ncx + 1))

    def w(k, dic, djc):
        return ci[k, 1 + djc:ncy + 1 + djc, 1 + dic:ncx + 1 + dic]

    phi[1, 1][I] = 1
    phi[1, 0][I] = w(LR, 0, 0)
    phi[1, 2][I] = w(LL, 1, 0)
    phi[0, 1][I] = w(LA, 0, 0)
    phi[2, 1][I] = w(LB, 0, 1)
    phi[0, 0][I] = w(LNE, 0, 0)
    phi[0, 2][I] = w(LNW, 1, 0)
    phi[2, 0][I] = w(LSE, 0, 1)
    phi[2, 2][I] = w(LSW, 1, 1)
    return wrap(phi, px, py)


def restrict(ci: np.ndarray, r: np.ndarray, px: bool, py: bool, fused: bool = False) -> np.ndarray:
    """f_c = P^T r in the term order of the Fig. 2 loop (boxmg.restrict), r
    with current ghost copies; f_c's copies refreshed."""
    ncy, ncx = ci.shape[-2] - 2, ci.shape[-1] - 2
    fc = np.zeros((ncy + 2, ncx + 2), dtype=r.dtype)

    def q(di, dj):
        return r[2 + dj:2 * ncy + 1 + dj:2, 2 + di:2 * ncx + 1 + di:2]

    def w(k, dic, djc):
        return ci[k, 1 + djc:ncy + 1 + djc, 1 + dic:ncx + 1 + dic]

    t = w(LNE, 0, 0) * q(-1, -1)
    t = madd(t, w(LA, 0, 0), q(0, -1), fused)
    t = madd(t, w(LNW, 1, 0), q(1, -1), fused)
    t = madd(t, w(LR, 0, 0), q(-1, 0), fused)
    t = t + q(0, 0)
    t = madd(t, w(LL, 1, 0), q(1, 0), fused)
    t = madd(t, w(LSE, 0, 1), q(-1, 1), fused)
    t = madd(t, w(LB, 0, 1), q(0, 1), fused)
    t = madd(t, w(LSW, 1, 1), q(1, 1), fused)
    fc[1:ncy + 1, 1:ncx + 1] = t
    return wrap(fc, px, py)


def interp_correct(ci: np.ndarray, ec: np.ndarray, x: np.ndarray, px: bool, py: bool,
                   fused: bool = False) -> None:
    """x += P e_c in the order of boxmg.interp_correct (e_c's ghost copies are
    refreshed first); x's copies refreshed after."""
    ncy, ncx = ci.shape[-2] - 2, ci.shape[-1] - 2
    ny, nx = x.shape[-2] - 2, x.shape[-1] - 2
    ky, kx = cell_count(ny, py), cell_count(nx, px)
    wrap(ec, px, py)
    Ay, Ax = slice(1, ncy + 1), slice(1, ncx + 1)
    By, Bx = slice(1, ky + 1), slice(1, kx + 1)
    Bmy, Bmx = slice(0, ky), slice(0, kx)
    ey, ex = slice(2, 2 * ncy + 1, 2), slice(2, 2 * ncx + 1, 2)
    oy, ox = slice(1, 2 * ky, 2), slice(1, 2 * kx, 2)
    x[ey, ex] = x[ey, ex] + ec[Ay, Ax]
    t = ci[LL, Ay, Bx] * ec[Ay, Bmx]
    t = madd(t, ci[LR, Ay, Bx], ec[Ay, Bx], fused)
    x[ey, ox] = x[ey, ox] + t
    t = ci[LB, By, Ax] * ec[Bmy, Ax]
    t = madd(t, ci[LA, By, Ax], ec[By, Ax], fused)
    x[oy, ex] = x[oy, ex] + t
    t = ci[LSW, By, Bx] * ec[Bmy, Bmx]
    t = madd(t, ci[LSE, By, Bx], ec[Bmy, Bx], fused)
    t = madd(t, ci[LNW, By, Bx], ec[By, Bmx], fused)
    t = madd(t, ci[LNE, By, Bx], ec[By, Bx], fused)
    x[oy, ox] = x[oy, ox] + t
    wrap(x, px, py)


# ---------------------------------------------------------------------------
# Galerkin coarse operator, dense form, hierarchy and solve loop
# ---------------------------------------------------------------------------

def _fine_index(nc: int, u: int, n: int, periodic: bool) -> np.ndarray:
    """0-based interior index of fine point 2c + u for c = 1..nc, wrapped on
    a periodic axis."""
    f = 2 * np.arange(1, nc + 1) + u
    if periodic:
        f = (f - 1) % n + 1
    return f - 1


def rap(planes: np.ndarray, ci: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """A_c = P^T A P entry by entry in the order of boxmg.rap (p over the 3x3
    fine block of c, dy outer and dx inner; q over the row of A at p in NBR
    order; structural zeros left out), with fine and coarse indices wrapped on
    periodic axes.  Returns the five coarse planes, couplings toward Dirichlet
    ghosts zero, ghost copies refreshed."""
    ny, nx = planes.shape[-2] - 2, planes.shape[-1] - 2
    ncy, ncx = ci.shape[-2] - 2, ci.shape[-1] - 2
    phi = basis(ci, px, py)
    A = {d: coupling(planes, *d) for d in NBR}
    out = np.zeros((5, ncy + 2, ncx + 2), dtype=planes.dtype)
    for t_idx, (tx, ty) in enumerate(RAP_TARGETS):
        acc = None
        for (ux, uy) in BLOCK:
            rows = _fine_index(ncy, uy, ny, py)
            cols = _fine_index(ncx, ux, nx, px)
            inner = None
            for (vx, vy) in NBR:
                ox, oy = ux + vx - 2 * tx, uy + vy - 2 * ty
                if abs(ox) > 1 or abs(oy) > 1:
                    continue
                term = A[(vx, vy)][np.ix_(rows, cols)] * phi[oy + 1, ox + 1, 1 + ty:ncy + 1 + ty, 1 + tx:ncx + 1 + tx]
                inner = term if inner is None else inner + term
            if inner is None:
                continue
            term = phi[uy + 1, ux + 1, 1:ncy + 1, 1:ncx + 1] * inner
            acc = term if acc is None else acc + term
        out[t_idx, 1:ncy + 1, 1:ncx + 1] = acc
    drop_dirichlet_couplings(out, px, py)
    return wrap(out, px, py)


def dense_matrix(planes: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """A over the interior unknowns, lexicographic (j outer, i inner); a
    coupling across a periodic side lands on the wrapped unknown (entries
    that land on one unknown add)."""
    ny, nx = planes.shape[-2] - 2, planes.shape[-1] - 2
    A = np.zeros((nx * ny, nx * ny))
    C = {d: coupling(planes, *d) for d in NBR}
    for j in range(1, ny + 1):
        for i in range(1, nx + 1):
            p = (j - 1) * nx + (i - 1)
            for (di, dj) in NBR:
                ii, jj = i + di, j + dj
                if px:
                    ii = (ii - 1) % nx + 1
                if py:
                    jj = (jj - 1) % ny + 1
                if 1 <= ii <= nx and 1 <= jj <= ny:
                    A[p, (jj - 1) * nx + (ii - 1)] += C[(di, dj)][j - 1, i - 1]
    return A


class Level:
    def __init__(self, nx, ny, kind, planes, px, py):
        self.nx, self.ny = nx, ny
        self.kind = kind
        self.planes = planes
        self.px, self.py = px, py
        self.dinv = np.zeros_like(planes[0])
        at(self.dinv, 0, 0)[...] = 1.0 / at(planes[0], 0, 0)
        wrap(self.dinv, px, py)
        self.ci = None
        self.L = None
        self.fused = False


def setup(kind: int, planes: np.ndarray, px: bool, py: bool, coarsest_m: int = 2,
          arith: str = "rounded") -> list[Level]:
    """Hierarchy on a grid with periodic axes: Dendy weights and Galerkin
    operators level by level, the Cholesky factor of the coarsest operator
    (boxmg.cholesky; SingularError for a singular coarsest operator)."""
    if arith not in ("rounded", "fused"):
        raise ValueError("arith must be 'rounded' or 'fused'")
    planes = prepare(kind, planes, px, py)
    ny, nx = planes.shape[-2] - 2, planes.shape[-1] - 2
    shapes = level_shapes(nx, ny, px, py, coarsest_m)
    levels = []
    for li, (lx, ly) in enumerate(shapes):
        lev = Level(lx, ly, kind, planes, px, py)
        lev.fused = arith == "fused"
        if li == len(shapes) - 1:
            lev.L = bx.cholesky(dense_matrix(planes, px, py))
        else:
            lev.ci = dendy_interp(planes, px, py)
            planes = rap(planes, lev.ci, px, py)
            kind = 9
        levels.append(lev)
    return levels


def coarse_solve(lev: Level, x: np.ndarray, f: np.ndarray) -> None:
    sol = bx.chol_solve(lev.L, at(f, 0, 0).reshape(-1))
    at(x, 0, 0)[...] = sol.reshape(lev.ny, lev.nx)
    wrap(x, lev.px, lev.py)


def vcycle(levels, l, x, f, nu1=2, nu2=1) -> None:
    """V(nu1, nu2) of Fig. 1 over the periodic hierarchy."""
    lev = levels[l]
    px, py = lev.px, lev.py
    if lev.L is not None:
        coarse_solve(lev, x, f)
        return
    fu = lev.fused
    for _ in range(nu1):
        gs_sweep(lev.kind, lev.planes, lev.dinv, x, f, px, py, fu)
    r = residual(lev.planes, x, f, px, py, fu)
    fc = restrict(lev.ci, r, px, py, fu)
    xc = np.zeros_like(fc)
    vcycle(levels, l + 1, xc, fc, nu1, nu2)
    interp_correct(lev.ci, xc, x, px, py, fu)
    for _ in range(nu2):
        gs_sweep(lev.kind, lev.planes, lev.dinv, x, f, px, py, fu)


def solve_fcg(levels, f, x0=None, tol=1e-10, maxit=100, nu1=2, nu2=1, inner=None):
    """Flexible CG, FCG(1), preconditioned by one periodic V(nu1, nu2) cycle
    from a zero guess: the recurrence of boxmg.solve_fcg (the same steps,
    inner products and updates) with this module's wrap-around residual and
    operator product.  inner(a, b): the interior inner product (default the
    plain dot).  Returns (x, history)."""
    lev = levels[0]
    px, py, fu = lev.px, lev.py, lev.fused

    def precond(r):
        z = np.zeros_like(r)
        vcycle(levels, 0, z, r, nu1, nu2)
        return z

    ops = (lambda x, g: residual(lev.planes, x, g, px, py, fu), lambda p: apply(lev.planes, p, px, py, fu))
    return bx._fcg(lev.planes, precond, f, x0, tol, maxit, fu, inner, ops)


def solve(levels, f, x0=None, tol=1e-10, maxit=100, nu1=2, nu2=1):
    """V(nu1, nu2) iterations until ||r_k|| / ||r_0|| <= tol or maxit cycles
    (boxmg.solve's loop); returns (x, history)."""
    lev = levels[0]
    px, py, fu = lev.px, lev.py, lev.fused
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    wrap(x, px, py)
    hist = [bx.norm(residual(lev.planes, x, f, px, py, fu))]
    if hist[0] == 0.0:
        return x, hist
    it = 0
    while it < maxit and hist[-1] / hist[0] > tol:
        vcycle(levels, 0, x, f, nu1, nu2)
        hist.append(bx.norm(residual(lev.planes, x, f, px, py, fu)))
        it += 1
    return x, hist
