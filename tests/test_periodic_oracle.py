"""Pins of the periodic-boundary oracle (oracle/periodic.py) against what the
mathematics fixes, on the CPU:

* with no periodic axis it is the Dirichlet oracle, bit for bit;
* the wrapped operator has the closed-form Fourier eigenpairs of the periodic
  Laplacian;
* its dense form is the matrix assembled here element by element, and its
  Gauss-Seidel sweep and residual are the point-by-point ones of that matrix;
* Dendy's weights are bilinear for constant coefficients, across the seam too;
* the coarse operator is the triple product P^T A P of the dense matrices,
  restriction is P^T, coefficients constant along a periodic axis give coarse
  operators constant along it, zero row sums survive coarsening;
* V(2,1) solves reach the dense direct solution with grid-independent factors.
"""
import numpy as np
import pytest

import workloads as w
from oracle import boxmg as bx
from oracle import periodic as pr

CASES = [(True, False), (False, True), (True, True)]


def shape_of(n, px, py):
    return (n + 1 if px else n), (n + 1 if py else n)


def random_cells(nx, ny, px, py, seed, lo=0.1, hi=10.0):
    cy = ny if py else ny + 1
    cx = nx if px else nx + 1
    return lo + (hi - lo) * w.uniform01(seed, cx * cy).reshape(cy, cx)


def assemble_dense(k, nx, ny, px, py, shift=0.0):
    """A of -div(k grad u) by summing Q1 element matrices over the cells, with
    the periodic node numbering wrapped; no stencil planes involved."""
    node = lambda i, j: (j - 1) * nx + (i - 1)
    Ke = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    A = np.zeros((nx * ny, nx * ny))
    cy, cx = k.shape
    for cj in range(cy):
        for ci in range(cx):
            # corners (ci, cj), (ci+1, cj), (ci+1, cj+1), (ci, cj+1) counter-clockwise
            corners = [(ci, cj), (ci + 1, cj), (ci + 1, cj + 1), (ci, cj + 1)]
            idx = []
            for (i, j) in corners:
                if px:
                    i = (i - 1) % nx + 1
                if py:
                    j = (j - 1) % ny + 1
                idx.append(node(i, j) if 1 <= i <= nx and 1 <= j <= ny else None)
            for a in range(4):
                for b in range(4):
                    if idx[a] is not None and idx[b] is not None:
                        A[idx[a], idx[b]] += k[cj, ci] * Ke[a, b]
    A[np.diag_indices_from(A)] += shift
    return A


def interior(a):
    return a[1:-1, 1:-1].reshape(-1)


def to_grid(v, nx, ny):
    g = np.zeros((ny + 2, nx + 2))
    g[1:-1, 1:-1] = v.reshape(ny, nx)
    return g


@pytest.mark.parametrize("kind,case", [(5, "poisson"), (9, "binary"), (9, "lognormal")])
def test_no_periodic_axis_is_the_dirichlet_oracle(kind, case):
    n = 31
    if case == "poisson":
        _, planes, f = w.poisson_problem(n, 1)
    elif case == "binary":
        _, planes, f = w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3)
    else:
        _, planes, f = w.lognormal_problem(n, 2.0, 8.0, seed_k=4, seed_f=7)
    for arith in ("rounded", "fused"):
        a = bx.setup(kind, planes, arith=arith)
        b = pr.setup(kind, planes, False, False, arith=arith)
        assert len(a) == len(b)
        for la, lb in zip(a, b):
            assert np.array_equal(la.planes, lb.planes)
            if la.ci is not None:
                assert np.array_equal(la.ci, lb.ci)
        assert np.array_equal(a[-1].L, b[-1].L)
        xa, ha = bx.solve(a, f, maxit=4)
        xb, hb = pr.solve(b, f, maxit=4)
        assert np.array_equal(xa, xb) and ha == hb
        xa, ha = bx.solve_fcg(a, f, tol=0.0, maxit=4)
        xb, hb = pr.solve_fcg(b, f, tol=0.0, maxit=4)
        assert np.array_equal(xa, xb) and ha == hb


@pytest.mark.parametrize("px,py", CASES)
def test_fourier_modes_of_the_periodic_laplacian(px, py):
    n = 15
    nx, ny = shape_of(n, px, py)
    planes = np.zeros((5, ny + 2, nx + 2))
    planes[0, 1:-1, 1:-1] = 4.0
    planes[1, 1:-1, 1:-1] = -1.0
    planes[2, 1:-1, 1:-1] = -1.0
    planes = pr.prepare(5, planes, px, py)
    i = np.arange(1, nx + 1)[None, :]
    j = np.arange(1, ny + 1)[:, None]
    for (kx, ky) in [(1, 1), (3, 2), (5, 7)]:
        ux = np.cos(2 * np.pi * kx * i / nx + 0.3) if px else np.sin(np.pi * kx * i / (nx + 1))
        uy = np.cos(2 * np.pi * ky * j / ny + 0.7) if py else np.sin(np.pi * ky * j / (ny + 1))
        lx = 2 - 2 * np.cos(2 * np.pi * kx / nx) if px else 2 - 2 * np.cos(np.pi * kx / (nx + 1))
        ly = 2 - 2 * np.cos(2 * np.pi * ky / ny) if py else 2 - 2 * np.cos(np.pi * ky / (ny + 1))
        u = to_grid((ux * uy).reshape(-1), nx, ny)
        r = pr.residual(planes, u, np.zeros_like(u), px, py)
        assert np.max(np.abs(interior(r) + (lx + ly) * interior(u))) < 1e-13


@pytest.mark.parametrize("px,py", CASES)
def test_dense_form_gs_and_residual_are_the_assembled_matrix(px, py):
    n = 7
    nx, ny = shape_of(n, px, py)
    k = random_cells(nx, ny, px, py, 60 + 2 * px + py)
    shift = 0.5 if px and py else 0.0
    planes = w.fe9_periodic(k, px, py)
    planes[0, 1:-1, 1:-1] += shift
    A = assemble_dense(k, nx, ny, px, py, shift)
    P = pr.prepare(9, planes, px, py)
    assert np.allclose(pr.dense_matrix(P, px, py), A, rtol=0, atol=1e-13 * np.abs(A).max())
    x = to_grid(w.uniform_pm1(70, nx * ny), nx, ny)
    f = to_grid(w.uniform_pm1(71, nx * ny), nx, ny)
    r = pr.residual(P, x.copy(), f, px, py)
    assert np.allclose(interior(r), interior(f) - A @ interior(x), rtol=0, atol=1e-12)
    # one sweep, point by point in the colour order, from the assembled matrix
    v = interior(x).copy()
    fv = interior(f)
    for (pi, pj) in bx.COLOURS9:
        for jj in range(1, ny + 1):
            for ii in range(1, nx + 1):
                if ii % 2 == pi and jj % 2 == pj:
                    p = (jj - 1) * nx + (ii - 1)
                    v[p] = (fv[p] - (A[p] @ v - A[p, p] * v[p])) / A[p, p]
    lev = pr.Level(nx, ny, 9, P, px, py)
    xs = x.copy()
    pr.gs_sweep(9, P, lev.dinv, xs, f, px, py)
    assert np.allclose(interior(xs), v, rtol=0, atol=1e-12)
    # a sweep that forgets the wrap-around neighbours gives other values
    xd = x.copy()
    bx.gs_sweep(9, P, lev.dinv, xd, f)
    assert not np.allclose(interior(xd), v, rtol=0, atol=1e-6)


@pytest.mark.parametrize("px,py", CASES)
def test_dendy_weights_bilinear_for_constant_coefficients(px, py):
    n = 15
    nx, ny = shape_of(n, px, py)
    k = np.full((ny if py else ny + 1, nx if px else nx + 1), 3.0)
    planes = pr.prepare(9, w.fe9_periodic(k, px, py), px, py)
    ci = pr.dendy_interp(planes, px, py)
    ncx, ncy = pr.coarse_count(nx, px), pr.coarse_count(ny, py)
    kx, ky = pr.cell_count(nx, px), pr.cell_count(ny, py)
    # cells whose fine points are away from a Dirichlet side (all cells along a periodic axis)
    cx = slice(1, kx + 1) if px else slice(2, kx)
    cy = slice(1, ky + 1) if py else slice(2, ky)
    for lab in (bx.LL, bx.LR):
        assert np.allclose(ci[lab, 1:ncy + 1, cx], 0.5, rtol=0, atol=1e-15)
    for lab in (bx.LB, bx.LA):
        assert np.allclose(ci[lab, cy, 1:ncx + 1], 0.5, rtol=0, atol=1e-15)
    for lab in (bx.LSW, bx.LSE, bx.LNW, bx.LNE):
        assert np.allclose(ci[lab, cy, cx], 0.25, rtol=0, atol=1e-15)


def prolongation(ci, nx, ny, px, py):
    """Dense P: column c = the interpolation of the unit coarse vector e_c."""
    ncx, ncy = pr.coarse_count(nx, px), pr.coarse_count(ny, py)
    P = np.zeros((nx * ny, ncx * ncy))
    for c in range(ncx * ncy):
        ec = to_grid(np.eye(ncx * ncy)[c], ncx, ncy)
        x = np.zeros((ny + 2, nx + 2))
        pr.interp_correct(ci, ec, x, px, py)
        P[:, c] = interior(x)
    return P


@pytest.mark.parametrize("px,py", CASES)
def test_coarse_operator_is_the_galerkin_product(px, py):
    n = 15
    nx, ny = shape_of(n, px, py)
    k = random_cells(nx, ny, px, py, 80 + 2 * px + py, 1.0, 100.0)
    shift = 0.25 if px and py else 0.0
    planes = w.fe9_periodic(k, px, py)
    planes[0, 1:-1, 1:-1] += shift
    A = assemble_dense(k, nx, ny, px, py, shift)
    P0 = pr.prepare(9, planes, px, py)
    ci = pr.dendy_interp(P0, px, py)
    P = prolongation(ci, nx, ny, px, py)
    Ac = pr.rap(P0, ci, px, py)
    ncx, ncy = pr.coarse_count(nx, px), pr.coarse_count(ny, py)
    want = P.T @ A @ P
    got = pr.dense_matrix(Ac, px, py)
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    assert np.allclose(got, got.T, rtol=0, atol=1e-12 * np.abs(want).max())
    # the coincident weight is 1 and every fine point interpolates from its neighbours only
    assert np.count_nonzero(np.abs(P) > 0, axis=1).max() <= 4
    # restriction is P^T
    r = to_grid(w.uniform_pm1(90, nx * ny), nx, ny)
    pr.wrap(r, px, py)
    fc = pr.restrict(ci, r, px, py)
    assert np.allclose(interior(fc), P.T @ interior(r), rtol=0, atol=1e-13)
    assert fc.shape == (ncy + 2, ncx + 2)


def test_coefficients_constant_along_the_periodic_axis_stay_so():
    n = 63
    nx, ny = shape_of(n, True, False)
    rows = 0.5 + w.uniform01(95, ny + 1) * 20.0
    k = np.repeat(rows[:, None], nx, axis=1)
    levels = pr.setup(9, w.fe9_periodic(k, True, False), True, False)
    for lev in levels:
        inner = lev.planes[:, 1:-1, 1:-1]
        assert np.array_equal(inner, np.repeat(inner[:, :, :1], lev.nx, axis=2))
        if lev.ci is not None:
            kx = pr.cell_count(lev.nx, True)
            cells = lev.ci[:, 1:-1, 1:kx + 1]
            assert np.array_equal(cells, np.repeat(cells[:, :, :1], kx, axis=2))


def test_zero_row_sums_survive_coarsening_on_the_torus():
    n = 31
    nx, ny = shape_of(n, True, True)
    k = random_cells(nx, ny, True, True, 97, 1.0, 50.0)
    P = pr.prepare(9, w.fe9_periodic(k, True, True), True, True)
    for _ in range(3):
        A = pr.dense_matrix(P, True, True)
        assert np.max(np.abs(A.sum(axis=1))) < 1e-12 * np.abs(A).max()
        ci = pr.dendy_interp(P, True, True)
        # Dendy's weights are a partition of unity here: P 1 = 1
        ny_, nx_ = P.shape[-2] - 2, P.shape[-1] - 2
        ones = np.ones((pr.coarse_count(ny_, True) + 2, pr.coarse_count(nx_, True) + 2))
        x = np.zeros((ny_ + 2, nx_ + 2))
        pr.interp_correct(ci, ones, x, True, True)
        assert np.allclose(interior(x), 1.0, rtol=0, atol=1e-13)
        P = pr.rap(P, ci, True, True)


@pytest.mark.parametrize("px,py", CASES)
@pytest.mark.parametrize("arith", ["rounded", "fused"])
def test_solve_reaches_the_direct_solution(px, py, arith):
    n = 15
    shift = 0.3 if px and py else 0.0
    kind, planes, f, _, _ = w.periodic_problem(n, "x" * px + "y" * py, std=1.0, corr_len=4.0, seed_k=52,
                                               seed_f=53, shift=shift)
    nx, ny = shape_of(n, px, py)
    levels = pr.setup(kind, planes, px, py, arith=arith)
    assert [(lv.nx, lv.ny) for lv in levels] == pr.level_shapes(nx, ny, px, py)
    assert (levels[-1].nx, levels[-1].ny) == ((4 if px else 3), (4 if py else 3))
    x, hist = pr.solve(levels, f, tol=1e-12, maxit=60)
    assert hist[-1] / hist[0] <= 1e-12
    A = pr.dense_matrix(levels[0].planes, px, py)
    want = np.linalg.solve(A, interior(f))
    assert np.allclose(interior(x), want, rtol=0, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("px,py", CASES)
@pytest.mark.parametrize("arith", ["rounded", "fused"])
def test_fcg_reaches_the_direct_solution_in_fewer_steps(px, py, arith):
    """FCG(1) preconditioned by the periodic V-cycle solves to the dense
    direct solution, in fewer steps than the stationary iteration; its
    residual history is that of the true residual of its iterate."""
    n = 31
    shift = 0.3 if px and py else 0.0
    kind, planes, f, _, _ = w.periodic_problem(n, "x" * px + "y" * py, std=2.0, corr_len=4.0, seed_k=56,
                                               seed_f=57, shift=shift)
    levels = pr.setup(kind, planes, px, py, arith=arith)
    x, hist = pr.solve_fcg(levels, f, tol=1e-12, maxit=60)
    _, hs = pr.solve(levels, f, tol=1e-12, maxit=60)
    assert hist[-1] / hist[0] <= 1e-12 and len(hist) < len(hs)
    A = pr.dense_matrix(levels[0].planes, px, py)
    want = np.linalg.solve(A, interior(f))
    assert np.allclose(interior(x), want, rtol=0, atol=1e-9 * np.abs(want).max())
    r = interior(f) - A @ interior(x)
    assert abs(np.linalg.norm(r) - hist[-1]) <= 1e-6 * hist[0]


@pytest.mark.parametrize("px,py", CASES)
def test_factors_are_grid_independent(px, py):
    factors = []
    for n in (31, 63, 127):
        shift = 1e-3 if px and py else 0.0
        kind, planes, f, _, _ = w.periodic_problem(n, "x" * px + "y" * py, std=1.0, corr_len=4.0, seed_k=54,
                                                   seed_f=55, shift=shift)
        levels = pr.setup(kind, planes, px, py)
        _, hist = pr.solve(levels, f, tol=1e-30, maxit=6)
        factors.append((hist[6] / hist[2]) ** (1 / 4))
    assert max(factors) < 0.2
    assert max(factors) - min(factors) < 0.05


def test_sizes_are_checked():
    with pytest.raises(ValueError):
        pr.level_shapes(15, 15, True, False)        # a periodic axis needs 2^m points
    with pytest.raises(ValueError):
        pr.level_shapes(32, 15, True, False)        # the two axes must coarsen together
    assert pr.level_shapes(16, 15, True, False) == [(16, 15), (8, 7), (4, 3)]
