"""Pins of the CPU oracle to facts that do not come from the oracle itself:
closed-form eigenpairs, element-by-element finite-element assembly, bilinear
and 1D flux-continuity interpolation weights, the adjoint identity R = P^T,
library sparse triple products and Cholesky factors, closed-form Galerkin
stencils, dense direct solves and the iteration-matrix spectral radius."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w
from oracle import boxmg as bx
from oracle import mixed as mx

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def interior(a):
    n = a.shape[-1] - 2
    return a[..., 1:n + 1, 1:n + 1]


def sine_mode(n, p, q):
    I = np.arange(1, n + 1)
    v = np.zeros((n + 2, n + 2))
    v[1:n + 1, 1:n + 1] = np.outer(np.sin(q * np.pi * I / (n + 1)), np.sin(p * np.pi * I / (n + 1)))
    return v


def q1_assembled_matrix(k):
    """Dense stiffness matrix of -div(k grad u), Q1 elements, zero Dirichlet
    boundary, assembled cell by cell from the textbook element matrix."""
    Ke = np.loadtxt(os.path.join(GOLDEN, "q1_element.txt")) / 6.0
    n = k.shape[0] - 1
    A = np.zeros((n * n, n * n))
    for cj in range(n + 1):
        for ci in range(n + 1):
            nodes = [(ci, cj), (ci + 1, cj), (ci + 1, cj + 1), (ci, cj + 1)]
            for a, (ia, ja) in enumerate(nodes):
                for b, (ib, jb) in enumerate(nodes):
                    if 1 <= ia <= n and 1 <= ja <= n and 1 <= ib <= n and 1 <= jb <= n:
                        A[(ja - 1) * n + ia - 1, (jb - 1) * n + ib - 1] += k[cj, ci] * Ke[a, b]
    return A


def prolongation_matrix(ci, n):
    """Dense P by interpolating every coarse unit vector."""
    nc = (n - 1) // 2
    P = np.zeros((n * n, nc * nc))
    for jc in range(1, nc + 1):
        for ic in range(1, nc + 1):
            ec = np.zeros((nc + 2, nc + 2))
            ec[jc, ic] = 1.0
            x = np.zeros((n + 2, n + 2))
            bx.interp_correct(ci, ec, x)
            P[:, (jc - 1) * nc + ic - 1] = interior(x).reshape(-1)
    return P


# --------------------------------------------------------------------------
# Inputs
# --------------------------------------------------------------------------

def test_splitmix64_published_values():
    want = [int(s, 16) for s in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")).read().split()
            if s.startswith("0x")]
    assert [int(v) for v in w.splitmix64(0, 3)] == want


def test_fe_stencil_is_element_assembly():
    n = 7
    k = np.exp(w.normal(11, (n + 1) ** 2).reshape(n + 1, n + 1))
    A = bx.dense_matrix(w.fe9_from_cells(k))
    B = q1_assembled_matrix(k)
    assert np.abs(A - B).max() <= 1e-14 * np.abs(B).max()


# --------------------------------------------------------------------------
# Operator apply (A1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p,q", [(1, 1), (2, 5), (7, 3), (15, 15)])
def test_eigenpairs_5pt(p, q):
    n = 15
    a, b = p * np.pi / (n + 1), q * np.pi / (n + 1)
    lam = 4 - 2 * np.cos(a) - 2 * np.cos(b)
    v = sine_mode(n, p, q)
    y = bx.apply(w.poisson5(n), v)
    assert np.abs(y - lam * v).max() <= 1e-13 * max(lam, 1.0)


@pytest.mark.parametrize("p,q", [(1, 1), (3, 2), (9, 14), (31, 1)])
def test_eigenpairs_fe9(p, q):
    n = 31
    a, b = p * np.pi / (n + 1), q * np.pi / (n + 1)
    lam = 8 / 3 - (2 / 3) * (np.cos(a) + np.cos(b)) - (4 / 3) * np.cos(a) * np.cos(b)
    v = sine_mode(n, p, q)
    y = bx.apply(w.fe9_from_cells(np.ones((n + 1, n + 1))), v)
    assert np.abs(y - lam * v).max() <= 1e-13 * max(lam, 1.0)


def test_apply_and_residual_match_assembled_matrix():
    n = 15
    k = w.binary_blocks(n, 4, 1.0, 1e4, 3)
    planes = w.fe9_from_cells(k)
    A = q1_assembled_matrix(k)
    x = w.rhs_uniform(n, 21)
    f = w.rhs_uniform(n, 22)
    Ax = A @ interior(x).reshape(-1)
    assert np.abs(interior(bx.apply(planes, x)).reshape(-1) - Ax).max() <= 1e-12 * np.abs(Ax).max()
    r = interior(f).reshape(-1) - Ax
    assert np.abs(interior(bx.residual(planes, x, f)).reshape(-1) - r).max() <= 1e-11 * np.abs(Ax).max()


# --------------------------------------------------------------------------
# Dendy interpolation (A2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("make", [w.poisson5, lambda n: w.fe9_from_cells(np.ones((n + 1, n + 1)))])
def test_dendy_constant_coefficients_is_bilinear(make):
    n = 31
    nc = 15
    ci = bx.dendy_interp(make(n))
    C = (slice(1, nc + 2), slice(1, nc + 2))
    # weights toward interior coarse points only (ghost-bound weights are 0)
    for k, (dic, djc) in [(bx.LNE, (0, 0)), (bx.LNW, (-1, 0)), (bx.LSE, (0, -1)), (bx.LSW, (-1, -1))]:
        wk = ci[k][C]
        for jc in range(nc + 1):
            for ic in range(nc + 1):
                tic, tjc = ic + 1 + dic, jc + 1 + djc
                expect = 0.25 if (1 <= tic <= nc and 1 <= tjc <= nc) else 0.0
                assert abs(wk[jc, ic] - expect) <= 1e-15, (k, ic, jc)
    assert np.allclose(ci[bx.LL, 1:nc + 1, 2:nc + 2], 0.5, rtol=0, atol=1e-15)
    assert np.allclose(ci[bx.LR, 1:nc + 1, 1:nc + 1], 0.5, rtol=0, atol=1e-15)
    assert np.allclose(ci[bx.LB, 2:nc + 2, 1:nc + 1], 0.5, rtol=0, atol=1e-15)
    assert np.allclose(ci[bx.LA, 1:nc + 1, 1:nc + 1], 0.5, rtol=0, atol=1e-15)


def test_dendy_layered_is_flux_continuity():
    """k = k(x): the y-collapsed x-edge row reduces to the 1D operator
    -(k_L u_W - (k_L + k_R) u_p + k_R u_E), so w_W = k_L / (k_L + k_R)."""
    n = 31
    vals = np.exp(w.normal(5, n + 1) * 3.0)
    planes = w.fe9_from_cells(w.layered_cells(n, vals))
    ci = bx.dendy_interp(planes)
    nc = 15
    for ic in range(1, nc + 2):
        i = 2 * ic - 1
        kL, kR = vals[i - 1], vals[i]
        for jc in range(1, nc + 1):
            if ic > 1:
                assert abs(ci[bx.LL, jc, ic] - kL / (kL + kR)) <= 1e-14
            if ic < nc + 1:
                assert abs(ci[bx.LR, jc, ic] - kR / (kL + kR)) <= 1e-14


def test_dendy_centre_rows_solve_the_local_equation():
    """Centre weights make (A P)(p, :) = 0 at every centre point p."""
    n = 31
    planes = w.fe9_from_cells(w.lognormal_cells(n, 2.0, 4.0, 9))
    ci = bx.dendy_interp(planes)
    P = prolongation_matrix(ci, n)
    A = bx.dense_matrix(planes)
    AP = A @ P
    centre = [(j - 1) * n + (i - 1) for j in range(1, n + 1, 2) for i in range(1, n + 1, 2)]
    assert np.abs(AP[centre]).max() <= 1e-13 * np.abs(AP).max()


def test_interpolation_preserves_constants_in_the_interior():
    n = 63
    planes = w.fe9_from_cells(w.binary_blocks(n, 8, 1.0, 1e4, 2))
    ci = bx.dendy_interp(planes)
    nc = 31
    ec = np.zeros((nc + 2, nc + 2))
    ec[1:nc + 1, 1:nc + 1] = 1.0
    x = np.zeros((n + 2, n + 2))
    bx.interp_correct(ci, ec, x)
    inner = x[3:n - 1, 3:n - 1]          # rows that are zero-sum and see only interior coarse points
    assert np.abs(inner - 1.0).max() <= 1e-13


# --------------------------------------------------------------------------
# Restriction (A6, Fig. 2) and interpolation (A8)
# --------------------------------------------------------------------------

def test_restriction_is_adjoint_of_interpolation():
    n = 63
    nc = 31
    ci = bx.dendy_interp(w.fe9_from_cells(w.lognormal_cells(n, 2.0, 8.0, 4)))
    r = w.rhs_uniform(n, 31)
    ec = w.rhs_uniform(nc, 32)
    x = np.zeros_like(r)
    bx.interp_correct(ci, ec, x)
    lhs = float(np.sum(interior(bx.restrict(ci, r)) * interior(ec)))
    rhs = float(np.sum(interior(r) * interior(x)))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_restriction_weights_coincident_point_by_one():
    n = 15
    ci = bx.dendy_interp(w.poisson5(n))
    r = np.zeros((n + 2, n + 2))
    r[8, 8] = 1.0                        # coarse point (4, 4)
    fc = bx.restrict(ci, r)
    assert fc[4, 4] == 1.0 and np.count_nonzero(fc) == 1


# --------------------------------------------------------------------------
# Galerkin RAP (A3)
# --------------------------------------------------------------------------

def sparse_A(planes):
    n = bx.size_of(planes)
    rows, cols, vals = [], [], []
    J, I = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    for d in bx.NBR:
        c = bx.coupling(planes, *d)
        ii, jj = I + d[0], J + d[1]
        m = (ii >= 1) & (ii <= n) & (jj >= 1) & (jj <= n)
        rows.append(((J - 1) * n + I - 1)[m])
        cols.append(((jj - 1) * n + ii - 1)[m])
        vals.append(c[m])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n * n, n * n))


@pytest.mark.parametrize("case", ["binary", "lognormal", "poisson"])
def test_rap_matches_sparse_triple_product(case):
    n = 63
    if case == "binary":
        planes = w.fe9_from_cells(w.binary_blocks(n, 4, 1.0, 1e4, 7))
    elif case == "lognormal":
        planes = w.fe9_from_cells(w.lognormal_cells(n, 2.0, 8.0, 8))
    else:
        planes = w.poisson5(n)
    ci = bx.dendy_interp(planes)
    coarse = bx.rap(planes, ci)
    P = sp.csr_matrix(prolongation_matrix(ci, n))
    Ac = (P.T @ sparse_A(planes) @ P).toarray()
    mine = bx.dense_matrix(coarse)
    scale = np.abs(Ac).max()
    assert np.abs(mine - Ac).max() <= 1e-13 * scale
    # nothing outside the 3x3 coarse neighbourhood
    assert np.abs(Ac[mine == 0]).max(initial=0.0) <= 1e-13 * scale


def test_rap_zero_row_sums_in_the_interior():
    n = 127
    planes = w.fe9_from_cells(w.lognormal_cells(n, 2.0, 8.0, 12))
    ci = bx.dendy_interp(planes)
    coarse = bx.rap(planes, ci)
    rs = sum(bx.coupling(coarse, *d) for d in bx.NBR)
    nc = 63
    inner = rs[2:nc - 2, 2:nc - 2]
    assert np.abs(inner).max() <= 1e-12 * np.abs(bx.coupling(coarse, 0, 0)).max()


def test_rap_poisson_closed_form():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "poisson_galerkin_stencil.txt")) if l[0] != "#"]
    want = {k: float(v) for k, v in rows if k != "plane"}
    n = 31
    coarse = bx.rap(w.poisson5(n), bx.dendy_interp(w.poisson5(n)))
    nc = 15
    for idx, name in enumerate(w.PLANES):
        vals = coarse[idx, 1:nc + 1, 1:nc + 1]
        if name == "O":
            assert np.abs(vals - want[name]).max() <= 1e-15
        else:
            # couplings toward ghost coarse points are dropped; all others take the closed form
            nz = vals != 0
            assert np.abs(vals[nz] - want[name]).max() <= 1e-15
            assert nz.sum() >= (nc - 1) ** 2


def test_rap_fe_galerkin_invariance_every_level():
    """Nested Q1 spaces: the Galerkin operator of the constant-k FE stencil is
    the same stencil (8/3, -1/3) on every level."""
    n = 63
    levels = bx.setup(9, w.fe9_from_cells(np.ones((n + 1, n + 1))))
    for lev in levels:
        m = lev.n
        O = interior(lev.planes[0])
        assert np.abs(O - 8 / 3).max() <= 1e-13
        for k in range(1, 5):
            v = interior(lev.planes[k])
            nz = v != 0
            assert np.abs(v[nz] + 1 / 3).max() <= 1e-13
            assert nz.sum() >= (m - 1) ** 2


# --------------------------------------------------------------------------
# Coarsest Cholesky (A4, A7)
# --------------------------------------------------------------------------

def test_cholesky_matches_numpy():
    levels = bx.setup(9, w.fe9_from_cells(w.lognormal_cells(15, 2.0, 4.0, 3)))
    lev = levels[-1]
    A = bx.dense_matrix(lev.planes)
    assert A.shape == (9, 9)
    L = bx.cholesky(A)
    assert np.abs(L - np.linalg.cholesky(A)).max() <= 1e-14 * np.abs(L).max()
    assert np.abs(L @ L.T - A).max() <= 1e-14 * np.abs(A).max()
    b = np.arange(1.0, 10.0)
    assert np.allclose(bx.chol_solve(L, b), np.linalg.solve(A, b), rtol=1e-13, atol=0)


def test_cholesky_rejects_indefinite():
    with pytest.raises(bx.SingularError):
        bx.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


# --------------------------------------------------------------------------
# Smoother and cycle (A5-A9)
# --------------------------------------------------------------------------

def poisson5_dense(n):
    """Dense 5-point Laplacian (4 on the diagonal, -1 to the four neighbours),
    unknown p = (j - 1) n + (i - 1), as a Kronecker sum of 1D second differences."""
    T = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return np.kron(np.eye(n), T) + np.kron(T, np.eye(n))


# Colour order of the sweeps (Fig. 1): four colours by (i mod 2, j mod 2) for
# the 9-point stencil, (odd, odd), (even, odd), (odd, even), (even, even);
# red (i + j even) then black for the 5-point one.
ORDER9 = [[(1, 1)], [(0, 1)], [(1, 0)], [(0, 0)]]
ORDER5 = [[(1, 1), (0, 0)], [(0, 1), (1, 0)]]


def pointwise_gauss_seidel(A, x, f, n, order):
    """Textbook Gauss-Seidel on the dense matrix: the points of each colour in
    turn, each x_p = (f_p - sum_{q != p} a_pq x_q) / a_pp from the latest values."""
    u, b = interior(x).reshape(-1).copy(), interior(f).reshape(-1)
    for group in order:
        for j in range(1, n + 1):
            for i in range(1, n + 1):
                if (i % 2, j % 2) in group:
                    p = (j - 1) * n + i - 1
                    u[p] = (b[p] - A[p] @ u + A[p, p] * u[p]) / A[p, p]
    return u


def smoother_case(kind, n=15):
    if kind == 5:
        return w.poisson5(n), poisson5_dense(n)
    k = w.binary_blocks(n, 4, 1.0, 1e4, 5)
    return w.fe9_from_cells(k), q1_assembled_matrix(k)


@pytest.mark.parametrize("kind", [5, 9])
def test_sweep_is_pointwise_gauss_seidel_in_the_stated_colour_order(kind):
    """One sweep equals the dense point-by-point Gauss-Seidel of the stated
    colour order (to rounding); the reversed order is far from it, so the pin
    fixes the order as well as the update."""
    n = 15
    planes, A = smoother_case(kind, n)
    lev = bx.setup(kind, planes)[0]
    x0, f = w.rhs_uniform(n, 31), w.rhs_uniform(n, 32)
    x = x0.copy()
    bx.gs_sweep(kind, lev.planes, lev.dinv, x, f)
    order = ORDER5 if kind == 5 else ORDER9
    want = pointwise_gauss_seidel(A, x0, f, n, order)
    scale = np.abs(want).max()
    assert np.abs(interior(x).reshape(-1) - want).max() <= 1e-12 * scale
    other = pointwise_gauss_seidel(A, x0, f, n, order[::-1])
    assert np.abs(other - want).max() > 1e-6 * scale


@pytest.mark.parametrize("kind", [5, 9])
def test_colour_pass_solves_its_own_equations(kind):
    """After one colour's pass the residual of the dense system vanishes (to
    rounding) on that colour's points, and no other point has moved."""
    n = 15
    planes, A = smoother_case(kind, n)
    lev = bx.setup(kind, planes)[0]
    x, f = w.rhs_uniform(n, 33), w.rhs_uniform(n, 34)
    J, I = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    for pi, pj in (ORDER5[0] + ORDER5[1] if kind == 5 else [g[0] for g in ORDER9]):
        before = x.copy()
        bx.gs_colour(lev.planes, lev.dinv, x, f, pi, pj)
        mine = ((I % 2 == pi) & (J % 2 == pj)).reshape(-1)
        u = interior(x).reshape(-1)
        r = interior(f).reshape(-1) - A @ u
        assert np.abs(r[mine]).max() <= 1e-12 * np.abs(A).max() * np.abs(u).max()
        assert np.array_equal(u[~mine], interior(before).reshape(-1)[~mine])
        assert not np.array_equal(u[mine], interior(before).reshape(-1)[mine])

@pytest.mark.parametrize("n", [3, 7, 15])
@pytest.mark.parametrize("case", ["binary", "lognormal"])
def test_solution_matches_dense_direct_solve(n, case):
    if case == "binary":
        k = w.binary_blocks(n, 2, 1.0, 1e4, 40 + n)
    else:
        k = w.lognormal_cells(n, 2.0, 2.0, 50 + n)
    planes = w.fe9_from_cells(k)
    f = w.rhs_uniform(n, 60 + n)
    levels = bx.setup(9, planes)
    x, hist = bx.solve(levels, f, tol=1e-14, maxit=200)
    u = np.linalg.solve(q1_assembled_matrix(k), interior(f).reshape(-1))
    assert np.abs(interior(x).reshape(-1) - u).max() <= 1e-10 * np.abs(u).max()


@pytest.mark.parametrize("kind", [5, 9])
def test_manufactured_eigenvector_solution(kind):
    n = 63
    p, q = 3, 2
    a, b = p * np.pi / (n + 1), q * np.pi / (n + 1)
    if kind == 5:
        planes, lam = w.poisson5(n), 4 - 2 * np.cos(a) - 2 * np.cos(b)
    else:
        planes = w.fe9_from_cells(np.ones((n + 1, n + 1)))
        lam = 8 / 3 - (2 / 3) * (np.cos(a) + np.cos(b)) - (4 / 3) * np.cos(a) * np.cos(b)
    v = sine_mode(n, p, q)
    levels = bx.setup(kind, planes)
    x, _ = bx.solve(levels, v, tol=1e-12, maxit=50)
    u = v / lam
    kappa = 8.0 / lam
    assert np.abs(x - u).max() <= kappa * 1e-12 * np.abs(u).max() * 10


def iteration_matrix(levels):
    n = levels[0].n
    m = n * n
    M = np.zeros((m, m))
    f = np.zeros((n + 2, n + 2))
    for c in range(m):
        x = np.zeros((n + 2, n + 2))
        x[1 + c // n, 1 + c % n] = 1.0
        bx.vcycle(levels, 0, x, f)
        M[:, c] = interior(x).reshape(-1)
    return M


@pytest.mark.parametrize("n", [15, 31])
def test_poisson_vcycle_spectral_radius(n):
    levels = bx.setup(5, w.poisson5(n))
    rho = max(abs(np.linalg.eigvals(iteration_matrix(levels))))
    assert rho < 0.1                      # textbook V(2,1) red-black GS, bilinear P, R = P^T
    f = w.rhs_uniform(n, 77)
    x = np.zeros_like(f)
    _, hist = bx.solve(levels, f, tol=0.0, maxit=8)
    measured = (hist[8] / hist[4]) ** 0.25
    assert abs(measured - rho) <= 0.05 * rho + 0.005


def test_high_contrast_vcycle_spectral_radius_matches_measured_factor():
    n = 31
    levels = bx.setup(9, w.fe9_from_cells(w.binary_blocks(n, 4, 1.0, 1e4, 2)))
    rho = max(abs(np.linalg.eigvals(iteration_matrix(levels))))
    assert rho < 1.0
    f = w.rhs_uniform(n, 78)
    _, hist = bx.solve(levels, f, tol=0.0, maxit=30)
    measured = (hist[30] / hist[20]) ** 0.1
    assert abs(measured - rho) <= 0.05 * rho


def test_poisson_factor_is_grid_independent():
    factors = []
    for n in (127, 255, 511):
        levels = bx.setup(5, w.poisson5(n))
        _, hist = bx.solve(levels, w.rhs_uniform(n, 1), tol=0.0, maxit=6)
        factors.append((hist[6] / hist[2]) ** 0.25)
    assert max(factors) - min(factors) <= 0.02
    assert max(factors) < 0.1


def test_golden_poisson_history():
    want = [float(l) for l in open(os.path.join(GOLDEN, "poisson127_history.txt")) if l[0] != "#"]
    kind, planes, f = w.poisson_problem(127, 1)
    _, hist = bx.solve(bx.setup(kind, planes), f, tol=1e-10, maxit=50)
    assert len(hist) == len(want)
    assert np.allclose(hist, want, rtol=1e-12, atol=0)


def test_zero_rhs_takes_no_cycle():
    levels = bx.setup(5, w.poisson5(15))
    x, hist = bx.solve(levels, np.zeros((17, 17)))
    assert hist == [0.0] and not x.any()


def test_level_sizes():
    assert bx.level_sizes(127) == [127, 63, 31, 15, 7, 3]
    assert bx.level_sizes(3) == [3]
    assert bx.level_sizes(8191)[-1] == 3 and len(bx.level_sizes(8191)) == 12
    for bad in (0, 1, 2, 4, 100, 128):
        with pytest.raises(ValueError):
            bx.level_sizes(bad)


# --------------------------------------------------------------------------
# Mixed precision (A10)
# --------------------------------------------------------------------------

def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.concatenate([w.normal(3, 50000) * 1e3, w.normal(4, 50000) * 1e-3]).astype(np.float32)
    ties = np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8)], dtype=np.float32)
    a = np.concatenate([a, ties])
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mx.bf16_round(a), want)
    assert mx.bf16_round(ties)[0] == 1.0           # tie to even (down)
    assert mx.bf16_round(ties)[1] == 1.0 + 2 ** -6  # tie to even (up)


def test_bf16_levels_keep_row_sums():
    n = 63
    levels = bx.setup(9, w.fe9_from_cells(w.binary_blocks(n, 8, 1.0, 1e4, 2)))
    l32 = mx.lower(levels, bf16_levels=2)
    p = l32[0].planes
    for k in range(1, 5):
        assert np.array_equal(mx.bf16_round(p[k]), p[k])
    rs64 = sum(bx.coupling(levels[0].planes, *d) for d in bx.NBR)
    rs32 = sum(bx.coupling(p, *d).astype(np.float64) for d in bx.NBR)
    scale = np.abs(bx.coupling(p, 0, 0)).max()
    assert np.abs(rs32 - rs64).max() <= 1e-6 * scale


@pytest.mark.parametrize("bf16", [0, 2])
def test_iterative_refinement_reaches_fp64_accuracy(bf16):
    kind, planes, f = w.binary_contrast_problem(127, 8, seed_k=2, seed_f=3)
    levels = bx.setup(kind, planes)
    x, hist = mx.solve_ir(levels, mx.lower(levels, bf16), f, tol=1e-10, maxit=200)
    assert hist[-1] <= 1e-10 * hist[0]
    assert bx.norm(bx.residual(levels[0].planes, x, f)) == hist[-1]
    _, h64 = bx.solve(levels, f, tol=1e-10, maxit=200)
    assert abs(len(hist) - len(h64)) <= 3


@pytest.mark.parametrize("case", ["binary", "lognormal", "poisson"])
def test_fp32_cycle_is_the_fp64_cycle_to_fp32_rounding(case):
    """One FP32 V(2,1) cycle from zero is the FP64 cycle to FP32 rounding
    (1e-5 relative); with BF16-stored stencils on the two finest levels it
    moves by the BF16 coefficient rounding (between 1e-5 and 1e-2), and not at
    all when every coefficient is a BF16 number (Poisson: 4 and -1)."""
    if case == "binary":
        kind, planes, f = w.binary_contrast_problem(63, 8, seed_k=2, seed_f=3)
    elif case == "lognormal":
        kind, planes, f = 9, w.fe9_from_cells(w.lognormal_cells(63, 2.0, 8.0, 4)), w.rhs_uniform(63, 5)
    else:
        kind, planes, f = w.poisson_problem(63, 1)
    levels = bx.setup(kind, planes)
    e64 = np.zeros_like(f)
    bx.vcycle(levels, 0, e64, f, 2, 1)
    e32 = mx.inner_cycle(mx.lower(levels, 0), f.astype(np.float32))
    ebf = mx.inner_cycle(mx.lower(levels, 2), f.astype(np.float32))
    rel = lambda e: np.linalg.norm(e.astype(np.float64) - e64) / np.linalg.norm(e64)
    assert e32.dtype == np.float32 and rel(e32) <= 1e-5
    if case == "poisson":
        assert np.array_equal(ebf, e32)
    else:
        assert 1e-5 < rel(ebf) <= 1e-2


def test_ir_scale_is_power_of_two():
    for rho in (1.0, 0.75, 3e-11, 123456.0):
        s = mx.scale_of(rho)
        assert math.frexp(s)[0] == 0.5 and 0.5 <= rho / s < 1.0


# --------------------------------------------------------------------------
# Reductions and flexible CG
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [3, 7, 255, 1023, 1500])
def test_norm_and_dot_are_the_sums(n):
    """The l2 norm and the inner product against math.fsum, the correctly
    rounded sum: within n^2 rounding errors of the sum of magnitudes (numpy's
    pairwise sum is far inside that), exact on integer-valued data."""
    v = w.normal(900 + n, n * n).reshape(n, n)
    u = w.normal(1900 + n, n * n).reshape(n, n)
    pad = lambda a: np.pad(a, 1)
    exact = math.fsum((v * v).reshape(-1))
    assert abs(bx.norm(pad(v)) ** 2 - exact) <= 4 * n * n * 2.3e-16 * exact
    assert abs(bx.dot(pad(v), pad(u)) - math.fsum((v * u).reshape(-1))) <= 4 * n * n * 2.3e-16 * np.abs(v * u).sum()
    ints = np.round(v * 1000)                      # integer-valued: every order is exact
    assert bx.norm(pad(ints)) == math.sqrt(math.fsum((ints * ints).reshape(-1)))
    assert bx.dot(pad(ints), pad(ints + 1)) == math.fsum((ints * (ints + 1)).reshape(-1))


def test_fcg_single_level_is_one_direct_step():
    levels = bx.setup(9, w.fe9_from_cells(w.lognormal_cells(3, 2.0, 2.0, 5)))
    f = w.rhs_uniform(3, 6)
    x, hist = bx.solve_fcg(levels, f, tol=1e-14)
    assert len(hist) == 2 and hist[1] <= 1e-14 * hist[0]


@pytest.mark.parametrize("n", [7, 15])
def test_fcg_matches_dense_direct_solve(n):
    k = w.binary_blocks(n, 2, 1.0, 1e4, 70 + n)
    levels = bx.setup(9, w.fe9_from_cells(k))
    f = w.rhs_uniform(n, 71 + n)
    x, hist = bx.solve_fcg(levels, f, tol=1e-13, maxit=100)
    u = np.linalg.solve(q1_assembled_matrix(k), interior(f).reshape(-1))
    assert np.abs(interior(x).reshape(-1) - u).max() <= 1e-9 * np.abs(u).max()


def test_fcg_beats_stagnating_vcycle_on_high_contrast():
    kind, planes, f = w.binary_contrast_problem(255, 8, 1.0, 1e6, seed_k=6, seed_f=7)
    levels = bx.setup(kind, planes)
    _, hv = bx.solve(levels, f, tol=1e-8, maxit=40)
    x, hf = bx.solve_fcg(levels, f, tol=1e-8, maxit=200)
    assert hv[-1] / hv[0] > 1e-8            # the stationary cycle has not got there in 40
    assert hf[-1] <= 1e-8 * hf[0] and len(hf) - 1 < 150
    true = bx.norm(bx.residual(levels[0].planes, x, f))
    assert true <= 1e-6 * hf[0]             # recursive and true residual agree to the FP64 floor


def test_fcg_ir_reaches_fp64_accuracy():
    kind, planes, f = w.binary_contrast_problem(127, 8, seed_k=2, seed_f=3)
    levels = bx.setup(kind, planes)
    x, hist = mx.solve_fcg_ir(levels, mx.lower(levels, 2), f, tol=1e-10, maxit=200)
    assert hist[-1] <= 1e-10 * hist[0]
    assert bx.norm(bx.residual(levels[0].planes, x, f)) <= 1e-9 * hist[0]


# --------------------------------------------------------------------------
# Line relaxation (Fig. 1 "Line"; zebra x-lines)
# --------------------------------------------------------------------------

def _row_coupled_only(n, seed):
    """Random diagonally dominant stencil with couplings along x only."""
    planes = np.zeros((5, n + 2, n + 2))
    u = w.uniform01(seed, 2 * n * n).reshape(2, n, n)
    planes[1, 1:-1, 1:-1] = -(0.5 + u[0])                 # W
    planes[0, 1:-1, 1:-1] = 3.0 + u[1]                    # O > |W| + |E|
    return w.zero_ghost_couplings(planes)


def test_line_sweep_solves_rows_without_cross_coupling_exactly():
    """With no coupling between rows A is block diagonal by rows, so one line
    sweep is a direct solve (compared with a dense LU solve)."""
    n = 31
    planes = _row_coupled_only(n, 41)
    f = w.rhs_uniform(n, 42)
    x = w.rhs_uniform(n, 43)                              # any initial guess
    bx.line_sweep(5, planes, x, f)
    A = sparse_A(planes).toarray()
    xs = np.linalg.solve(A, bx.at(f, 0, 0).reshape(-1))
    assert np.allclose(bx.at(x, 0, 0).reshape(-1), xs, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("case", ["lognormal", "binary"])
def test_line_sweep_leaves_the_last_rows_exact(case):
    """The even rows are solved last with the odd rows held at their final
    values, so after a sweep every even row's equations hold to rounding
    (residual from an independently assembled sparse A); the odd rows' do
    not (they saw the old even rows)."""
    n = 31
    kind, planes, f = (w.lognormal_problem(n, 2.0, 8.0, seed_k=4, seed_f=7) if case == "lognormal"
                       else w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3))
    planes = bx.drop_ghost_couplings(np.array(planes))
    x = w.rhs_uniform(n, 44)
    bx.line_sweep(kind, planes, x, f)
    A = sparse_A(planes)
    r = (bx.at(f, 0, 0).reshape(-1) - A @ bx.at(x, 0, 0).reshape(-1)).reshape(n, n)
    scale = np.abs(bx.at(f, 0, 0)).max() + np.abs(A).max() * np.abs(x).max()
    assert np.abs(r[1::2, :]).max() <= 1e-12 * scale      # rows j = 2, 4, ... (index j - 1 odd)
    assert np.abs(r[0::2, :]).max() > 1e-6 * scale        # odd rows moved afterwards


def test_line_relaxation_handles_strong_x_coupling():
    """-(u_xx + eps u_yy), eps = 1e-3: point Gauss-Seidel V-cycles stall, x-line
    V-cycles converge fast (measured asymptotic factors)."""
    n, eps = 63, 1e-3
    planes = w.anisotropic5(n, eps)
    f = w.rhs_uniform(n, 5)
    factors = {}
    for sm in ("point", "line"):
        levels = bx.setup(5, planes, smoother=sm)
        x, hist = bx.solve(levels, f, tol=1e-12, maxit=30)
        k = min(len(hist) - 1, 8)
        factors[sm] = (hist[k] / hist[k - 3]) ** (1 / 3)
    assert factors["point"] > 0.9 and factors["line"] < 0.1, factors


transposed = w.transposed_stencil


@pytest.mark.parametrize("case", ["lognormal", "binary"])
def test_yline_sweep_is_the_xline_sweep_of_the_transposed_problem(case):
    """A y-line sweep on A equals, bit for bit, the x-line sweep (pinned above)
    of the transposed problem, transposed back: the same operations on the
    same operands with the axes exchanged."""
    n = 31
    kind, planes, f = (w.lognormal_problem(n, 2.0, 8.0, seed_k=4, seed_f=7) if case == "lognormal"
                       else w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3))
    planes = bx.drop_ghost_couplings(np.array(planes))
    x = w.rhs_uniform(n, 44)
    xt = np.ascontiguousarray(x.T)
    bx.line_sweep_y(kind, planes, x, f)
    bx.line_sweep(kind, transposed(planes), xt, np.ascontiguousarray(f.T))
    assert np.array_equal(x, xt.T)
    # and the transposition itself: the residual of the transposed problem is the transposed
    # residual (to rounding: the residual's term order is not symmetric in x and y)
    r = bx.residual(planes, x, f)
    rt = bx.residual(transposed(planes), xt, np.ascontiguousarray(f.T))
    scale = 9 * np.abs(planes).max() * np.abs(x).max() + np.abs(f).max()
    assert np.abs(bx.at(r, 0, 0) - bx.at(rt, 0, 0).T).max() <= 1e-14 * scale
    assert np.abs(bx.at(r, 0, 0)).max() > 1e-3 * scale   # not trivially zero


def test_yline_sweep_solves_columns_without_cross_coupling_exactly():
    """With couplings along y only, A is block diagonal by columns and one
    y-line sweep is a direct solve (dense LU)."""
    n = 31
    planes = transposed(_row_coupled_only(n, 41))
    f = w.rhs_uniform(n, 42)
    x = w.rhs_uniform(n, 43)
    bx.line_sweep_y(5, planes, x, f)
    A = sparse_A(planes).toarray()
    xs = np.linalg.solve(A, bx.at(f, 0, 0).reshape(-1))
    assert np.allclose(bx.at(x, 0, 0).reshape(-1), xs, rtol=1e-12, atol=1e-13)


def test_line_directions_follow_the_anisotropy():
    """-(eps u_xx + u_yy), eps = 1e-3 (the transposed x-anisotropy): point
    Gauss-Seidel and x-lines stall, y-lines and alternating lines converge
    fast; on -(u_xx + eps u_yy) alternating lines converge fast as well."""
    n, eps = 63, 1e-3
    px = w.anisotropic5(n, eps)
    py = transposed(px)
    f = w.rhs_uniform(n, 5)
    factor = {}
    for name, planes in (("y", py), ("x", px)):
        for sm in ("point", "line", "yline", "xyline"):
            if name == "x" and sm in ("point", "line"):
                continue                                  # pinned by the x-line test above
            levels = bx.setup(5, planes, smoother=sm)
            x, hist = bx.solve(levels, f, tol=1e-12, maxit=30)
            k = min(len(hist) - 1, 8)
            factor[name, sm] = (hist[k] / hist[k - 3]) ** (1 / 3)
    assert factor["y", "point"] > 0.9 and factor["y", "line"] > 0.9, factor
    assert factor["y", "yline"] < 0.1 and factor["y", "xyline"] < 0.1, factor
    assert factor["x", "yline"] > 0.9 and factor["x", "xyline"] < 0.1, factor


@pytest.mark.parametrize("case", ["lognormal", "binary", "aniso"])
def test_transposed_stencil_is_the_permuted_operator(case):
    """workloads.transposed_stencil: the assembled matrix of the transposed
    planes is P A P^T, P the permutation (i, j) -> (j, i) of the unknowns, and
    transposing twice gives the planes back."""
    n = 15
    if case == "aniso":
        planes = w.anisotropic5(n, 1e-2)
    else:
        _, planes, _ = (w.lognormal_problem(n, 2.0, 8.0, seed_k=4, seed_f=7) if case == "lognormal"
                        else w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3))
    planes = bx.drop_ghost_couplings(np.array(planes))
    A = sparse_A(planes).toarray()
    B = sparse_A(transposed(planes)).toarray()
    idx = np.arange(n * n).reshape(n, n)        # unknown (i, j) at row j, column i
    perm = idx.T.reshape(-1)                    # (i, j) of the transposed grid is (j, i) of the original
    assert np.array_equal(B, A[np.ix_(perm, perm)])
    assert np.array_equal(transposed(transposed(planes))[:, 1:-1, 1:-1], planes[:, 1:-1, 1:-1])
