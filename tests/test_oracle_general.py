"""Pins of the oracle's general-size rule: a problem on an nx x ny grid of any
size is embedded in the smallest 2^m - 1 square with identity rows outside the
caller's points.  The embedded multigrid solution is checked against a dense
direct solve of the caller's own system, which the test assembles from the
caller's planes with the symmetric-plane rule written out here (not through
the oracle); the extra unknowns must be exactly zero, the cycle must converge
like the square case, and a 2^m - 1 square must embed to itself."""
import numpy as np
import pytest

import workloads as w
from oracle import boxmg as bx

SIZES = [(5, 9), (10, 10), (16, 7), (20, 33), (37, 12), (64, 64), (3, 1), (1, 6)]


def caller_matrix(planes):
    """Dense A of the caller's nx x ny grid: row p, column q = a(p, q), the
    couplings read from O, W, S, SW, NW and their symmetric partners, with no
    coupling to a point outside [1, nx] x [1, ny]."""
    O, W, S, SW, NW = planes
    ny, nx = O.shape[0] - 2, O.shape[1] - 2
    idx = lambda i, j: (j - 1) * nx + (i - 1)
    A = np.zeros((nx * ny, nx * ny))
    inside = lambda i, j: 1 <= i <= nx and 1 <= j <= ny
    for j in range(1, ny + 1):
        for i in range(1, nx + 1):
            p = idx(i, j)
            A[p, p] = O[j, i]
            nb = {(-1, 0): W[j, i], (1, 0): W[j, i + 1], (0, -1): S[j, i], (0, 1): S[j + 1, i],
                  (-1, -1): SW[j, i], (1, 1): SW[j + 1, i + 1], (-1, 1): NW[j, i], (1, -1): NW[j - 1, i + 1]}
            for (di, dj), a in nb.items():
                if inside(i + di, j + dj):
                    A[p, idx(i + di, j + dj)] = a
    return A


@pytest.mark.parametrize("kind", [5, 9])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_embedded_solution_solves_the_caller_system(kind, nx, ny):
    _, planes, f = w.general_size_problem(nx, ny, kind)
    pn, fn = bx.embed(planes, f)
    n = pn.shape[-1] - 2
    assert n == bx.embed_size(nx, ny) and n >= max(nx, ny, 3) and ((n + 1) & n) == 0
    x_n, h = bx.solve(bx.setup(kind, pn), fn, tol=1e-13, maxit=100)
    assert h[-1] <= 1e-13 * h[0]
    outside = np.ones((n + 2, n + 2), dtype=bool)
    outside[1:ny + 1, 1:nx + 1] = False
    assert np.all(x_n[outside] == 0.0)                     # the extra unknowns stay exactly zero
    x = bx.extract(x_n, nx, ny)
    A = caller_matrix(w.zero_ghost_couplings(planes.copy()))
    ref = np.linalg.solve(A, f[1:ny + 1, 1:nx + 1].reshape(-1)).reshape(ny, nx)
    assert np.allclose(x[1:ny + 1, 1:nx + 1], ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("kind", [5, 9])
@pytest.mark.parametrize("nx,ny", [(100, 37), (129, 40), (64, 64)])
def test_embedded_cycle_converges_like_the_square_case(kind, nx, ny):
    """V(2,1) on the embedded grid: the measured factor stays below 0.15, the
    range of the 2^m - 1 squares (Poisson 127^2: about 0.1)."""
    _, planes, f = w.general_size_problem(nx, ny, kind)
    pn, fn = bx.embed(planes, f)
    _, h = bx.solve(bx.setup(kind, pn), fn, tol=1e-10, maxit=60)
    factor = (h[-1] / h[0]) ** (1.0 / (len(h) - 1))
    assert factor < 0.15


@pytest.mark.parametrize("n", [7, 15])
def test_level_size_square_embeds_to_itself(n):
    kind, planes, f = w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3)
    pn, fn = bx.embed(planes, f)
    assert pn.shape == planes.shape
    assert np.array_equal(pn, bx.drop_ghost_couplings(planes.copy()))
    assert np.array_equal(fn, f)
    _, h1 = bx.solve(bx.setup(kind, pn), fn, tol=1e-10)
    _, h2 = bx.solve(bx.setup(kind, planes), f, tol=1e-10)
    assert h1 == h2


def test_extra_rows_are_identity_and_decoupled():
    _, planes, f = w.general_size_problem(10, 6, 9)
    pn, fn = bx.embed(planes, f)
    n = pn.shape[-1] - 2
    A = caller_matrix(pn)                                   # the whole n x n grid, read the same way
    real = np.zeros((n, n), dtype=bool)
    real[:6, :10] = True
    r = real.reshape(-1)
    assert np.all(A[np.ix_(~r, ~r)] == np.eye((~r).sum()))
    assert np.all(A[np.ix_(r, ~r)] == 0) and np.all(A[np.ix_(~r, r)] == 0)
    assert np.all(fn[1:n + 1, 1:n + 1].reshape(-1)[~r] == 0)


# ---- Neumann sides through the stencil ---------------------------------------------------

@pytest.mark.parametrize("sides", ["E", "EN", "WS"])
@pytest.mark.parametrize("nx,ny", [(31, 31), (40, 23)])
def test_neumann_sides_solve_the_caller_system(sides, nx, ny):
    """Natural boundary conditions enter through the stencil (zero-k cells
    beyond the side): the multigrid solution equals the dense solve of the
    assembled system, and the cycle keeps a square-like factor."""
    kind, planes, f = w.neumann_problem(nx, ny, sides)
    pn, fn = bx.embed(planes, f)
    x_n, h = bx.solve(bx.setup(kind, pn), fn, tol=1e-12, maxit=100)
    assert h[-1] <= 1e-12 * h[0]
    factor = (h[-1] / h[0]) ** (1.0 / (len(h) - 1))
    assert factor < 0.3                               # 0.05 - 0.22 measured
    x = bx.extract(x_n, nx, ny)
    A = caller_matrix(w.zero_ghost_couplings(planes.copy()))
    ref = np.linalg.solve(A, f[1:ny + 1, 1:nx + 1].reshape(-1)).reshape(ny, nx)
    assert np.allclose(x[1:ny + 1, 1:nx + 1], ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_neumann_rows_have_zero_row_sum_and_no_outward_coupling():
    """A Neumann node of constant k: its stencil row sums to zero (no Dirichlet
    term) and has no coupling across the side; a Dirichlet-side node keeps a
    positive row sum."""
    nx, ny = 12, 10
    k = np.ones((ny + 1, nx + 1))
    k[:, nx] = 0.0                                    # Neumann on the east side
    planes = w.fe9_from_cells(k)
    A = caller_matrix(w.zero_ghost_couplings(planes.copy()))
    rows = A.sum(axis=1).reshape(ny, nx)
    assert np.allclose(rows[1:-1, nx - 1], 0.0, atol=1e-14)     # east nodes away from the corners
    assert np.all(rows[1:-1, 0] > 0.1)                           # west (Dirichlet) nodes
    assert np.all(planes[1][:, nx + 1] == 0.0) and np.all(planes[3][:, nx + 1] == 0.0)
