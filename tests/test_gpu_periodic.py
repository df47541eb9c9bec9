"""Periodic sides on the GPU (bmg_opts.periodic) against the periodic oracle
(oracle/periodic.py): the hierarchy bit for bit, the iterates of the V(2,1)
cycles bit for bit, the residual histories bit for bit in the device's
summation order and at the stated reading against the plain norm, and the
solve to 1e-10 confirmed by the oracle's own residual."""
import ctypes
import functools

import numpy as np
import pytest
import torch

import workloads as w
from oracle import boxmg as bx
from oracle import periodic as pr
from reduction_order import device_norm

pytestmark = pytest.mark.gpu

AXES = ["x", "y", "xy"]


def problem(n, axes, seed=52, kind=9):
    shift = 0.3 if axes == "xy" else 0.0
    if kind == 5:
        nx, ny = w.periodic_shape(n, axes)
        planes = np.zeros((5, ny + 2, nx + 2))
        planes[0, 1:-1, 1:-1] = 4.0 + shift
        planes[1, 1:-1, 1:-1] = -1.0
        planes[2, 1:-1, 1:-1] = -1.0
        return 5, planes, w.rhs_uniform(nx, seed + 1, ny), "x" in axes, "y" in axes
    return w.periodic_problem(n, axes, std=2.0, corr_len=8.0, seed_k=seed, seed_f=seed + 1, shift=shift)


def hierarchy(bmg, kind, planes, axes, **kw):
    return bmg.Hierarchy(kind, torch.from_numpy(planes).cuda(), periodic=axes, **kw)


def interior(a):
    return np.asarray(a)[..., 1:-1, 1:-1]


@pytest.mark.parametrize("axes", AXES)
@pytest.mark.parametrize("n", [15, 63, 255])
def test_hierarchy_bitwise(bmg, axes, n):
    kind, planes, f, px, py = problem(n, axes)
    levels = pr.setup(kind, planes, px, py)
    h = hierarchy(bmg, kind, planes, axes)
    assert h.num_levels == len(levels)
    for l, lev in enumerate(levels):
        assert h.level_shape(l) == (lev.nx, lev.ny)
        assert np.array_equal(interior(h.stencil(l).cpu().numpy()), interior(lev.planes))
        if lev.ci is not None:
            ci = h.interp(l).cpu().numpy()
            kx, ky = pr.cell_count(lev.nx, px), pr.cell_count(lev.ny, py)
            assert np.array_equal(ci[:, 1:ky + 1, 1:kx + 1], lev.ci[:, 1:ky + 1, 1:kx + 1])
            assert not ci[:, 0].any() and not ci[:, :, 0].any()
    h.close()


def oracle_cycles(levels, f, cycles, fused):
    """Iterates and device-order residual norms of `cycles` V(2,1) cycles."""
    lev = levels[0]
    x = np.zeros_like(f)
    r = pr.residual(lev.planes, x, f, lev.px, lev.py, fused)
    hist = [device_norm(r, fused)]
    plain = [bx.norm(r)]
    for _ in range(cycles):
        pr.vcycle(levels, 0, x, f)
        r = pr.residual(lev.planes, x, f, lev.px, lev.py, fused)
        hist.append(device_norm(r, fused))
        plain.append(bx.norm(r))
    return x, hist, plain


@pytest.mark.parametrize("axes", AXES)
@pytest.mark.parametrize("arith", ["rounded", "fused"])
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("smoother", ["auto", "rows", "tile"])
def test_cycles_bitwise(bmg, axes, arith, use_graph, smoother):
    """9-point levels swept by the two row-parity launches (rows), by the
    one-pass strip kernel (tile), or per level by the faster one (auto)."""
    n = 127
    kind, planes, f, px, py = problem(n, axes, seed=56)
    levels = pr.setup(kind, planes, px, py, arith=arith)
    x_o, hist_o, plain_o = oracle_cycles(levels, f, 5, arith == "fused")
    h = hierarchy(bmg, kind, planes, axes, arith=arith, use_graph=use_graph, smoother=smoother)
    rhs = torch.from_numpy(f).cuda()
    x, it, rr, ok = h.solve(rhs, tol=0.0, maxit=5)
    assert it == 5 and not ok
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_o))
    hist = h.history()
    assert hist == hist_o
    for g, t in zip(hist, plain_o):
        assert abs(g - t) <= 1e-12 * plain_o[0]
        if t >= 1e-3 * plain_o[0]:
            assert abs(g - t) <= 1e-12 * t
    h.close()


@pytest.mark.parametrize("axes", ["x", "y"])
def test_five_point_cycles_bitwise(bmg, axes):
    """5-point level 0 (one launch per colour, in place) over strip-swept
    9-point coarse levels."""
    kind, planes, f, px, py = problem(63, axes, kind=5)
    levels = pr.setup(kind, planes, px, py)
    x_o, hist_o, _ = oracle_cycles(levels, f, 4, False)
    h = hierarchy(bmg, kind, planes, axes)
    x, it, _, _ = h.solve(torch.from_numpy(f).cuda(), tol=0.0, maxit=4)
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_o))
    assert h.history() == hist_o
    h.close()


@pytest.mark.parametrize("axes", AXES)
def test_solve_to_tolerance(bmg, axes):
    n = 511
    kind, planes, f, px, py = problem(n, axes, seed=58)
    h = hierarchy(bmg, kind, planes, axes, arith="fused")
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), tol=1e-10, maxit=100)
    assert ok and rr <= 1e-10 and it < 60
    P = pr.prepare(kind, planes, px, py)
    xo = x.cpu().numpy()
    r = pr.residual(P, xo, f, px, py)
    assert bx.norm(r) <= 1.01e-10 * bx.norm(pr.residual(P, np.zeros_like(f), f, px, py))
    h.close()


@functools.lru_cache(maxsize=1)
def full_size_oracle():
    kind, planes, f, px, py = w.periodic_problem(4095, "x", seed_k=50, seed_f=51)
    levels = pr.setup(kind, planes, px, py, arith="fused")
    x_o = np.zeros_like(f)
    for _ in range(2):
        pr.vcycle(levels, 0, x_o, f)
    return kind, planes, f, x_o


@pytest.mark.parametrize("smoother", ["auto", "tile"])
def test_full_size_cycles_bitwise(bmg, smoother):
    """4096 x 4095, periodic in x: two cycles bitwise, in the launch
    configuration the bench times (auto) and with strips on every level."""
    kind, planes, f, x_o = full_size_oracle()
    h = hierarchy(bmg, kind, planes, "x", arith="fused", smoother=smoother)
    x, it, _, _ = h.solve(torch.from_numpy(f).cuda(), tol=0.0, maxit=2)
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_o))
    h.close()


def test_singular_torus_is_reported(bmg):
    kind, planes, f, px, py = w.periodic_problem(15, "xy", std=1.0, corr_len=4.0)
    with pytest.raises(bx.SingularError):
        pr.setup(kind, planes, px, py)
    with pytest.raises(bmg.BmgError) as e:
        hierarchy(bmg, kind, planes, "xy")
    assert e.value.code == bmg.BMG_ESINGULAR


@pytest.mark.parametrize("shape,axes", [((15, 15), "x"), ((32, 15), "x"), ((16, 16), "x"), ((16, 15), "y"),
                                        ((16, 15), "xy")])
def test_bad_periodic_sizes(bmg, shape, axes):
    nx, ny = shape
    planes = np.zeros((5, ny + 2, nx + 2))
    planes[0] = 4.0
    with pytest.raises(bmg.BmgError) as e:
        hierarchy(bmg, 9, planes, axes)
    assert e.value.code == bmg.BMG_EINVAL


@pytest.mark.parametrize("kw", [dict(precision="fp32"), dict(precision="bf16"), dict(smoother="tile1"),
                                dict(smoother="pair"), dict(smoother="line"), dict(coarsest=7)])
def test_unsupported_options(bmg, kw):
    kind, planes, f, px, py = problem(63, "x")
    with pytest.raises(bmg.BmgError) as e:
        hierarchy(bmg, kind, planes, "x", **kw)
    assert e.value.code == bmg.BMG_EINVAL


def test_square_only_calls_refuse(bmg):
    kind, planes, f, px, py = problem(63, "x")
    h = hierarchy(bmg, kind, planes, "x")
    assert bmg.lib.bmg_level_size(h._h, 0) == bmg.BMG_EINVAL
    out = ctypes.c_void_p()
    assert bmg.lib.bmg_batch_rhs(h._h, 2, None, ctypes.byref(out)) == bmg.BMG_EINVAL
    h.close()


@pytest.mark.parametrize("smoother", ["auto", "rows", "tile"])
def test_sweep_choice_is_reported(bmg, smoother):
    kind, planes, f, px, py = problem(255, "xy")
    h = hierarchy(bmg, kind, planes, "xy", smoother=smoother)
    got = [h.tuned_cluster(l) for l in range(h.num_levels)]
    assert got[-1] == 0
    want = {"rows": 1, "tile": bmg.TILE_SWEEP}.get(smoother)
    assert all(c == want if want else c in (1, bmg.TILE_SWEEP) for c in got[:-1])
    with pytest.raises(bmg.BmgError):
        h.tuned_cluster(h.num_levels)
    h.close()


@pytest.mark.parametrize("axes", AXES)
def test_smallest_grid_is_one_direct_solve(bmg, axes):
    """Periodic 4 points (Dirichlet 3) per axis: the hierarchy is its coarsest
    level alone, and one iteration solves the system to rounding."""
    kind, planes, f, px, py = problem(3, axes)
    levels = pr.setup(kind, planes, px, py)
    assert len(levels) == 1
    h = hierarchy(bmg, kind, planes, axes)
    assert h.num_levels == 1
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), tol=1e-12, maxit=5)
    assert ok and it == 1 and rr <= 1e-13
    x_o, _ = pr.solve(levels, f, tol=1e-12, maxit=5)
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_o))
    h.close()


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (0, 2), (3, 0), (2, 3)])
@pytest.mark.parametrize("smoother", ["rows", "tile"])
def test_other_sweep_counts_bitwise(bmg, nu1, nu2, smoother):
    """Odd and even sweep counts: with strips the cycle alternates between two
    iterates, and the interpolation writes the one from which the post-sweeps
    end in x."""
    kind, planes, f, px, py = problem(63, "xy", seed=60)
    levels = pr.setup(kind, planes, px, py, arith="fused")
    x_o = np.zeros_like(f)
    for _ in range(3):
        pr.vcycle(levels, 0, x_o, f, nu1, nu2)
    h = hierarchy(bmg, kind, planes, "xy", arith="fused", nu1=nu1, nu2=nu2, smoother=smoother)
    x, it, _, _ = h.solve(torch.from_numpy(f).cuda(), tol=0.0, maxit=3)
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_o))
    h.close()


def test_zero_rhs_maxit_zero_and_nan(bmg):
    kind, planes, f, px, py = problem(63, "x")
    h = hierarchy(bmg, kind, planes, "x")
    x, it, rr, ok = h.solve(torch.zeros_like(torch.from_numpy(f)).cuda())
    assert ok and it == 0 and not x.any()
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), maxit=0)
    assert not ok and it == 0 and not x.any()
    g = f.copy()
    g[5, 7] = np.nan
    with pytest.raises(bmg.BmgError) as e:
        h.solve(torch.from_numpy(g).cuda())
    assert e.value.code == -5
    h.close()


@pytest.mark.parametrize("axes", AXES)
@pytest.mark.parametrize("arith", ["rounded", "fused"])
@pytest.mark.parametrize("smoother", ["auto", "rows"])
def test_fcg_matches_oracle(bmg, axes, arith, smoother):
    """FCG(1) with the periodic V(2,1) preconditioner: iterates and history
    bit for bit against the oracle's FCG run in the device's inner-product
    order, iteration counts equal to the plain-sum oracle's."""
    from reduction_order import device_inner
    kind, planes, f, px, py = problem(127, axes, seed=62)
    levels = pr.setup(kind, planes, px, py, arith=arith)
    x_d, h_d = pr.solve_fcg(levels, f, tol=1e-10, maxit=60, inner=device_inner(arith == "fused"))
    x_p, h_p = pr.solve_fcg(levels, f, tol=1e-10, maxit=60)
    h = hierarchy(bmg, kind, planes, axes, arith=arith, krylov="fcg", smoother=smoother)
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), tol=1e-10, maxit=60)
    assert ok and it == len(h_d) - 1
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_d))
    hist = h.history()
    assert hist == h_d
    assert abs(len(h_p) - len(h_d)) <= 1
    h.close()


def test_fcg_needs_fewer_steps_and_solves(bmg):
    """At 511 x 512 (periodic in y) FCG reaches 1e-10 in fewer steps than the
    stationary cycle, and the oracle's own residual of the returned x confirms it."""
    kind, planes, f, px, py = w.periodic_problem(511, "y", std=2.0, corr_len=8.0, seed_k=64, seed_f=65)
    h = hierarchy(bmg, kind, planes, "y", arith="fused", krylov="fcg")
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), tol=1e-10, maxit=100)
    h.close()
    s = hierarchy(bmg, kind, planes, "y", arith="fused")
    _, its, _, oks = s.solve(torch.from_numpy(f).cuda(), tol=1e-10, maxit=100)
    s.close()
    assert ok and oks and it < its
    P = pr.prepare(kind, planes, px, py)
    r = pr.residual(P, x.cpu().numpy(), f, px, py)
    assert bx.norm(r) <= 2e-10 * bx.norm(pr.residual(P, np.zeros_like(f), f, px, py))


@pytest.mark.parametrize("axes", AXES)
def test_fcg_on_the_smallest_grid_is_one_direct_solve(bmg, axes):
    """A one-level periodic hierarchy: the preconditioner is the coarsest
    solve itself, so one FCG step reaches the solution to rounding, bit for
    bit the oracle's step in the device's inner-product order."""
    from reduction_order import device_inner
    kind, planes, f, px, py = problem(3, axes)
    levels = pr.setup(kind, planes, px, py)
    assert len(levels) == 1
    x_d, h_d = pr.solve_fcg(levels, f, tol=1e-12, maxit=5, inner=device_inner(False))
    h = hierarchy(bmg, kind, planes, axes, krylov="fcg")
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), tol=1e-12, maxit=5)
    assert ok and it == 1 == len(h_d) - 1 and rr <= 1e-13
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_d))
    assert h.history() == h_d
    h.close()


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (2, 2)])
def test_fcg_other_sweep_counts_bitwise(bmg, nu1, nu2):
    """FCG around periodic cycles of other sweep counts (odd and even numbers of
    post-sweeps move the strip levels' iterate differently)."""
    from reduction_order import device_inner
    kind, planes, f, px, py = problem(63, "xy", seed=66)
    levels = pr.setup(kind, planes, px, py, arith="fused")
    x_d, h_d = pr.solve_fcg(levels, f, tol=1e-10, maxit=40, nu1=nu1, nu2=nu2, inner=device_inner(True))
    h = hierarchy(bmg, kind, planes, "xy", arith="fused", krylov="fcg", nu1=nu1, nu2=nu2, smoother="tile")
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), tol=1e-10, maxit=40)
    assert ok and it == len(h_d) - 1
    assert np.array_equal(interior(x.cpu().numpy()), interior(x_d))
    assert h.history() == h_d
    h.close()


def test_fcg_zero_rhs_maxit_zero_and_nan(bmg):
    kind, planes, f, px, py = problem(63, "x")
    h = hierarchy(bmg, kind, planes, "x", krylov="fcg")
    x, it, rr, ok = h.solve(torch.zeros_like(torch.from_numpy(f)).cuda())
    assert ok and it == 0 and not x.any()
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), maxit=0)
    assert not ok and it == 0 and not x.any()
    g = f.copy()
    g[5, 7] = np.nan
    with pytest.raises(bmg.BmgError) as e:
        h.solve(torch.from_numpy(g).cuda())
    assert e.value.code == -5
    x, it, rr, ok = h.solve(torch.from_numpy(f).cuda(), tol=1e-10, maxit=60)   # still usable
    assert ok
    h.close()
