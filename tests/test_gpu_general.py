"""GPU parity of general grid sizes: an nx x ny problem of any size solved
through the C ABI (embedded by the library in the next 2^m - 1 square, with
rhs and x in the caller's (ny+2) x (nx+2) layout) against the oracle's
embedding of the same problem: iterates on the caller's grid and residual
histories within the stated tolerance (flexible CG: bit for bit against the
oracle run with the device's summation order), in every precision and
arithmetic mode."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle import boxmg as bx
from oracle import mixed as mx

from reduction_order import device_inner
from test_gpu_parity import check_fcg, check_history, dev, host

pytestmark = pytest.mark.gpu

SIZES = [(100, 37), (37, 100), (200, 129), (64, 64), (5, 9), (1, 6), (255, 31)]


def oracle_solve(kind, planes, f, precision, nbf, krylov, arith, tol=1e-10, maxit=200, device_order=False):
    pn, fn = bx.embed(planes, f)
    levels = bx.setup(kind, pn, arith=arith)
    inner = device_inner(arith == "fused") if device_order else None
    if precision == "fp64":
        run = bx.solve if krylov == "none" else bx.solve_fcg
        x, h = run(levels, fn, tol=tol, maxit=maxit, inner=inner)
    else:
        run = mx.solve_ir if krylov == "none" else mx.solve_fcg_ir
        x, h = run(levels, mx.lower(levels, nbf), fn, tol=tol, maxit=maxit, inner=inner)
    ny, nx = f.shape[0] - 2, f.shape[1] - 2
    return bx.extract(x, nx, ny), h


def caller_planes(kind, planes):
    return dev(planes[:3] if kind == 5 else planes)


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("kind", [5, 9])
@pytest.mark.parametrize("arith", ["rounded", "fused"])
def test_general_size_fp64_solve_bitwise(bmg, nx, ny, kind, arith):
    _, planes, f = w.general_size_problem(nx, ny, kind)
    xw, hw = oracle_solve(kind, planes, f, "fp64", None, "none", arith)
    h = bmg.Hierarchy(kind, caller_planes(kind, planes), arith=arith)
    assert h.n == bx.embed_size(nx, ny)
    x0 = torch.full((ny + 2, nx + 2), 7.0, dtype=torch.float64, device="cuda")
    x0[1:ny + 1, 1:nx + 1] = 0.0                            # zero guess, ghost ring holding 7
    x, it, rr, ok = h.solve(dev(f), x0, tol=1e-10, maxit=200)
    assert ok and it == len(hw) - 1
    xg = host(x)
    assert np.array_equal(xg[1:ny + 1, 1:nx + 1], xw[1:ny + 1, 1:nx + 1])
    assert np.all(xg[0] == 7.0) and np.all(xg[:, 0] == 7.0)  # the caller's ghost ring is not written
    check_history(h.history(), hw)
    h.close()


@pytest.mark.parametrize("nx,ny", [(100, 37), (200, 129)])
@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("krylov", ["none", "fcg"])
@pytest.mark.parametrize("graph", [True, False])
def test_general_size_refinement_and_fcg_bitwise(bmg, nx, ny, precision, nbf, krylov, graph):
    _, planes, f = w.general_size_problem(nx, ny, 9)
    xw, hw = oracle_solve(9, planes, f, precision, nbf, krylov, "fused")
    h = bmg.Hierarchy(9, dev(planes), precision=precision, krylov=krylov, use_graph=graph, arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok
    if krylov == "fcg":
        check_fcg(x, h.history(), (xw, hw), oracle_solve(9, planes, f, precision, nbf, krylov, "fused",
                                                         device_order=True), True)
    else:
        assert it == len(hw) - 1
        assert np.array_equal(host(x)[1:ny + 1, 1:nx + 1], xw[1:ny + 1, 1:nx + 1])
        check_history(h.history(), hw)
    h.close()


def test_general_size_fp64_fcg_and_one_pass_kernel(bmg):
    nx, ny = 300, 200
    _, planes, f = w.general_size_problem(nx, ny, 9)
    h = bmg.Hierarchy(9, dev(planes), krylov="fcg", smoother="tile0", arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok
    check_fcg(x, h.history(), oracle_solve(9, planes, f, "fp64", None, "fcg", "fused"),
              oracle_solve(9, planes, f, "fp64", None, "fcg", "fused", device_order=True), False)
    h.close()


def test_general_size_timing_profile_and_repeat_solves(bmg):
    """time_cycles and profile take the caller's layout too; a second solve
    from the returned x starts from the residual the first one ended with."""
    nx, ny = 90, 45
    _, planes, f = w.general_size_problem(nx, ny, 9)
    h = bmg.Hierarchy(9, dev(planes), arith="fused")
    rhs = dev(f)
    x = torch.zeros_like(rhs)
    ms = h.time_cycles(rhs, x, 3)
    assert ms > 0 and torch.count_nonzero(x) > 0
    rows = h.profile(rhs, torch.zeros_like(rhs), 2)
    assert rows and all(r["ms"] >= 0 for r in rows)
    x, it1, rr1, ok1 = h.solve(rhs, torch.zeros_like(rhs), tol=1e-6, maxit=100)
    h1 = h.history()
    x, it2, rr2, ok2 = h.solve(rhs, x, tol=1e-3, maxit=100)
    assert ok1 and ok2 and h.history()[0] == h1[-1]
    h.close()


def test_batched_and_rhs_batches_need_level_sizes(bmg):
    _, planes, f = w.general_size_problem(20, 20, 9)
    with pytest.raises(bmg.BmgError):
        bmg.Batch(9, [dev(planes)])
    h = bmg.Hierarchy(9, dev(planes))
    with pytest.raises(bmg.BmgError):
        bmg.Batch.from_hierarchy(h, 2)
    h.close()


@pytest.mark.parametrize("sides", ["E", "EN", "WS"])
@pytest.mark.parametrize("nx,ny,precision", [(255, 255, "fp64"), (200, 129, "fp64"), (255, 255, "fp32")])
def test_neumann_sides_bitwise(bmg, sides, nx, ny, precision):
    """Natural boundary conditions enter through the stencil (zero-k cells
    beyond the Neumann sides): the library solves them like any other stencil."""
    kind, planes, f = w.neumann_problem(nx, ny, sides)
    nbf = None if precision == "fp64" else 0
    xw, hw = oracle_solve(kind, planes, f, precision, nbf, "none", "fused")
    h = bmg.Hierarchy(kind, dev(planes), precision=precision, arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok and it == len(hw) - 1
    assert np.array_equal(host(x)[1:ny + 1, 1:nx + 1], xw[1:ny + 1, 1:nx + 1])
    check_history(h.history(), hw)
    h.close()


@pytest.mark.parametrize("smoother", ["line", "yline", "xyline"])
@pytest.mark.parametrize("nx,ny,kind", [(100, 37, 9), (37, 100, 5), (200, 129, 9)])
@pytest.mark.parametrize("precision,nbf", [("fp64", None), ("fp32", 0)])
def test_general_size_line_relaxation_bitwise(bmg, smoother, nx, ny, kind, precision, nbf):
    """Line relaxation in either direction (and alternating) on an embedded
    nx x ny problem: the identity rows outside the caller's grid decouple, so
    the embedded lines are solved as the oracle's embedding solves them."""
    _, planes, f = w.general_size_problem(nx, ny, kind)
    pn, fn = bx.embed(planes, f)
    levels = bx.setup(kind, pn, smoother=smoother)
    if precision == "fp64":
        xw, hw = bx.solve(levels, fn, tol=1e-10, maxit=100)
    else:
        xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), fn, tol=1e-10, maxit=100)
    xw = bx.extract(xw, nx, ny)
    h = bmg.Hierarchy(kind, caller_planes(kind, planes), precision=precision, smoother=smoother)
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
    assert ok and it == len(hw) - 1
    assert np.array_equal(host(x)[1:ny + 1, 1:nx + 1], xw[1:ny + 1, 1:nx + 1])
    check_history(h.history(), hw)
    h.close()
