"""GPU parity of the fused-arithmetic mode (arith="fused", BMG_ARITH_FUSED)
against the oracle's fused mode: every multiply-add of the cycle is one fused
multiply-add on both sides (CUDA's __fma_rn / __fmaf_rn, the C library's
fma / fmaf in the oracle), the expressions and their order are otherwise those
of the rounded mode, so iterates agree bit for bit again and histories to the
stated tolerance (flexible CG: bit for bit against the oracle run with the
device's summation order).  The
fused histories are also held to the rounded ones by the stated tolerance
(1e-12 of ||r_0|| per entry, the same iteration counts)."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle import boxmg as bx
from oracle import mixed as mx

from reduction_order import device_inner
from test_gpu_parity import batch_problems, check_fcg, check_history, dev, host, problem

pytestmark = pytest.mark.gpu


def oracle_solve(kind, planes, f, precision, nbf, krylov="none", arith="fused", smoother="point", tol=1e-10,
                 maxit=200, device_order=False):
    levels = bx.setup(kind, planes, smoother=smoother, arith=arith)
    inner = device_inner(arith == "fused") if device_order else None
    if precision == "fp64":
        run = bx.solve if krylov == "none" else bx.solve_fcg
        return run(levels, f, tol=tol, maxit=maxit, inner=inner)
    run = mx.solve_ir if krylov == "none" else mx.solve_fcg_ir
    return run(levels, mx.lower(levels, nbf), f, tol=tol, maxit=maxit, inner=inner)


def gpu_planes(kind, planes):
    return dev(planes[:3] if kind == 5 else planes)


@pytest.mark.parametrize("case,n", [("poisson", 127), ("binary", 255), ("lognormal", 255), ("binary", 7),
                                    ("poisson", 3)])
@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("krylov", ["none", "fcg"])
def test_fused_fp64_solve_bitwise(bmg, case, n, graph, krylov):
    kind, planes, f = problem(case, n)
    xw, hw = oracle_solve(kind, planes, f, "fp64", None, krylov)
    h = bmg.Hierarchy(kind, gpu_planes(kind, planes), use_graph=graph, krylov=krylov, arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok
    if krylov == "fcg":
        check_fcg(x, h.history(), (xw, hw), oracle_solve(kind, planes, f, "fp64", None, krylov, device_order=True),
                  False)
    else:
        assert it == len(hw) - 1
        assert np.array_equal(host(x), xw)
        check_history(h.history(), hw)
        assert h.history() == oracle_solve(kind, planes, f, "fp64", None, device_order=True)[1]
    h.close()


@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("case,n", [("binary", 255), ("lognormal", 255), ("poisson", 127)])
@pytest.mark.parametrize("krylov", ["none", "fcg"])
def test_fused_refinement_solve_bitwise(bmg, precision, nbf, case, n, krylov):
    kind, planes, f = problem(case, n)
    xw, hw = oracle_solve(kind, planes, f, precision, nbf, krylov)
    h = bmg.Hierarchy(kind, gpu_planes(kind, planes), precision=precision, krylov=krylov, arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok
    if krylov == "fcg":
        check_fcg(x, h.history(), (xw, hw), oracle_solve(kind, planes, f, precision, nbf, krylov, device_order=True),
                  True)
    else:
        assert it == len(hw) - 1
        assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
        check_history(h.history(), hw)
    levels = bx.setup(kind, planes)
    assert bx.norm(bx.residual(levels[0].planes, host(x), f)) <= 1e-10 * hw[0]


@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("smoother", ["rows", "tile0", "tile1", "tile2", "tile3", "tile4", "tile5", "pair0", "pair1",
                                      "pair2", "pair3"])
def test_fused_one_pass_kernels_bitwise(bmg, precision, nbf, smoother):
    """The one-pass and two-sweep FP32 kernels, forced on every level, give the
    oracle's fused cycle bit for bit (511^2: several strips and a ragged edge)."""
    kind, planes, f = problem("lognormal", 511)
    xw, hw = oracle_solve(kind, planes, f, precision, nbf, maxit=6, tol=1e-14)
    h = bmg.Hierarchy(kind, dev(planes), precision=precision, smoother=smoother, arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-14, maxit=6)
    assert it == 6
    assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    check_history(h.history(), hw)


@pytest.mark.parametrize("precision,nbf", [("fp64", None), ("fp32", 0)])
@pytest.mark.parametrize("smoother", ["line", "xyline"])
def test_fused_line_relaxation_solve_bitwise(bmg, precision, nbf, smoother):
    """Line relaxation keeps its own (rounded) arithmetic; the residual,
    restriction and interpolation around it are fused."""
    kind, planes, f = 5, w.anisotropic5(127, 0.01), w.rhs_uniform(127, 1)
    xw, hw = oracle_solve(kind, planes, f, precision, nbf, smoother=smoother)
    h = bmg.Hierarchy(kind, dev(planes[:3]), precision=precision, smoother=smoother, arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok and it == len(hw) - 1
    assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    check_history(h.history(), hw)


@pytest.mark.parametrize("precision,nbf,smoother", [("fp64", None, "auto"), ("fp32", 0, "auto"),
                                                    ("fp32", 0, "pair3"), ("bf16", 2, "tile2")])
@pytest.mark.parametrize("graph", [True, False])
def test_fused_batched_matches_oracle_per_problem(bmg, precision, nbf, smoother, graph):
    sizes = [63, 255, 7, 127, 63, 3, 255, 31]
    probs = batch_problems(sizes)
    B = bmg.Batch(9, [dev(p[1]) for p in probs], precision=precision, use_graph=graph, smoother=smoother,
                  arith="fused")
    xs, its, rrs, ok = B.solve([dev(p[2]) for p in probs], tol=1e-9, maxit=100)
    assert ok
    for k, (kind, planes, f) in enumerate(probs):
        xw, hw = oracle_solve(kind, planes, f, precision, nbf, tol=1e-9, maxit=100)
        assert its[k] == len(hw) - 1, k
        assert np.array_equal(bx.at(host(xs[k]), 0, 0), bx.at(xw, 0, 0)), k
        check_history(B.history(k), hw)
    B.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_batch_of_right_hand_sides_equals_solo(bmg, precision):
    n, k = 255, 3
    kind, planes, f = problem("lognormal", n)
    h = bmg.Hierarchy(kind, dev(planes), precision=precision, arith="fused")
    rhs = [dev(w.rhs_uniform(n, 400 + q)) for q in range(k)]
    B = bmg.Batch.from_hierarchy(h, k)
    xs, its, rrs, ok = B.solve(rhs, tol=1e-10, maxit=300)
    assert ok
    for q, r in enumerate(rhs):
        x, it, rr, okk = h.solve(r, tol=1e-10, maxit=300)
        assert okk and it == its[q] and torch.equal(x, xs[q]) and h.history() == B.history(q)
    B.close()
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_history_tracks_the_rounded_one(bmg, precision):
    """The two arithmetic modes round differently (different iterates) but meet
    the stated history tolerance against each other: FP64 cycles, every entry
    within 1e-12 of ||r_0|| and the same number of cycles; FP32 cycles inside
    FP64 refinement differ at FP32 rounding level, every entry within 1e-6 of
    ||r_0|| and at most one step apart."""
    kind, planes, f = problem("binary", 255)
    hs = {}
    for arith in ("rounded", "fused"):
        h = bmg.Hierarchy(kind, dev(planes), precision=precision, arith=arith)
        x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
        assert ok
        hs[arith] = (host(x), h.history())
        h.close()
    (xr, hr), (xf, hf) = hs["rounded"], hs["fused"]
    assert not np.array_equal(xr, xf)
    if precision == "fp64":
        assert len(hr) == len(hf)
        assert max(abs(a - b) for a, b in zip(hr, hf)) <= 1e-12 * hr[0]
    else:
        assert abs(len(hr) - len(hf)) <= 1
        assert max(abs(a - b) for a, b in zip(hr, hf)) <= 1e-6 * hr[0]


@pytest.mark.slow
@pytest.mark.parametrize("precision,nbf", [("fp64", None), ("fp32", 0)])
def test_fused_bench_workload_first_cycles_bitwise(bmg, precision, nbf):
    """2047^2 bench workload, graph launch configuration, autotuned kernels:
    three fused cycles (refinement steps) against the oracle over every point."""
    kind, planes, f = w.binary_contrast_problem(2047, 16, seed_k=2, seed_f=3)
    xw, hw = oracle_solve(kind, planes, f, precision, nbf, tol=1e-14, maxit=3)
    h = bmg.Hierarchy(kind, dev(planes), precision=precision, arith="fused")
    x, it, rr, ok = h.solve(dev(f), tol=1e-14, maxit=3)
    assert it == 3
    assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    check_history(h.history(), hw)


def test_bad_arith_is_rejected(bmg):
    kind, planes, f = problem("binary", 63)
    with pytest.raises(KeyError):
        bmg.Hierarchy(kind, dev(planes), arith="fast")
    import ctypes
    o = bmg._lib.Opts()
    o.arith = 2
    coef = dev(planes)
    st = bmg._lib.Stencil(kind, bmg._lib._ptr(coef))
    hh = ctypes.c_void_p()
    rc = bmg._lib.lib.bmg_setup(ctypes.byref(st), 63, 63, ctypes.byref(o), ctypes.byref(hh))
    assert rc == bmg._lib.BMG_EINVAL
