"""GPU parity: every step of the hot path through the C ABI against the CPU
oracle on the same seeded inputs.  The FP64 path rounds every operation the
way the oracle does, so iterates, weights and coarse operators must agree bit
for bit.  Norms are summed in another order than the oracle's plain sum, so
residual histories are compared at the stated tolerance; the device's own
summation order is checked bit for bit with tests/reduction_order.py."""
import numpy as np
import pytest
import torch

import workloads as w
from oracle import boxmg as bx
from oracle import mixed as mx
from reduction_order import device_inner, device_norm

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy()


def problem(case, n):
    if case == "poisson":
        return w.poisson_problem(n, 1)
    if case == "binary":
        return w.binary_contrast_problem(n, 16 if n >= 127 else 4, seed_k=2, seed_f=3)
    if case == "lognormal":
        return w.lognormal_problem(n, 2.0, 8.0, seed_k=4, seed_f=7)
    raise ValueError(case)


CASES = [("poisson", 63), ("poisson", 255), ("binary", 127), ("binary", 255), ("lognormal", 255)]


@pytest.mark.parametrize("case,n", CASES)
def test_dendy_interp_bitwise(bmg, case, n):
    kind, planes, _ = problem(case, n)
    want = bx.dendy_interp(planes)
    got = host(bmg.dendy_interp(dev(planes)))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("case,n", CASES)
def test_rap_bitwise(bmg, case, n):
    kind, planes, _ = problem(case, n)
    ci = bx.dendy_interp(planes)
    want = bx.rap(planes, ci)
    got = host(bmg.rap(dev(planes), dev(ci)))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("case,n", CASES)
@pytest.mark.parametrize("sweeps", [1, 2])
def test_relax_bitwise(bmg, case, n, sweeps):
    kind, planes, f = problem(case, n)
    x0 = w.rhs_uniform(n, 99) * 0.1
    want = x0.copy()
    dinv = np.zeros_like(f)
    bx.at(dinv, 0, 0)[...] = 1.0 / bx.at(planes[0], 0, 0)
    for _ in range(sweeps):
        bx.gs_sweep(kind, planes, dinv, want, f)
    xg = dev(x0)
    bmg.relax(kind, dev(planes), dev(f), xg, sweeps)
    assert np.array_equal(host(xg), want)


@pytest.mark.parametrize("case,n", CASES)
def test_resid_restrict_bitwise(bmg, case, n):
    kind, planes, f = problem(case, n)
    x = w.rhs_uniform(n, 98) * 0.3
    ci = bx.dendy_interp(planes)
    want = bx.restrict(ci, bx.residual(planes, x, f))
    got = host(bmg.resid_restrict(kind, dev(planes), dev(ci), dev(x), dev(f)))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("case,n", CASES)
def test_interp_correct_bitwise(bmg, case, n):
    kind, planes, _ = problem(case, n)
    ci = bx.dendy_interp(planes)
    nc = (n - 1) // 2
    ec = w.rhs_uniform(nc, 97)
    x = w.rhs_uniform(n, 96)
    want = x.copy()
    bx.interp_correct(ci, ec, want)
    xg = dev(x)
    bmg.interp_correct(dev(ci), dev(ec), xg)
    assert np.array_equal(host(xg), want)


@pytest.mark.parametrize("case,n", CASES)
def test_residual_and_norm(bmg, case, n):
    kind, planes, f = problem(case, n)
    x = w.rhs_uniform(n, 95)
    want = bx.residual(planes, x, f)
    r, nrm = bmg.residual(kind, dev(planes), dev(x), dev(f))
    assert np.array_equal(host(r), want)
    assert nrm == device_norm(want)                      # the device's stated summation order
    assert nrm == pytest.approx(bx.norm(want), rel=1e-14, abs=0)


@pytest.mark.parametrize("n", [3, 7, 15])
def test_coarse_factor_and_solve_bitwise(bmg, n):
    kind, planes, f = problem("lognormal", n)
    A = bx.dense_matrix(planes)
    Lw = bx.cholesky(A)
    Lg = bmg.coarse_factor(dev(planes))
    assert np.array_equal(host(Lg), Lw)
    want = np.zeros_like(f)
    bx.at(want, 0, 0)[...] = bx.chol_solve(Lw, bx.at(f, 0, 0).reshape(-1)).reshape(n, n)
    xg = torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda")
    bmg.coarse_solve(Lg, dev(f), xg)
    assert np.array_equal(host(xg), want)


def test_coarse_factor_rejects_indefinite(bmg):
    planes = w.poisson5(3)
    planes[0] *= -1.0
    with pytest.raises(bmg.BmgError) as e:
        bmg.coarse_factor(dev(planes))
    assert e.value.code == -4


@pytest.mark.parametrize("case,n", [("poisson", 127), ("binary", 255), ("lognormal", 127)])
def test_hierarchy_bitwise(bmg, case, n):
    kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes)
    coef = dev(planes[:3] if kind == 5 else planes)
    h = bmg.Hierarchy(kind, coef)
    assert h.num_levels == len(levels)
    for l, lev in enumerate(levels):
        assert h.level_size(l) == lev.n
        assert np.array_equal(host(h.stencil(l)), lev.planes)
        if lev.ci is not None:
            assert np.array_equal(host(h.interp(l)), lev.ci)
    h.close()


def check_history(got, want):
    """The stated reading of "residual histories match to 1e-12": the same
    number of entries (iteration counts), every entry within 1e-12 ||r_0||, and
    within 1e-12 relative while above 1e-3 ||r_0||.  The iterates behind the
    histories are compared bit for bit by the callers; only the summation
    order of the norms differs."""
    assert len(got) == len(want)
    r0 = want[0]
    for g, t in zip(got, want):
        assert abs(g - t) <= 1e-12 * r0
        if t >= 1e-3 * r0:
            assert abs(g - t) <= 1e-12 * t


def check_fcg(bmg_x, got_hist, want, want_dev, mixed, planes=None, f=None, tol=None):
    """Flexible CG, where the inner products feed back into the iterates.
    want_dev = the oracle's FCG run with the device's summation order
    (tests/reduction_order.py): iterates and history equal bit for bit.
    want = the oracle's plain-sum run: the reading for FCG, identical
    iteration counts, entries above 1e-3 r0 within 1e-6 relative and the
    others within 1e-9 r0.  The rounding of alpha and beta propagates through
    the recurrences, amplified by the conditioning (measured up to 4e-9
    relative in FP64 at contrast 1e6, where the history is not monotone) and,
    with an FP32/BF16 preconditioner, by the FP32 rounding of z (up to 9e-9
    relative, 1e-10 r0).  With planes and f given, the oracle's FP64 residual
    of the returned x meets the tolerance."""
    xd, hd = want_dev
    assert np.array_equal(host(bmg_x)[1:-1, 1:-1], xd[1:-1, 1:-1])
    assert list(got_hist) == list(hd)
    xw, hw = want
    assert len(got_hist) == len(hw)
    r0 = hw[0]
    for g, t in zip(got_hist, hw):
        assert abs(g - t) <= (1e-6 * t if t >= 1e-3 * r0 else 1e-9 * r0)
    if planes is not None:
        p64 = bx.drop_ghost_couplings(np.array(planes, dtype=np.float64))
        assert bx.norm(bx.residual(p64, host(bmg_x), f)) <= 2 * tol * r0


@pytest.mark.parametrize("case,n", [("poisson", 127), ("binary", 255), ("lognormal", 255), ("poisson", 7),
                                    ("binary", 3)])
@pytest.mark.parametrize("graph", [True, False])
def test_fp64_solve_matches_oracle(bmg, case, n, graph):
    kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes)
    xw, hw = bx.solve(levels, f, tol=1e-10, maxit=200)
    h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), use_graph=graph)
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok and it == len(hw) - 1
    assert np.array_equal(host(x), xw)
    check_history(h.history(), hw)
    # the device norms of the same iterates, in the device's summation order
    _, hd = bx.solve(levels, f, tol=1e-10, maxit=200, inner=device_inner())
    assert h.history() == hd
    assert rr <= 1e-10
    h.close()


def test_fp64_solve_with_initial_guess_and_maxit(bmg):
    kind, planes, f = problem("binary", 127)
    levels = bx.setup(kind, planes)
    x0 = w.rhs_uniform(127, 5)
    xw, hw = bx.solve(levels, f, x0=x0, tol=1e-12, maxit=3)
    h = bmg.Hierarchy(kind, dev(planes))
    x, it, rr, ok = h.solve(dev(f), dev(x0), tol=1e-12, maxit=3)
    assert not ok and it == 3
    assert np.array_equal(host(x), xw)
    check_history(h.history(), hw)


def test_zero_rhs_and_zero_maxit(bmg):
    kind, planes, f = problem("poisson", 63)
    h = bmg.Hierarchy(kind, dev(planes[:3]))
    x, it, rr, ok = h.solve(torch.zeros((65, 65), dtype=torch.float64, device="cuda"))
    assert ok and it == 0 and not x.any()
    x, it, rr, ok = h.solve(dev(f), maxit=0)
    assert not ok and it == 0 and not x.any()


def test_nan_rhs_reports_enan(bmg):
    kind, planes, f = problem("poisson", 63)
    f[10, 10] = np.nan
    h = bmg.Hierarchy(kind, dev(planes[:3]))
    with pytest.raises(bmg.BmgError) as e:
        h.solve(dev(f))
    assert e.value.code == -5


def test_setup_rejects_bad_sizes_and_indefinite(bmg):
    planes = w.poisson5(63)
    with pytest.raises(bmg.BmgError):                     # a learned hierarchy needs a 2^m - 1 square
        bmg.Hierarchy(5, dev(planes[:3, :64, :64].copy()), mlp=bmg.Mlp(np.zeros(bmg._lib.MLP_PARAMS, np.float32)))
    bad = planes.copy()
    bad[0] *= -1
    with pytest.raises(bmg.BmgError) as e:
        bmg.Hierarchy(5, dev(bad[:3]))
    assert e.value.code == -4


# ---- mixed precision -----------------------------------------------------------

@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("case,n", [("binary", 255), ("lognormal", 127), ("poisson", 63)])
def test_inner_cycle_bitwise(bmg, precision, nbf, case, n):
    kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes)
    l32 = mx.lower(levels, nbf)
    r32 = (w.rhs_uniform(n, 94)).astype(np.float32)
    want = mx.inner_cycle(l32, r32)
    h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), precision=precision)
    got = host(h.inner_cycle(dev(r32, torch.float32)))
    assert np.array_equal(bx.at(got, 0, 0), bx.at(want, 0, 0))


@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("case,n", [("binary", 255), ("lognormal", 255), ("poisson", 127)])
def test_ir_solve_matches_oracle(bmg, precision, nbf, case, n):
    kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes)
    xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), f, tol=1e-10, maxit=200)
    h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), precision=precision)
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok and it == len(hw) - 1
    assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    check_history(h.history(), hw)
    # the refined solution is FP64-accurate: its oracle residual meets the tolerance
    assert bx.norm(bx.residual(levels[0].planes, host(x), f)) <= 1e-10 * hw[0]


# ---- full size of the bench workload ----------------------------------------------

@pytest.mark.slow
def test_bench_workload_first_cycles_bitwise(bmg):
    """2047^2, 9-point, k in {1, 1e4} on 16x16 blocks: setup and three V(2,1)
    cycles in the launch configuration the bench times (CUDA graph), compared
    with the oracle over every grid point."""
    kind, planes, f = w.binary_contrast_problem(2047, 16, seed_k=2, seed_f=3)
    levels = bx.setup(kind, planes)
    xw, hw = bx.solve(levels, f, tol=1e-14, maxit=3)
    h = bmg.Hierarchy(kind, dev(planes))
    for l in (0, 1):
        assert np.array_equal(host(h.stencil(l)), levels[l].planes)
    x, it, rr, ok = h.solve(dev(f), tol=1e-14, maxit=3)
    assert it == 3
    assert np.array_equal(host(x), xw)
    check_history(h.history(), hw)


def test_time_cycles_and_profile(bmg):
    kind, planes, f = problem("binary", 255)
    h = bmg.Hierarchy(kind, dev(planes))
    x = torch.zeros((257, 257), dtype=torch.float64, device="cuda")
    before = h.launch_count
    ms = h.time_cycles(dev(f), x, 5)
    assert ms > 0 and h.launch_count > before
    levels = bx.setup(kind, planes)
    xw = np.zeros_like(f)
    for _ in range(5):
        bx.vcycle(levels, 0, xw, f)
    assert np.array_equal(host(x), xw)
    rows = h.profile(dev(f), torch.zeros_like(x), 2)
    kinds = {(r["level"], r["kernel"]) for r in rows}
    assert (0, "relax") in kinds and (0, "resid_restrict") in kinds and (0, "residual_norm") in kinds
    # the coarse levels run either step by step or as one level-fused launch
    assert (len(levels) - 1, "coarse_solve") in kinds or any(k == "tail" for _, k in kinds)
    assert all(r["ms"] > 0 and r["launches"] > 0 for r in rows)


# ---- flexible CG --------------------------------------------------------------------

@pytest.mark.parametrize("precision,nbf", [("fp64", None), ("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("case,n", [("binary", 255), ("lognormal", 127), ("poisson", 63)])
def test_fcg_solve_bitwise(bmg, precision, nbf, case, n):
    kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes)
    if precision == "fp64":
        run = lambda inner=None: bx.solve_fcg(levels, f, tol=1e-10, maxit=200, inner=inner)
    else:
        l32 = mx.lower(levels, nbf)
        run = lambda inner=None: mx.solve_fcg_ir(levels, l32, f, tol=1e-10, maxit=200, inner=inner)
    h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), precision=precision, krylov="fcg")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok
    check_fcg(x, h.history(), run(), run(device_inner()), precision != "fp64", planes, f, 1e-10)


def test_fcg_high_contrast_converges_where_cycles_stall(bmg):
    kind, planes, f = w.binary_contrast_problem(255, 8, 1.0, 1e6, seed_k=6, seed_f=7)
    h = bmg.Hierarchy(kind, dev(planes), krylov="fcg")
    x, it, rr, ok = h.solve(dev(f), tol=1e-8, maxit=300)
    assert ok and rr <= 1e-8
    levels = bx.setup(kind, planes)
    check_fcg(x, h.history(), bx.solve_fcg(levels, f, tol=1e-8, maxit=300),
              bx.solve_fcg(levels, f, tol=1e-8, maxit=300, inner=device_inner()), False)


# ---- batched solves -----------------------------------------------------------------

def batch_problems(sizes, std=1.0):
    out = []
    for b, n in enumerate(sizes):
        k = w.lognormal_cells(n, std, 8.0, 20000 + 2 * b)
        out.append((9, w.fe9_from_cells(k), w.rhs_uniform(n, 20001 + 2 * b)))
    return out


@pytest.mark.parametrize("precision,nbf,smoother", [("fp64", None, "auto"), ("fp32", 0, "auto"), ("bf16", 2, "auto"),
                                                    ("fp32", 0, "tile0"), ("fp32", 0, "tile3"), ("bf16", 2, "tile2"),
                                                    ("fp32", 0, "pair0"), ("bf16", 2, "pair3"), ("fp64", None, "tile0"),
                                                    ("fp64", None, "tile1"), ("fp64", None, "tile2"),
                                                    ("fp64", None, "tile3")])
@pytest.mark.parametrize("graph", [True, False])
def test_batched_matches_oracle_per_problem(bmg, precision, nbf, smoother, graph):
    """Uneven sizes (several problems per size, sizes from 3 to 255, ragged
    tiles), every problem's iterate and history equal its oracle solve; with
    the one-pass / two-sweep kernels forced on the FP32 stages as well."""
    sizes = [63, 255, 7, 127, 63, 3, 255, 31, 15, 127, 63]
    probs = batch_problems(sizes)
    B = bmg.Batch(9, [dev(p[1]) for p in probs], precision=precision, use_graph=graph, smoother=smoother)
    xs, its, rrs, ok = B.solve([dev(p[2]) for p in probs], tol=1e-9, maxit=100)
    assert ok
    for k, (kind, planes, f) in enumerate(probs):
        levels = bx.setup(kind, planes)
        if precision == "fp64":
            xw, hw = bx.solve(levels, f, tol=1e-9, maxit=100)
        else:
            xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), f, tol=1e-9, maxit=100)
        assert its[k] == len(hw) - 1, k
        assert np.array_equal(bx.at(host(xs[k]), 0, 0), bx.at(xw, 0, 0)), k
        check_history(B.history(k), hw)
    B.close()


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (1, 2), (3, 0), (0, 3), (2, 2)])
@pytest.mark.parametrize("arith", ["rounded", "fused"])
def test_batched_fp64_one_pass_any_sweep_counts(bmg, nu1, nu2, arith):
    """The batched FP64 one-pass sweep moves each iterate between x and a
    second array; odd and even sweep counts on both sides of the coarse
    correction must leave the oracle's iterate in the caller's x."""
    sizes = [255, 127, 511, 63, 255]
    probs = batch_problems(sizes)
    B = bmg.Batch(9, [dev(p[1]) for p in probs], nu1=nu1, nu2=nu2, smoother="tile0", arith=arith)
    xs, its, rrs, ok = B.solve([dev(p[2]) for p in probs], tol=1e-14, maxit=4)
    for k, (kind, planes, f) in enumerate(probs):
        xw, hw = bx.solve(bx.setup(kind, planes, arith=arith), f, tol=1e-14, maxit=4, nu1=nu1, nu2=nu2)
        assert its[k] == len(hw) - 1, k
        assert np.array_equal(bx.at(host(xs[k]), 0, 0), bx.at(xw, 0, 0)), k
        check_history(B.history(k), hw)
    B.close()


def test_batched_fp64_tuner_and_right_hand_sides(bmg):
    """Autotuned FP64 batch (row kernel or one-pass shape per stage) and an
    FP64 batch of right-hand sides with the one-pass kernel forced: both equal
    the solo solves bit for bit."""
    probs = batch_problems([511, 255, 255, 1023])
    B = bmg.Batch(9, [dev(p[1]) for p in probs])
    xs, its, rrs, ok = B.solve([dev(p[2]) for p in probs], tol=1e-10, maxit=100)
    assert ok
    assert B.tuned_cluster(8) in (1, 2, 4, 8, 16, 17, 18, 19)   # n = 1023
    for k, (kind, planes, f) in enumerate(probs):
        h = bmg.Hierarchy(kind, dev(planes))
        x, it, rr, okk = h.solve(dev(f), tol=1e-10, maxit=100)
        assert it == its[k] and torch.equal(x, xs[k]) and h.history() == B.history(k)
        h.close()
    B.close()
    kind, planes, f = problem("lognormal", 511)
    h = bmg.Hierarchy(kind, dev(planes))
    rhs = [dev(w.rhs_uniform(511, 500 + q)) for q in range(3)]
    R = bmg.Batch.from_hierarchy(h, 3, smoother="tile2")
    xs, its, rrs, ok = R.solve(rhs, tol=1e-10, maxit=100)
    assert ok
    for q, r in enumerate(rhs):
        x, it, rr, okk = h.solve(r, tol=1e-10, maxit=100)
        assert okk and it == its[q] and torch.equal(x, xs[q]) and h.history() == R.history(q)
    R.close()
    h.close()


def test_batched_fp64_pair_is_rejected(bmg):
    probs = batch_problems([63, 127])
    with pytest.raises(bmg.BmgError):
        bmg.Batch(9, [dev(p[1]) for p in probs], smoother="pair0")


@pytest.mark.parametrize("smoother", ["auto", "pair3"])
def test_batched_equals_solo_solve(bmg, smoother):
    sizes = [127, 255, 63, 511]
    probs = batch_problems(sizes, std=2.0)
    B = bmg.Batch(9, [dev(p[1]) for p in probs], precision="fp32", smoother=smoother)
    xs, its, rrs, ok = B.solve([dev(p[2]) for p in probs], tol=1e-9, maxit=200)
    for k, (kind, planes, f) in enumerate(probs):
        h = bmg.Hierarchy(kind, dev(planes), precision="fp32")
        x, it, rr, okk = h.solve(dev(f), tol=1e-9, maxit=200)
        assert it == its[k] and torch.equal(x, xs[k]) and h.history() == B.history(k)
        h.close()


def test_batched_time_cycles_and_tuner(bmg):
    probs = batch_problems([255, 255, 511, 127])
    B = bmg.Batch(9, [dev(p[1]) for p in probs], precision="fp32")
    rhs = [dev(p[2]) for p in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    ms = B.time_cycles(rhs, xs, 3)
    assert ms > 0
    # stages of n >= 127 were tuned to an admissible row-kernel cluster size
    # or (FP32, n >= 255) a one-pass shape
    for stage in range(1, 8):
        cl = B.tuned_cluster(stage)
        assert cl in (0, 1, 2, 4, 8, 16, 17, 18, 19)
    assert B.tuned_cluster(6) in (1, 2, 4, 8, 16, 17, 18, 19)   # n = 255
    B.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_level_fused_tail_is_bitwise_the_stepwise_cycle(bmg, precision):
    """use_graph=True runs the coarse levels as one fused launch; use_graph=False
    launches every step; both must give the same bits (and the oracle's)."""
    for case, n in [("binary", 255), ("poisson", 63), ("lognormal", 31)]:
        kind, planes, f = problem(case, n)
        coef = dev(planes[:3] if kind == 5 else planes)
        outs = []
        for graph in (True, False):
            h = bmg.Hierarchy(kind, coef, precision=precision, use_graph=graph)
            x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
            outs.append((host(x), h.history()))
            if graph:
                prof = h.profile(dev(f), torch.zeros_like(x), 1)
                assert any(r["kernel"] == "tail" for r in prof), (case, n)
            h.close()
        assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


# ---- one-pass four-colour sweep (FP32 levels, warp strips) -----------------------------

@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("shape", ["tile0", "tile1", "tile2", "tile3", "tile4", "tile5"])
@pytest.mark.parametrize("graph", [False, True])
def test_tile_sweep_inner_cycle_bitwise(bmg, precision, nbf, shape, graph):
    """The one-pass kernel recomputes halo points redundantly and alternates
    two iterates; every level's result must still be the oracle's bits."""
    for case, n in [("binary", 255), ("lognormal", 127), ("poisson", 63)]:
        kind, planes, f = problem(case, n)
        levels = bx.setup(kind, planes)
        r32 = w.rhs_uniform(n, 95).astype(np.float32)
        want = mx.inner_cycle(mx.lower(levels, nbf), r32)
        h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), precision=precision, smoother=shape,
                          use_graph=graph)
        got = host(h.inner_cycle(dev(r32, torch.float32)))
        assert np.array_equal(bx.at(got, 0, 0), bx.at(want, 0, 0)), (case, n)
        if kind == 9:
            assert h.tuned_cluster(0) == bmg.TILE_SWEEP + int(shape[-1])
        h.close()


@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("shape", ["pair0", "pair1", "pair2", "pair3"])
@pytest.mark.parametrize("graph", [False, True])
def test_two_sweep_pass_inner_cycle_bitwise(bmg, precision, nbf, shape, graph):
    """Two sweeps in one pass (48-column strips, sweep 2 one step behind
    sweep 1, rows streamed once): every level's result is the oracle's bits."""
    for case, n in [("binary", 255), ("lognormal", 127), ("poisson", 63)]:
        kind, planes, f = problem(case, n)
        levels = bx.setup(kind, planes)
        r32 = w.rhs_uniform(n, 97).astype(np.float32)
        want = mx.inner_cycle(mx.lower(levels, nbf), r32)
        h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), precision=precision, smoother=shape,
                          use_graph=graph)
        got = host(h.inner_cycle(dev(r32, torch.float32)))
        assert np.array_equal(bx.at(got, 0, 0), bx.at(want, 0, 0)), (case, n)
        if kind == 9:
            assert h.tuned_pair(0) == int(shape[-1])
        h.close()


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (1, 2), (3, 0), (0, 3), (2, 2), (4, 1), (3, 3)])
@pytest.mark.parametrize("one_pass", ["tile", "pair"])
def test_tile_sweep_any_sweep_counts_equal_row_kernel(bmg, nu1, nu2, one_pass):
    """Odd and even numbers of alternating sweeps (single or paired) before and
    after the coarse correction: the refinement solve equals the row-kernel one."""
    kind, planes, f = problem("lognormal", 255)
    outs = []
    for sm in ("rows", one_pass):
        h = bmg.Hierarchy(kind, dev(planes), precision="fp32", smoother=sm, nu1=nu1, nu2=nu2, use_graph=False)
        x, it, rr, ok = h.solve(dev(f), tol=1e-9, maxit=60)
        outs.append((host(x), h.history()))
        h.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_tile_sweep_fcg_and_bf16_solve_match_oracle(bmg):
    kind, planes, f = problem("binary", 255)
    levels = bx.setup(kind, planes)
    for precision, nbf in (("fp32", 0), ("bf16", 2)):
        l32 = mx.lower(levels, nbf)
        h = bmg.Hierarchy(kind, dev(planes), precision=precision, krylov="fcg", smoother="tile")
        x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
        assert ok
        check_fcg(x, h.history(), mx.solve_fcg_ir(levels, l32, f, tol=1e-10, maxit=200),
                  mx.solve_fcg_ir(levels, l32, f, tol=1e-10, maxit=200, inner=device_inner()), True)
        h.close()


def test_autotuner_picks_a_valid_kernel_per_level(bmg):
    kind, planes, f = problem("lognormal", 511)
    for precision in ("fp32", "bf16", "fp64"):
        h = bmg.Hierarchy(kind, dev(planes), precision=precision)
        shapes = 4 if precision == "fp64" else 6
        for l in range(h.num_levels - 1):
            c = h.tuned_cluster(l)
            assert c in (0, 1, 2, 4, 8) or bmg.TILE_SWEEP <= c < bmg.TILE_SWEEP + shapes, (l, c)
            assert h.tuned_pair(l) in (-1, 0, 1, 2, 3)
            assert h.tuned_pair(l) == -1 or c >= bmg.TILE_SWEEP
        assert h.tuned_cluster(0) != 0
        h.close()


@pytest.mark.parametrize("shape", ["tile0", "tile1", "tile2", "tile3"])
@pytest.mark.parametrize("arith", ["rounded", "fused"])
@pytest.mark.parametrize("case,n", [("lognormal", 511), ("binary", 127), ("poisson", 63)])
@pytest.mark.parametrize("graph", [True, False])
def test_fp64_one_pass_sweep_solve_bitwise(bmg, shape, arith, case, n, graph):
    """The FP64 one-pass kernel forced on every 9-point level (strips of 56
    columns over 511, 127 and 63 points: several strips, ragged right and top
    edges, a grid narrower than one strip): iterates and histories equal the
    oracle's, in both arithmetic modes."""
    kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes, arith=arith)
    xw, hw = bx.solve(levels, f, tol=1e-10, maxit=200)
    h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), smoother=shape, use_graph=graph, arith=arith)
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok and it == len(hw) - 1
    assert np.array_equal(host(x), xw)
    check_history(h.history(), hw)
    h.close()


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (3, 0), (0, 3), (2, 2), (1, 2)])
def test_fp64_one_pass_any_sweep_counts_and_fcg(bmg, nu1, nu2):
    kind, planes, f = problem("lognormal", 255)
    levels = bx.setup(kind, planes)
    run = lambda inner=None: bx.solve_fcg(levels, f, tol=1e-10, maxit=200, nu1=nu1, nu2=nu2, inner=inner)
    h = bmg.Hierarchy(kind, dev(planes), smoother="tile1", nu1=nu1, nu2=nu2, krylov="fcg")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok
    check_fcg(x, h.history(), run(), run(device_inner()), False)
    h.close()


def test_fp64_rejects_smoothers_without_an_fp64_kernel(bmg):
    kind, planes, f = problem("binary", 63)
    for sm in ("tile4", "tile5", "pair0", "pair3"):
        with pytest.raises(bmg.BmgError):
            bmg.Hierarchy(kind, dev(planes), smoother=sm)


@pytest.mark.slow
@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
def test_bench_workload_fp32_cycle_bitwise(bmg, precision, nbf):
    """2047^2 bench workload: one FP32 (BF16) inner cycle in the launch
    configuration the bench times (autotuned kernels, graph), and with the
    one-pass kernel forced, against the oracle over every grid point."""
    kind, planes, f = w.binary_contrast_problem(2047, 16, seed_k=2, seed_f=3)
    levels = bx.setup(kind, planes)
    r32 = w.rhs_uniform(2047, 96).astype(np.float32)
    want = mx.inner_cycle(mx.lower(levels, nbf), r32)
    for sm in ("auto", "tile", "pair"):
        h = bmg.Hierarchy(kind, dev(planes), precision=precision, smoother=sm)
        got = host(h.inner_cycle(dev(r32, torch.float32)))
        assert np.array_equal(got, want), sm
        h.close()


def test_bounded_wait_gives_up_and_context_stays_usable(bmg):
    """The bulk-copy sweep's mbarrier wait has a poll limit: a wait on a phase
    that nothing completes must give up, be reported, and leave the context
    working (a solve afterwards still matches the oracle)."""
    assert bmg.lib.bmg_wait_selftest() == 0, bmg.lib.bmg_last_error().decode()
    kind, planes, f = problem("binary", 127)
    levels = bx.setup(kind, planes)
    xw, hw = mx.solve_ir(levels, mx.lower(levels, 0), f, tol=1e-10, maxit=200)
    h = bmg.Hierarchy(kind, dev(planes), precision="fp32", smoother="tile")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=200)
    assert ok and np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    h.close()


# ---- zebra line relaxation (x-lines, y-lines, alternating) ---------------------------------

def line_problem(case, n):
    if case == "aniso":                                   # -(u_xx + eps u_yy)
        return 5, w.anisotropic5(n, 1e-3), w.rhs_uniform(n, 5)
    if case == "anisoy":                                  # -(eps u_xx + u_yy)
        return 5, w.transposed_stencil(w.anisotropic5(n, 1e-3)), w.rhs_uniform(n, 5)
    return problem(case, n)


@pytest.mark.parametrize("case,n", [("poisson", 3), ("lognormal", 7), ("poisson", 63), ("lognormal", 255),
                                    ("binary", 127), ("aniso", 127), ("anisoy", 127)])
@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_line_relax_step_bitwise(bmg, case, n, sweeps, axis):
    kind, planes, f = line_problem(case, n)
    planes = bx.drop_ghost_couplings(np.array(planes))
    x0 = w.rhs_uniform(n, 98)
    want = x0.copy()
    for _ in range(sweeps):
        (bx.line_sweep if axis == "x" else bx.line_sweep_y)(kind, planes, want, f)
    got = host(bmg.relax_line(kind, dev(planes[:3] if kind == 5 else planes), dev(f), dev(x0), sweeps, axis=axis))
    assert np.array_equal(bx.at(got, 0, 0), bx.at(want, 0, 0))


@pytest.mark.parametrize("smoother,case,n", [("line", "aniso", 127), ("line", "lognormal", 255),
                                             ("line", "binary", 127), ("yline", "anisoy", 127),
                                             ("yline", "lognormal", 255), ("xyline", "aniso", 127),
                                             ("xyline", "anisoy", 127), ("xyline", "binary", 127)])
@pytest.mark.parametrize("graph", [True, False])
def test_line_solve_matches_oracle(bmg, smoother, case, n, graph):
    kind, planes, f = line_problem(case, n)
    levels = bx.setup(kind, planes, smoother=smoother)
    xw, hw = bx.solve(levels, f, tol=1e-10, maxit=100)
    h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), smoother=smoother, use_graph=graph)
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
    assert ok and it == len(hw) - 1
    assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    check_history(h.history(), hw)
    h.close()


@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("smoother,case", [("line", "aniso"), ("yline", "anisoy"), ("xyline", "anisoy")])
def test_line_refinement_and_fcg_match_oracle(bmg, precision, nbf, smoother, case):
    kind, planes, f = line_problem(case, 127)
    levels = bx.setup(kind, planes, smoother=smoother)
    xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), f, tol=1e-10, maxit=100)
    h = bmg.Hierarchy(kind, dev(planes[:3]), precision=precision, smoother=smoother)
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
    assert ok and it == len(hw) - 1
    assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    check_history(h.history(), hw)
    h.close()
    kind, planes, f = line_problem("lognormal", 127)
    levels = bx.setup(kind, planes, smoother=smoother)
    h = bmg.Hierarchy(kind, dev(planes), smoother=smoother, krylov="fcg")
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
    assert ok
    check_fcg(x, h.history(), bx.solve_fcg(levels, f, tol=1e-10, maxit=100),
              bx.solve_fcg(levels, f, tol=1e-10, maxit=100, inner=device_inner()), False)
    h.close()


@pytest.mark.parametrize("case", ["aniso", "anisoy"])
def test_line_relaxation_solves_anisotropy_point_gs_does_not(bmg, case):
    """Lines along the strong coupling (x-lines for aniso, y-lines for anisoy)
    and alternating lines converge in a few cycles; point Gauss-Seidel and
    lines across the strong coupling do not."""
    kind, planes, f = line_problem(case, 255)
    its = {}
    for sm in ("auto", "line", "yline", "xyline"):
        h = bmg.Hierarchy(kind, dev(planes[:3]), smoother=sm)
        x, it, rr, ok = h.solve(dev(f), tol=1e-8, maxit=60)
        its[sm] = (it, ok)
        h.close()
    along, across = ("line", "yline") if case == "aniso" else ("yline", "line")
    for sm in (along, "xyline"):
        assert its[sm][1] and its[sm][0] <= 10, its
    assert not its["auto"][1] and not its[across][1], its
    for sm in ("line", "yline", "xyline"):
        with pytest.raises(bmg.BmgError):
            bmg.Batch(5, [dev(planes[:3])], smoother=sm)


@pytest.mark.parametrize("coarsest", [7, 15])
@pytest.mark.parametrize("precision,nbf", [("fp64", None), ("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("case,n", [("lognormal", 255), ("binary", 15), ("poisson", 7)])
def test_coarsest_size_and_single_level_hierarchies(bmg, coarsest, precision, nbf, case, n):
    """A larger coarsest level (dense Cholesky of up to 225 unknowns), and
    hierarchies whose finest level is the coarsest (n <= coarsest: one direct
    solve per iteration)."""
    kind, planes, f = problem(case, n)
    levels = bx.setup(kind, planes, coarsest=min(coarsest, n))
    if precision == "fp64":
        xw, hw = bx.solve(levels, f, tol=1e-10, maxit=100)
    else:
        xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), f, tol=1e-10, maxit=100)
    h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), precision=precision, coarsest=coarsest)
    assert h.num_levels == len(levels)
    x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
    assert ok and it == len(hw) - 1
    assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0))
    check_history(h.history(), hw)
    h.close()


# ---- full benchmark sizes: properties the oracle can check at that scale -------------------

@pytest.mark.slow
def test_config3_full_size_setup_and_solves():
    """8191^2 log-normal (sigma 2, 32-cell correlation): the Galerkin stencil of
    the second level equals the oracle's bit for bit, and the stationary FP64
    and BF16-refinement solves (which test the true FP64 residual each
    iteration) return x whose oracle FP64 residual meets the tolerance."""
    import paper_2502_05279_gb300 as bmg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kind, planes, f = w.lognormal_problem(8191, 2.0, 32.0, seed_k=4, seed_f=7)
    p64 = bx.drop_ghost_couplings(np.array(planes))
    f0 = bx.norm(bx.at(f, 0, 0))
    coef, rhs = dev(planes), dev(f)
    h = bmg.Hierarchy(kind, coef)
    lv0 = bx.Level(8191, kind, p64)
    lv0.ci = bx.dendy_interp(p64)
    assert np.array_equal(host(h.interp(0)), lv0.ci)
    assert np.array_equal(host(h.stencil(1)), bx.rap(p64, lv0.ci))
    for hh, fu in ((h, False), (bmg.Hierarchy(kind, coef, precision="bf16"), False),
                   (bmg.Hierarchy(kind, coef, arith="fused"), True),
                   (bmg.Hierarchy(kind, coef, precision="fp32", arith="fused"), True)):
        x, it, rr, ok = hh.solve(rhs, tol=1e-10, maxit=100)
        assert ok
        assert bx.norm(bx.residual(p64, host(x), f)) <= 1e-10 * f0
        # the last history entry is the norm of the true FP64 residual, in the solve's own arithmetic
        assert hh.history()[-1] == pytest.approx(bx.norm(bx.residual(p64, host(x), f, fused=fu)), rel=1e-12, abs=0)
        hh.close()


@pytest.mark.slow
@pytest.mark.parametrize("arith", ["rounded", "fused"])
def test_config4_full_batch_converges_to_oracle_residuals(arith):
    """The 256-problem batch (sides 63 .. 1023, 80 M unknowns): every problem's
    FP32-refinement solution meets tol 1e-8 by the oracle's FP64 residual."""
    import paper_2502_05279_gb300 as bmg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    probs = w.batched_problems(256, 5, 1.0, 32.0)
    B = bmg.Batch(9, [dev(p[1]) for p in probs], precision="fp32", arith=arith)
    xs, its, rrs, ok = B.solve([dev(p[2]) for p in probs], tol=1e-8, maxit=100)
    assert ok
    for (kind, planes, f), x in zip(probs, xs):
        p64 = bx.drop_ghost_couplings(np.array(planes))
        assert bx.norm(bx.residual(p64, host(x), f)) <= 1e-8 * bx.norm(bx.at(f, 0, 0))
    B.close()


# ---- many right-hand sides of one operator -------------------------------------------------

@pytest.mark.parametrize("precision,nbf", [("fp64", None), ("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_of_right_hand_sides_equals_solo_solves(bmg, precision, nbf, graph):
    """k right-hand sides share one hierarchy's operator: every member's iterate
    and history equal the hierarchy's own solve of that right-hand side, which
    equals the oracle's; the hierarchy is unchanged by the batch."""
    n, k = 255, 5
    kind, planes, f = problem("lognormal", n)
    h = bmg.Hierarchy(kind, dev(planes), precision=precision)
    rhs = [dev(w.rhs_uniform(n, 300 + q)) for q in range(k)]
    B = bmg.Batch.from_hierarchy(h, k, use_graph=graph)
    xs, its, rrs, ok = B.solve(rhs, tol=1e-10, maxit=300)
    assert ok
    for q, r in enumerate(rhs):
        x, it, rr, okk = h.solve(r, tol=1e-10, maxit=300)
        assert okk and it == its[q] and torch.equal(x, xs[q]) and h.history() == B.history(q)
    levels = bx.setup(kind, planes)
    fq = w.rhs_uniform(n, 302)
    if precision == "fp64":
        xw, hw = bx.solve(levels, fq, tol=1e-10, maxit=300)
    else:
        xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), fq, tol=1e-10, maxit=300)
    assert np.array_equal(bx.at(host(xs[2]), 0, 0), bx.at(xw, 0, 0))
    check_history(B.history(2), hw)
    B.close()
    h.close()


def test_batch_of_right_hand_sides_rejects_bad_arguments(bmg):
    kind, planes, f = problem("binary", 63)
    h = bmg.Hierarchy(kind, dev(planes), precision="fp32")
    with pytest.raises(bmg.BmgError):
        bmg.Batch.from_hierarchy(h, 0)
    o = bmg._lib.Opts(bmg._lib._PREC["fp64"], 0, 0, 2, 1, 1, 0, 1, 0, None, None, 0)
    b = __import__("ctypes").c_void_p()
    rc = bmg.lib.bmg_batch_rhs(h._h, 3, __import__("ctypes").byref(o), __import__("ctypes").byref(b))
    assert rc == bmg._lib.BMG_EINVAL and "precision" in bmg.lib.bmg_last_error().decode()
    h.close()


def test_concurrent_setups_on_two_host_threads(bmg):
    """Two hierarchies set up at once from two host threads (ctypes releases the
    GIL; the autotuner caches are shared): both solve exactly as one built alone."""
    import threading
    kind, planes, f = problem("lognormal", 511)
    hs, errs = [None, None], []

    def build(k, precision):
        try:
            torch.cuda.set_device(0)
            hs[k] = bmg.Hierarchy(kind, dev(planes), precision=precision, arith="fused")
        except Exception as e:   # surfaced below
            errs.append(e)

    ts = [threading.Thread(target=build, args=(0, "fp32")), threading.Thread(target=build, args=(1, "fp64"))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs
    for h, precision in zip(hs, ("fp32", "fp64")):
        x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
        ref = bmg.Hierarchy(kind, dev(planes), precision=precision, arith="fused")
        x2, it2, rr2, ok2 = ref.solve(dev(f), tol=1e-10, maxit=100)
        assert ok and it == it2 and torch.equal(x, x2) and h.history() == ref.history()
        ref.close()
        h.close()


# ---- temporal blocking: two sweeps, residual and restriction in one pass --------------------

@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("shape", ["pair0", "pair1"])
@pytest.mark.parametrize("arith", ["rounded", "fused"])
@pytest.mark.parametrize("graph", [False, True])
def test_pair_restrict_pass_inner_cycle_bitwise(bmg, precision, nbf, shape, arith, graph):
    """The one-pass pre-smoothing with the residual and its restriction (44-
    column strips, coarse right-hand sides written from the walk) forced on
    every level: the inner cycle is the oracle's bit for bit, over grids with
    several strips and bands, ragged right and top edges, and a grid narrower
    than one strip."""
    for case, n in [("lognormal", 511), ("binary", 255), ("lognormal", 127), ("poisson", 63)]:
        kind, planes, f = problem(case, n)
        levels = bx.setup(kind, planes, arith=arith)
        r32 = w.rhs_uniform(n, 91).astype(np.float32)
        want = mx.inner_cycle(mx.lower(levels, nbf), r32)
        h = bmg.Hierarchy(kind, dev(planes[:3] if kind == 5 else planes), precision=precision, smoother=shape,
                          use_graph=graph, arith=arith, fuse_restrict="on")
        got = host(h.inner_cycle(dev(r32, torch.float32)))
        assert np.array_equal(bx.at(got, 0, 0), bx.at(want, 0, 0)), (case, n)
        if kind == 9 and not graph:
            prof = h.profile(dev(f), torch.zeros_like(dev(f)), 1)
            assert any(r["kernel"] == "pair_restrict" for r in prof), (case, n)
        h.close()


@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
def test_pair_restrict_solve_matches_oracle_and_tuner_choice(bmg, precision, nbf):
    """Refinement solves with the fused pass forced equal the oracle's
    iterates bit for bit; with the autotuner the pass is chosen or not per
    level and the solve is the same bits either way."""
    kind, planes, f = problem("lognormal", 1023)
    levels = bx.setup(kind, planes, arith="fused")
    xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), f, tol=1e-10, maxit=100)
    outs = []
    for fr in ("on", "auto", "off"):
        h = bmg.Hierarchy(kind, dev(planes), precision=precision, smoother="pair0" if fr == "on" else "auto",
                          arith="fused", fuse_restrict=fr)
        x, it, rr, ok = h.solve(dev(f), tol=1e-10, maxit=100)
        assert ok and it == len(hw) - 1
        assert np.array_equal(bx.at(host(x), 0, 0), bx.at(xw, 0, 0)), fr
        check_history(h.history(), hw)
        outs.append(h.history())
        h.close()
    assert outs[0] == outs[1] == outs[2]


def test_pair_restrict_rejects_bad_option(bmg):
    kind, planes, f = problem("binary", 63)
    with pytest.raises(KeyError):
        bmg.Hierarchy(kind, dev(planes), fuse_restrict="maybe")
    import ctypes
    o = bmg._lib.Opts()
    o.fuse_restrict = 3
    st = bmg._lib.Stencil(kind, bmg._lib._ptr(dev(planes)))
    hh = ctypes.c_void_p()
    assert bmg._lib.lib.bmg_setup(ctypes.byref(st), 63, 63, ctypes.byref(o), ctypes.byref(hh)) == bmg._lib.BMG_EINVAL


# ---- block right-hand sides: one-pass sweeps with K members of one operator per warp ------------

@pytest.mark.parametrize("precision,nbf", [("fp32", 0), ("bf16", 2)])
@pytest.mark.parametrize("block,k", [(2, 5), (4, 5), (4, 8), ("auto", 6)])
@pytest.mark.parametrize("graph", [True, False])
def test_rhs_block_sweeps_equal_solo_solves(bmg, precision, nbf, block, k, graph):
    """A batch of k right-hand sides of one operator whose one-pass sweeps
    take 2 or 4 members per warp (the stencil row read once for them; k not a
    multiple of the block, so the last warp group is padded): every member's
    iterate and history equal the hierarchy's own solve, and one member the
    oracle's refinement solve."""
    n = 511
    kind, planes, f = problem("lognormal", n)
    h = bmg.Hierarchy(kind, dev(planes), precision=precision, arith="fused")
    rhs = [dev(w.rhs_uniform(n, 600 + q)) for q in range(k)]
    B = bmg.Batch.from_hierarchy(h, k, use_graph=graph, rhs_block=block,
                                 smoother="auto" if graph else "tile0")
    xs, its, rrs, ok = B.solve(rhs, tol=1e-10, maxit=300)
    assert ok
    for q, r in enumerate(rhs):
        x, it, rr, okk = h.solve(r, tol=1e-10, maxit=300)
        assert okk and it == its[q] and torch.equal(x, xs[q]) and h.history() == B.history(q), q
    levels = bx.setup(kind, planes, arith="fused")
    xw, hw = mx.solve_ir(levels, mx.lower(levels, nbf), w.rhs_uniform(n, 603), tol=1e-10, maxit=300)
    assert np.array_equal(bx.at(host(xs[3]), 0, 0), bx.at(xw, 0, 0))
    check_history(B.history(3), hw)
    B.close()
    h.close()


def test_rhs_block_rejects_bad_value(bmg):
    kind, planes, f = problem("binary", 63)
    h = bmg.Hierarchy(kind, dev(planes), precision="fp32")
    with pytest.raises(KeyError):
        bmg.Batch.from_hierarchy(h, 2, rhs_block=3)
    import ctypes
    o = bmg._lib.Opts(bmg._lib._PREC["fp32"], 0, 0, 2, 1, 1, 0, 1, 0, None, None, 0, 0, 0, 3)
    b = ctypes.c_void_p()
    assert bmg.lib.bmg_batch_rhs(h._h, 2, ctypes.byref(o), ctypes.byref(b)) == bmg._lib.BMG_EINVAL
    h.close()
