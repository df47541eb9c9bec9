"""Pins of the oracle's fused-arithmetic mode (arith="fused").

The fused multiply-add primitive is checked against exact rational arithmetic
(Python's Fraction, rounded to nearest-even by hand), and each fused kernel of
the oracle against a point-by-point Python loop that takes the same terms in
the same order through that exact primitive.  The loops read the stencil
through the symmetric five-plane rule written out here, not through the
oracle's helpers.  The fused cycle is then held to the rounded one: the same
iteration counts, residual histories within 1e-12 of ||r_0||, and the same
solution pins (manufactured solution, dense direct solve)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as w
from oracle import boxmg as bx
from oracle import mixed as mx
from oracle.fused import fma


def round_binary(q: Fraction, mant_bits: int) -> float:
    """Nearest-even rounding of a rational to a binary format with mant_bits
    significand bits (normal range only)."""
    if q == 0:
        return 0.0
    sign = -1.0 if q < 0 else 1.0
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    while q >= Fraction(2) ** (e + 1):
        e += 1
    while q < Fraction(2) ** e:
        e -= 1
    scaled = q / Fraction(2) ** (e - (mant_bits - 1))          # in [2^(p-1), 2^p)
    m = round(scaled)                                          # ties to even
    return sign * math.ldexp(float(m), e - (mant_bits - 1))


def fma_exact64(a, b, c) -> float:
    return round_binary(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)), 53)


def fma_exact32(a, b, c) -> np.float32:
    return np.float32(round_binary(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)), 24))


# ---- the primitive ----------------------------------------------------------------------

def test_round_binary_agrees_with_float_conversion():
    rng = np.random.default_rng(0)
    for v in rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200):
        q = Fraction(float(v)) * Fraction(3, 7)
        assert round_binary(q, 53) == float(q)                 # CPython's int / int is correctly rounded


def test_fma64_is_one_rounding():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(400) * 10.0 ** rng.integers(-8, 8, 400)
    b = rng.standard_normal(400)
    c = np.concatenate([-(a[:200] * b[:200]), rng.standard_normal(200)])   # cancellation: the product's error
    got = fma(a, b, c)
    want = np.array([fma_exact64(x, y, z) for x, y, z in zip(a, b, c)])
    assert np.array_equal(got, want)
    assert not np.array_equal(got, a * b + c)                 # a rounded product would lose these bits
    t = np.array([1.0 + 2.0 ** -27])
    assert fma(t, t, np.array([-1.0]))[0] == 2.0 ** -26 + 2.0 ** -54


def test_fma32_is_one_rounding():
    rng = np.random.default_rng(2)
    a = (rng.standard_normal(400) * 10.0 ** rng.integers(-4, 4, 400)).astype(np.float32)
    b = rng.standard_normal(400).astype(np.float32)
    c = np.concatenate([-(a[:200] * b[:200]), rng.standard_normal(200).astype(np.float32)])
    got = fma(a, b, c)
    assert got.dtype == np.float32
    want = np.array([fma_exact32(x, y, z) for x, y, z in zip(a, b, c)], dtype=np.float32)
    assert np.array_equal(got, want)
    assert not np.array_equal(got, (a * b + c).astype(np.float32))


# ---- the fused kernels against point loops ---------------------------------------------

def coupling_at(planes, i, j, di, dj):
    """a(p, p + (di, dj)) at p = (i, j) from the stored planes O, W, S, SW, NW and
    symmetry: E(i,j) = W(i+1,j), N(i,j) = S(i,j+1), NE(i,j) = SW(i+1,j+1),
    SE(i,j) = NW(i+1,j-1)."""
    O, W, S, SW, NW = planes
    return {(0, 0): O[j, i], (-1, 0): W[j, i], (1, 0): W[j, i + 1], (0, -1): S[j, i], (0, 1): S[j + 1, i],
            (-1, -1): SW[j, i], (1, 1): SW[j + 1, i + 1], (-1, 1): NW[j, i], (1, -1): NW[j - 1, i + 1]}[(di, dj)]


NBR = ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, 1), (-1, 1), (1, -1))


def random_level(n, seed, dtype=np.float64):
    kind, planes, f = w.binary_contrast_problem(n, 1, seed_k=seed, seed_f=seed + 1)
    levels = bx.setup(kind, planes, arith="fused")
    rng = np.random.default_rng(seed)
    x = np.zeros((n + 2, n + 2))
    x[1:n + 1, 1:n + 1] = rng.standard_normal((n, n))
    lev = levels[0]
    return lev.planes.astype(dtype), lev.dinv.astype(dtype), f.astype(dtype), x.astype(dtype), lev.ci


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_fused_residual_is_the_point_loop(dtype):
    n = 7
    planes, _, f, x, _ = random_level(n, 11, dtype)
    fx = fma_exact64 if dtype == np.float64 else fma_exact32
    got = bx.residual(planes, x, f, fused=True)
    for j in range(1, n + 1):
        for i in range(1, n + 1):
            s = f[j, i]
            for di, dj in NBR:
                s = fx(-coupling_at(planes, i, j, di, dj), x[j + dj, i + di], s)
            assert got[j, i] == s, (i, j)
    assert not np.array_equal(got, bx.residual(planes, x, f))


def test_fused_apply_is_the_point_loop():
    n = 7
    planes, _, _, x, _ = random_level(n, 12)
    got = bx.apply(planes, x, fused=True)
    for j in range(1, n + 1):
        for i in range(1, n + 1):
            s = coupling_at(planes, i, j, 0, 0) * x[j, i]
            for di, dj in NBR[1:]:
                s = fma_exact64(coupling_at(planes, i, j, di, dj), x[j + dj, i + di], s)
            assert got[j, i] == s


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_fused_gauss_seidel_sweep_is_the_point_loop(dtype):
    n = 7
    planes, dinv, f, x, _ = random_level(n, 13, dtype)
    fx = fma_exact64 if dtype == np.float64 else fma_exact32
    got = x.copy()
    bx.gs_sweep(9, planes, dinv, got, f, fused=True)
    want = x.copy()
    for pi, pj in ((1, 1), (0, 1), (1, 0), (0, 0)):            # the four colours in order
        for j in range(1, n + 1):
            for i in range(1, n + 1):
                if i % 2 != pi or j % 2 != pj:
                    continue
                s = f[j, i]
                for di, dj in NBR[1:]:
                    s = fx(-coupling_at(planes, i, j, di, dj), want[j + dj, i + di], s)
                want[j, i] = s * dinv[j, i]
    assert np.array_equal(got, want)


def test_fused_restriction_and_interpolation_are_the_point_loops():
    n = 15
    nc = 7
    _, _, _, r, ci = random_level(n, 14)
    got = bx.restrict(ci, r, fused=True)
    LSW, LSE, LNW, LNE, LL, LR, LB, LA = range(8)
    for jc in range(1, nc + 1):
        for ic in range(1, nc + 1):
            I, J = 2 * ic, 2 * jc
            t = ci[LNE, jc, ic] * r[J - 1, I - 1]
            t = fma_exact64(ci[LA, jc, ic], r[J - 1, I], t)
            t = fma_exact64(ci[LNW, jc, ic + 1], r[J - 1, I + 1], t)
            t = fma_exact64(ci[LR, jc, ic], r[J, I - 1], t)
            t = t + r[J, I]
            t = fma_exact64(ci[LL, jc, ic + 1], r[J, I + 1], t)
            t = fma_exact64(ci[LSE, jc + 1, ic], r[J + 1, I - 1], t)
            t = fma_exact64(ci[LB, jc + 1, ic], r[J + 1, I], t)
            t = fma_exact64(ci[LSW, jc + 1, ic + 1], r[J + 1, I + 1], t)
            assert got[jc, ic] == t
    rng = np.random.default_rng(3)
    ec = np.zeros((nc + 2, nc + 2))
    ec[1:nc + 1, 1:nc + 1] = rng.standard_normal((nc, nc))
    x = r.copy()
    bx.interp_correct(ci, ec, x, fused=True)
    want = r.copy()
    for jc in range(1, nc + 2):
        for ic in range(1, nc + 2):
            I, J = 2 * ic, 2 * jc
            if ic <= nc and jc <= nc:
                want[J, I] = r[J, I] + ec[jc, ic]
            if jc <= nc:
                t = ci[LL, jc, ic] * ec[jc, ic - 1]
                want[J, I - 1] = r[J, I - 1] + fma_exact64(ci[LR, jc, ic], ec[jc, ic], t)
            if ic <= nc:
                t = ci[LB, jc, ic] * ec[jc - 1, ic]
                want[J - 1, I] = r[J - 1, I] + fma_exact64(ci[LA, jc, ic], ec[jc, ic], t)
            t = ci[LSW, jc, ic] * ec[jc - 1, ic - 1]
            t = fma_exact64(ci[LSE, jc, ic], ec[jc - 1, ic], t)
            t = fma_exact64(ci[LNW, jc, ic], ec[jc, ic - 1], t)
            t = fma_exact64(ci[LNE, jc, ic], ec[jc, ic], t)
            want[J - 1, I - 1] = r[J - 1, I - 1] + t
    assert np.array_equal(x, want)


# ---- the fused cycle against the rounded one -----------------------------------------------

def problem(name, n):
    if name == "poisson":
        return 5, w.poisson5(n), w.rhs_uniform(n, 1)
    return w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3)


@pytest.mark.parametrize("name", ["poisson", "fe_binary"])
@pytest.mark.parametrize("krylov", ["none", "fcg"])
def test_fused_history_tracks_the_rounded_one(name, krylov):
    n = 31
    kind, planes, f = problem(name, n)
    run = bx.solve if krylov == "none" else bx.solve_fcg
    _, hr = run(bx.setup(kind, planes), f, tol=1e-10, maxit=60)
    xf, hf = run(bx.setup(kind, planes, arith="fused"), f, tol=1e-10, maxit=60)
    assert len(hf) == len(hr)
    assert hf != hr                                           # the two modes do round differently
    assert max(abs(a - b) for a, b in zip(hf, hr)) <= 1e-12 * hr[0]
    assert hf[-1] / hf[0] <= 1e-10


def test_fused_cycle_solves_the_manufactured_problem():
    n = 31
    kind, planes, _ = w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3)
    levels = bx.setup(kind, planes, arith="fused")
    rng = np.random.default_rng(5)
    u = np.zeros((n + 2, n + 2))
    u[1:n + 1, 1:n + 1] = rng.standard_normal((n, n))
    f = bx.apply(levels[0].planes, u)
    x, h = bx.solve(levels, f, tol=1e-13, maxit=200)
    A = bx.dense_matrix(levels[0].planes)
    kappa = np.linalg.cond(A)
    err = np.linalg.norm(x[1:n + 1, 1:n + 1] - u[1:n + 1, 1:n + 1]) / np.linalg.norm(u[1:n + 1, 1:n + 1])
    assert err <= kappa * 1e-13 * 10


@pytest.mark.parametrize("n", [7, 15])
def test_fused_cycle_matches_dense_direct_solve(n):
    kind, planes, f = w.binary_contrast_problem(n, 4, seed_k=6, seed_f=7)
    levels = bx.setup(kind, planes, arith="fused")
    x, _ = bx.solve(levels, f, tol=1e-14, maxit=200)
    A = bx.dense_matrix(levels[0].planes)
    ref = np.linalg.solve(A, f[1:n + 1, 1:n + 1].reshape(-1)).reshape(n, n)
    assert np.allclose(x[1:n + 1, 1:n + 1], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("bf16", [0, 2])
def test_fused_refinement_reaches_fp64_accuracy(bf16):
    n = 31
    kind, planes, f = w.binary_contrast_problem(n, 4, seed_k=2, seed_f=3)
    levels = bx.setup(kind, planes, arith="fused")
    l32 = mx.lower(levels, bf16)
    assert all(lv.fused for lv in l32)
    x, h = mx.solve_ir(levels, l32, f, tol=1e-10, maxit=60)
    _, hr = mx.solve_ir(bx.setup(kind, planes), mx.lower(bx.setup(kind, planes), bf16), f, tol=1e-10, maxit=60)
    assert h[-1] / h[0] <= 1e-10
    assert abs(len(h) - len(hr)) <= 1
    r = bx.residual(levels[0].planes, x, f)
    assert bx.norm(r) / bx.norm(f) <= 1e-10
