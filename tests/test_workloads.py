"""The seeded input recipe held to its stated definitions: uniform and normal
draws against their distributions, right-hand sides with a zero ghost ring,
binary-contrast tiles (two values, constant per tile, Bernoulli fraction),
Gaussian random fields (exact sample std, Gaussian covariance
exp(-r^2 / (2 l^2)) at lags l and 2 l), the batched size mix (uniform over
the five sides, expected sum of n^2 = 256 x 278 554.6), and the batched
problems' per-problem seeds.  Tolerances are several standard errors of the
sample statistic, so the pins hold the recipe, not one realisation."""
import math

import numpy as np
import pytest
from scipy import stats

import workloads as w


def test_uniform_draws_fill_their_intervals_evenly():
    N = 200_000
    u = w.uniform01(17, N)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) <= 5 * math.sqrt(1 / 12 / N)
    assert abs(u.var() - 1 / 12) <= 5 * math.sqrt(1 / 180 / N)   # Var of (U - 1/2)^2 is 1/180
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    v = w.uniform_pm1(18, N)
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) <= 5 * math.sqrt(1 / 3 / N)


def test_normal_draws_are_standard_normal():
    N = 200_001                                   # odd: the last Box-Muller pair is cut
    z = w.normal(19, N)
    assert z.shape == (N,) and np.all(np.isfinite(z))
    assert abs(z.mean()) <= 5 / math.sqrt(N)
    assert abs(z.var() - 1.0) <= 5 * math.sqrt(2 / N)
    tail = np.mean(np.abs(z) > 2.0)
    p = math.erfc(2 / math.sqrt(2))               # P(|Z| > 2)
    assert abs(tail - p) <= 5 * math.sqrt(p * (1 - p) / N)
    assert stats.kstest(z, "norm").pvalue > 1e-4


@pytest.mark.parametrize("nx,ny", [(31, 31), (40, 23)])
def test_rhs_has_zero_ghost_ring_and_uniform_interior(nx, ny):
    f = w.rhs_uniform(nx, 5, ny if ny != nx else None)
    assert f.shape == (ny + 2, nx + 2)
    ring = np.ones_like(f, dtype=bool)
    ring[1:ny + 1, 1:nx + 1] = False
    assert np.all(f[ring] == 0.0)
    inner = f[1:ny + 1, 1:nx + 1]
    assert inner.min() >= -1.0 and inner.max() < 1.0 and np.unique(inner).size == inner.size


def test_binary_contrast_tiles():
    """2048^2 cells in 16^2 tiles (the 2047^2 workload): two values, constant
    per tile, the high value on a Bernoulli(1/2) fraction of the 128^2 tiles."""
    n, b = 2047, 16
    k = w.binary_blocks(n, b, 1.0, 1e4, 2)
    assert k.shape == (n + 1, n + 1)
    assert set(np.unique(k)) == {1.0, 1e4}
    tiles = k.reshape((n + 1) // b, b, (n + 1) // b, b)
    assert np.all(tiles == tiles[:, :1, :, :1])
    frac = np.mean(tiles[:, 0, :, 0] == 1e4)
    T = tiles.shape[0] * tiles.shape[2]
    assert abs(frac - 0.5) <= 5 * math.sqrt(0.25 / T)
    assert np.mean(w.binary_blocks(255, 8, 1.0, 1e6, 3, p=0.2) == 1e6) < 0.35


def test_gaussian_field_std_and_covariance():
    """Sample mean 0 and sample std exactly sigma; the correlation at lag l is
    exp(-1/2) and at lag 2 l exp(-2) (Gaussian covariance of length l),
    averaged over both axes and four seeds on 64 l x 64 l periodic grids."""
    cells, ell, sigma = 512, 8.0, 2.0
    c1, c2 = [], []
    for seed in (4, 5, 6, 7):
        g = w.gaussian_field(cells, sigma, ell, seed)
        assert abs(g.mean()) <= 1e-12 and abs(g.std() - sigma) <= 1e-12
        var = np.mean(g * g)
        for ax in (0, 1):
            c1.append(np.mean(g * np.roll(g, int(ell), axis=ax)) / var)
            c2.append(np.mean(g * np.roll(g, int(2 * ell), axis=ax)) / var)
    assert abs(np.mean(c1) - math.exp(-0.5)) <= 0.03
    assert abs(np.mean(c2) - math.exp(-2.0)) <= 0.03
    assert abs(np.mean(c1) - math.exp(-0.25)) > 0.1     # a field of length l / sqrt(2) would fail


def test_lognormal_coefficients_are_exp_of_the_field():
    k = w.lognormal_cells(255, 2.0, 32.0, 4)
    g = w.gaussian_field(256, 2.0, 32.0, 4)
    assert k.shape == (256, 256) and np.all(k > 0)
    assert np.array_equal(k, np.exp(g))
    assert abs(np.log(k).std() - 2.0) <= 1e-12


def test_batched_size_mix():
    """256 sides drawn uniformly from {63, 127, 255, 511, 1023}: each side's
    count within 4 binomial standard deviations of 256 / 5, and the sum of
    n^2 within 4 standard deviations of its expectation 256 x 278 554.6."""
    choices = (63, 127, 255, 511, 1023)
    sizes = w.batched_sizes(256, 5)
    assert len(sizes) == 256 and set(sizes) <= set(choices)
    sd = math.sqrt(256 * 0.2 * 0.8)
    for c in choices:
        assert abs(sizes.count(c) - 256 / 5) <= 4 * sd
    sq = np.array(choices, dtype=np.float64) ** 2
    mean, var = sq.mean(), sq.var()
    assert mean == 1_392_773 / 5                  # 278 554.6
    total = sum(n * n for n in sizes)
    assert abs(total - 256 * mean) <= 4 * math.sqrt(256 * var)
    assert w.batched_sizes(10, 5, first=7) == w.batched_sizes(17, 5)[7:]


def test_batched_problem_seeds():
    """Problem b of the batch takes coefficient seed 10000 + 2 b and
    right-hand-side seed 10001 + 2 b, whichever call returns it."""
    n = w.batched_sizes(1, 5, choices=(15, 31), first=3)[0]
    kind, planes, f = w.batched_problems(1, 5, choices=(15, 31), first=3)[0]
    assert kind == 9
    assert np.array_equal(planes, w.fe9_from_cells(w.lognormal_cells(n, 1.0, 32.0, 10006)))
    assert np.array_equal(f, w.rhs_uniform(n, 10007))
    whole = w.batched_problems(4, 5, choices=(15, 31))
    assert np.array_equal(whole[3][1], planes) and np.array_equal(whole[3][2], f)
