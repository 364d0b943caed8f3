"""Pins of the oracle's ensemble statistics (Sec. 3.2 restriction; Sec. 3.4,
Eqs. mean, std, w1cont, w1disc, w1cdf).

W1 is checked against two other definitions: the optimal-transport minimum over
all couplings (for equal-size empirical laws, over all permutations; brute force
on tiny M) and the CDF form int |F_1 - F_2| d xi, evaluated exactly for step
functions.  The mean and population std are checked on samples with known
moments; the restriction against conservation of the integral.
"""

import itertools

import numpy as np
import pytest

from oracle import oracle as O
from tests import inputs


def w1_permutations(a, b):
    M = len(a)
    return min(np.abs(a - b[list(p)]).sum() / M for p in itertools.permutations(range(M)))


def w1_cdf(a, b):
    xs = np.sort(np.concatenate([a, b]))
    Fa = np.searchsorted(np.sort(a), xs[:-1], side="right") / len(a)
    Fb = np.searchsorted(np.sort(b), xs[:-1], side="right") / len(b)
    return np.sum(np.abs(Fa - Fb) * np.diff(xs))


def test_w1_equals_optimal_transport_bruteforce():
    rng = np.random.default_rng(0)
    for M in (1, 2, 3, 5, 7):
        for _ in range(10):
            a = rng.standard_normal((M, 1, 1)) * 3
            b = rng.standard_normal((M, 1, 1)) + 1
            *_, w1 = O.ensemble_stats(a, b)
            assert abs(w1[0, 0] - w1_permutations(a[:, 0, 0], b[:, 0, 0])) < 1e-12


def test_w1_equals_cdf_integral_and_handles_ties():
    for dist in ("lognormal", "ties"):
        a = inputs.random_samples(1, 64, 3, 4, dist)
        b = inputs.random_samples(2, 64, 3, 4, dist)
        *_, w1 = O.ensemble_stats(a, b)
        for j in range(3):
            for i in range(4):
                assert abs(w1[j, i] - w1_cdf(a[:, j, i], b[:, j, i])) < 1e-12


def test_w1_equals_library_wasserstein_at_ensemble_size():
    # an independent implementation (scipy's CDF-based distance) at the
    # ensemble size of the batched runs, M = 1000
    stats = pytest.importorskip("scipy.stats")
    a = inputs.random_samples(11, 1000, 2, 3)
    b = inputs.random_samples(12, 1000, 2, 3)
    *_, w1 = O.ensemble_stats(a, b)
    for j in range(2):
        for i in range(3):
            want = stats.wasserstein_distance(a[:, j, i], b[:, j, i])
            assert abs(w1[j, i] - want) <= 1e-12 * max(1.0, abs(want))


def test_w1_metric_properties():
    a = inputs.random_samples(3, 50, 2, 2)
    b = inputs.random_samples(4, 50, 2, 2)
    *_, w_ab = O.ensemble_stats(a, b)
    *_, w_ba = O.ensemble_stats(b, a)
    *_, w_aa = O.ensemble_stats(a, a)
    assert np.array_equal(w_ab, w_ba)
    assert np.all(w_aa == 0)
    # a shift by c moves every order statistic by c: W1 = |c|
    *_, w_shift = O.ensemble_stats(a, a + 0.75)
    assert np.allclose(w_shift, 0.75, rtol=1e-13)
    # permuting realizations does not change any statistic
    perm = np.random.default_rng(5).permutation(50)
    s1 = O.ensemble_stats(a, b)
    s2 = O.ensemble_stats(a[perm], b)
    for x, y in zip(s1, s2):
        assert np.allclose(x, y, rtol=1e-14, atol=0)


def test_mean_and_population_std_closed_forms():
    # two-point law {c - s, c + s}, equal weights: mean c, population std s
    M = 10
    c, s = 5.0, 0.3
    a = np.zeros((M, 1, 1))
    a[::2] = c - s
    a[1::2] = c + s
    mean_a, std_a, mean_b, std_b, _ = O.ensemble_stats(a, a)
    assert abs(mean_a[0, 0] - c) < 1e-14 and abs(std_a[0, 0] - s) < 1e-14
    # 1/M normalisation (population variance), not 1/(M-1)
    x = np.array([1.0, 2.0, 3.0, 4.0]).reshape(4, 1, 1)
    _, sd, *_ = O.ensemble_stats(x, x)
    assert abs(sd[0, 0] - np.sqrt(1.25)) < 1e-15
    # a degenerate (Dirac) law has zero std and zero W1 to itself
    d = np.full((6, 2, 2), 3.25)
    _, sd, _, _, w = O.ensemble_stats(d, d)
    assert np.all(sd == 0) and np.all(w == 0)


def test_restriction_block_average_conserves_integral():
    rng = np.random.default_rng(7)
    fine = rng.uniform(0, 10, (3, 8, 12))
    for r in (1, 2, 4):
        co = O.restrict(fine, r)
        assert co.shape == (3, 8 // r, 12 // r)
        assert np.allclose(co.sum(axis=(1, 2)) * r * r, fine.sum(axis=(1, 2)), rtol=1e-14)
        assert co[1, 0, 0] == fine[1, :r, :r].sum() / (r * r)
    const = np.full((1, 8, 8), 2.5)
    assert np.all(O.restrict(const, 4) == 2.5)


def test_statistics_between_levels_restrict_first():
    a = inputs.random_samples(8, 20, 3, 5)
    fine = inputs.random_samples(9, 20, 6, 10)
    ma, sa, mb, sb, w1 = O.stats_w1_mean_std(a, fine)
    b = O.restrict(fine, 2)
    assert np.allclose(mb, b.mean(axis=0), rtol=1e-14)
    assert np.allclose(sb, b.std(axis=0), rtol=1e-13)
    assert np.allclose(w1, np.abs(np.sort(a, 0) - np.sort(b, 0)).mean(0), rtol=1e-14)


# --- two-point Wasserstein distance (Sec. 3.4, Eq. (w2)) ----------------------


def _brute_w1_2d(a, b):
    import itertools

    M = len(a)
    best = np.inf
    for perm in itertools.permutations(range(M)):
        best = min(best, sum(np.hypot(*(a[i] - b[perm[i]])) for i in range(M)))
    return best / M


@pytest.mark.parametrize("M", [1, 2, 3, 5, 6])
def test_w1_2d_equals_brute_force(M):
    rng = np.random.default_rng(M)
    a, b = rng.normal(size=(M, 2)), rng.normal(size=(M, 2))
    assert abs(O.w1_points_2d(a, b) - _brute_w1_2d(a, b)) <= 1e-14 * max(1.0, _brute_w1_2d(a, b))


def test_w1_2d_on_the_diagonal_is_sqrt2_times_sorted_1d():
    # points (s, s) and (t, t): distance sqrt(2)|s - t|, the sorted matching is optimal
    rng = np.random.default_rng(7)
    s, t = rng.lognormal(size=40), rng.lognormal(size=40)
    want = np.sqrt(2.0) * np.abs(np.sort(s) - np.sort(t)).mean()
    got = O.w1_points_2d(np.stack([s, s], 1), np.stack([t, t], 1))
    assert abs(got - want) <= 1e-12 * want


def test_w1_2d_of_a_translation_is_its_length():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(30, 2))
    c = np.array([0.3, -0.4])
    assert abs(O.w1_points_2d(a, a + c) - 0.5) <= 1e-12


def test_two_point_distance_structure():
    rng = np.random.default_rng(11)
    M, ny, nx, npd = 6, 8, 10, 3
    a = rng.lognormal(size=(M, ny, nx))
    w, pairs = O.w1_two_point(a, a, npd)
    assert w == 0.0 and pairs.shape == (npd ** 4,)
    pts = O.two_point_points(nx, ny, npd)
    assert pts[0] == (1, 1) and pts[-1] == (8, 6) and len(set(pts)) == npd * npd
    # a fine ensemble that restricts to a + 0.1 everywhere: every joint law is translated by (0.1, 0.1)
    fine = np.repeat(np.repeat(a + 0.1, 2, axis=1), 2, axis=2)
    w, pairs = O.w1_two_point(a, fine, npd)
    assert np.allclose(pairs, 0.1 * np.sqrt(2.0), rtol=1e-12)
    # diagonal pairs (k, k) reduce to sqrt(2) times the one-point W1 at that cell
    b = rng.lognormal(size=(M, ny, nx))
    w, pairs = O.w1_two_point(a, b, npd)
    for k, (i, j) in enumerate(pts):
        one = np.abs(np.sort(a[:, j, i]) - np.sort(b[:, j, i])).mean()
        assert abs(pairs[k * len(pts) + k] - np.sqrt(2.0) * one) <= 1e-12 * max(one, 1e-300)
