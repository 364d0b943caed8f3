"""Pins of the oracle's error functionals and diagnostics (Sec. 3.3-3.4,
Sec. 4.3): closed forms and inequalities the definitions imply."""

import numpy as np
from scipy import stats as sps

from oracle import oracle as O
from tests import inputs


def test_functionals_of_identical_and_shifted_ensembles():
    a = inputs.random_samples(1, 40, 6, 8)
    assert O.error_functionals(a, a) == (0.0, 0.0, 0.0, 0.0)
    em, es, w11, st = O.error_functionals(a, a + 0.25)
    assert abs(em - 0.25) < 1e-14 and abs(w11 - 0.25) < 1e-14 and es < 1e-14
    # b = (1 + e) a: the relative L1 distance of every realization is e / (1 + e)
    e = 0.1
    *_, st = O.error_functionals(a, (1 + e) * a)
    assert abs(st - e / (1 + e)) < 1e-14


def test_w1_bounds_the_mean_error_and_strong_error_bounds_w1():
    # |E a - E b| <= W1(a, b) per cell (coupling argument), hence E_mean <= W_11;
    # the identity coupling is one coupling, hence W1 <= mean |a_m - b_m|.
    a = inputs.random_samples(2, 50, 5, 5)
    b = inputs.random_samples(3, 50, 10, 10)
    em, es, w11, st = O.error_functionals(a, b)
    assert em <= w11 + 1e-15
    bb = O.restrict(b, 2)
    pathwise = np.abs(a - bb).mean(axis=0).mean()
    assert w11 <= pathwise + 1e-15


def test_restriction_applies_before_the_functionals():
    a = inputs.random_samples(4, 10, 3, 4)
    fine = np.repeat(np.repeat(a, 2, axis=1), 2, axis=2)  # exact refinement of a
    assert O.error_functionals(a, fine) == (0.0, 0.0, 0.0, 0.0)


def test_quantiles_width_ratio_gaussian():
    # Sec. 4.3: Q_N = (Phi^-1(0.95) - Phi^-1(0.05)) / (Phi^-1(0.84) - Phi^-1(0.16)) ~ 1.65
    qn = (sps.norm.ppf(0.95) - sps.norm.ppf(0.05)) / (sps.norm.ppf(0.84) - sps.norm.ppf(0.16))
    assert round(qn, 2) == 1.65
    rng = np.random.default_rng(0)
    s = 3.0 + 0.7 * rng.standard_normal((20000, 2, 2))
    q = O.width_ratio(s)
    assert np.all(np.abs(q - qn) < 0.03)
    # quantile definition: inf{xi : F(xi) >= alpha}
    x = np.array([4.0, 1.0, 3.0, 2.0]).reshape(4, 1)
    assert O.quantile(x, 0.25)[0] == 1.0 and O.quantile(x, 0.26)[0] == 2.0 and O.quantile(x, 1.0)[0] == 4.0


def test_histogram_is_a_density_per_cell():
    a = inputs.random_samples(5, 300, 2, 3)
    edges = np.linspace(0.0, 40.0, 81)
    h = O.histogram(a, edges)
    mass = (h * np.diff(edges)[:, None, None]).sum(axis=0)
    inside = ((a >= edges[0]) & (a < edges[-1])).mean(axis=0)
    assert np.allclose(mass, inside, rtol=1e-14)


def test_rate_fit_recovers_a_power_law():
    dx = np.array([5e-3, 2.5e-3, 1.25e-3])
    r, c = O.rate_fit(dx, 3.0 * dx ** 0.67)
    assert abs(r - 0.67) < 1e-12 and abs(np.exp(c) - 3.0) < 1e-10
