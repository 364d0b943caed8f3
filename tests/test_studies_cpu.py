"""Host logic of the studies: the rate fit of Eq. (ratefit) and the C4/C3
bookkeeping that needs no GPU."""

import numpy as np

from paper_2605_25282_gb300 import studies


def test_rate_is_the_log_log_slope():
    h = np.array([5e-3, 2.5e-3, 1.25e-3])
    for r in (0.37, 0.77, 1.0, -1.09):
        assert abs(studies.rate(h, 3.0 * h ** r) - r) <= 1e-12


def test_rate_of_noisy_errors_is_the_least_squares_slope():
    h = np.array([5e-3, 2.5e-3, 1.25e-3])
    e = np.array([5.8e-3, 4.2e-3, 3.5e-3])
    slope = np.polyfit(np.log(h), np.log(e), 1)[0]
    assert abs(studies.rate(h, e) - slope) <= 1e-14


def test_rate_undefined_for_nonpositive_errors():
    assert studies.rate([1.0, 0.5], [0.0, 1.0]) is None
    assert studies.rate([1.0], [1.0]) is None


def test_ladders_are_the_configured_grids():
    assert studies.LADDER_PAPER == [(500, 400), (1000, 800), (2000, 1600), (4000, 3200)]
    assert studies.LADDER_C2[-1] == (5060, 2530)
    # the paper's grids have square cells on [0, 2.5] x [-1, 1]
    for nx, ny in studies.LADDER_PAPER:
        assert abs(2.5 / nx - 2.0 / ny) < 1e-15


def test_axial_profile_reads_the_head_and_the_axial_spread():
    # two axis rows of M realizations: jet density 5 +- 0.3 (population std)
    # upstream of x = 1.5, ambient 0.5 beyond; the head is the last x above 0.55
    import torch

    nx = 200  # four realizations (the signs below)
    x = np.arange(nx) * (2.5 / nx)
    base = np.where(x < 1.5, 5.0, 0.5)
    sign = np.array([1.0, -1.0, 1.0, -1.0])[:, None, None]
    rows = base[None, None, :] + 0.3 * sign * (x < 1.4)[None, None, :]
    axis = torch.tensor(np.repeat(rows, 2, axis=1), dtype=torch.float32)
    p = studies.axial_profile(axis)
    assert p["bow_shock_x"] == x[x < 1.5][-1]
    assert abs(p["axial_std_upstream_median"] - 0.3) < 1e-6
    assert abs(p["axial_std_peak"] - 0.3) < 1e-6 and p["axial_std_peak_x"] < 1.4
