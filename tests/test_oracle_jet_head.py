"""Loose physics pin of the oracle: where the Mach 2000 jet's head is at the
paper's final time, on the paper's own domain [0, 2.5] x [-1, 1].

The paper states a head speed of about 666.7 from tracking the primary bow
shock (Sec. 2.2) and the head's leading fringe near x = 2.27 at t = 0.0035
(Sec. 4) (`tests/golden/jet_head.txt`).  The head position depends on the
limiter (a reading here) and on the grid's numerical diffusion, so this pin
is loose: the oracle's bow shock at t = 0.0035 on 250 x 200 must lie within
10 % of v_head t, behind the paper's finest-grid fringe, and move forward
under refinement.  (Measured: 2.16 on 125 x 100, 2.21 on 250 x 200, 2.25 on
500 x 400.)  A dropped flux term, a wrong energy or a wrong inlet state moves
the head by far more than that.
"""

import os

import numpy as np

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "jet_head.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _bow_shock_at(nx, ny, t_end):
    """One realization (seed 0, m = 0) advanced to t_end with the landing rule;
    the bow shock is the largest x where the density on the axis (the mean of
    the two rows next to y = 0) exceeds the ambient density by 10 %."""
    grid = O.Grid(nx, ny, x_max=2.5, y_min=-1.0)
    prm, jet = O.Params(), O.Jet()
    inl = O.inlet(grid, prm, jet, 0, 0)
    u, pops, _ = O.init_state(grid, prm, jet, inl)
    t = 0.0
    while t < t_end:
        a = max(O.kinetic_speed(grid, prm, u), grid.dx / (t_end - t))
        landing = t + grid.dx / a >= t_end * (1.0 - 1e-15)
        u, pops, _ = O.step(grid, prm, a, u, pops, inl)
        t = t_end if landing else t + grid.dx / a
    axis = 0.5 * (u[0, ny // 2 - 1] + u[0, ny // 2])
    above = np.nonzero(axis > 1.1 * jet.rho_amb)[0]
    return above[-1] * grid.dx


def test_jet_head_at_the_final_time():
    g = _golden()
    x_coarse = _bow_shock_at(125, 100, g["t"])
    x_fine = _bow_shock_at(250, 200, g["t"])
    tracked = g["v_head"] * g["t"]
    assert abs(x_fine - tracked) <= 0.1 * tracked, (x_fine, tracked)
    assert x_fine <= g["x_fringe"] + 0.05, (x_fine, g["x_fringe"])
    assert x_coarse < x_fine, (x_coarse, x_fine)
