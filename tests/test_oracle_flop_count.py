"""The FP64 operation counter of the oracle (oracle/flop_count.cpp) runs the
oracle's own arithmetic: its counted step, compiled from the unchanged
oracle source with a counting stand-in for double, gives the plain oracle's
result bit for bit, so its counts are those of the oracle's step."""

import shutil

import pytest

from oracle import flop_count as FC
from oracle import oracle as O


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_counted_step_is_the_oracle_step():
    nx, ny, T = 40, 20, 5e-5
    (rec,) = FC.run(nx, ny, [T])
    grid, prm, jet = O.Grid(nx, ny), O.Params(), O.Jet()
    inl = O.inlet(grid, prm, jet, 0, 0)
    u, pops, _ = O.init_state(grid, prm, jet, inl)
    t = 0.0
    while t < T:
        a = max(O.kinetic_speed(grid, prm, u), grid.dx / (T - t))
        landing = t + grid.dx / a >= T * (1.0 - 1e-15)
        u, pops, _ = O.step(grid, prm, a, u, pops, inl)
        t = T if landing else t + grid.dx / a
    un, _, _ = O.step(grid, prm, O.kinetic_speed(grid, prm, u), u, pops, inl)
    check = 0.0
    for v in un.ravel():  # storage order, like the counter
        check += float(v)
    assert rec["check"] == check
    # every cell-update is hundreds of operations; divisions and square roots are few
    assert 500 < rec["arith"] < 2000 and rec["div"] < 100 and rec["sqrt"] < 3
