"""Pins of the oracle's jet boundaries (Sec. 2.2, Eqs. (inletBC), (outletBC),
(transverseBC)) on a rough, non-uniform state.

After one step of the jet problem the new level must satisfy, by the paper's
rules and the reading of their order (inlet column Dirichlet; outlet column
and then the first and last rows copy the nearest interior node):
  - inlet column i = 0, every row (corners included): the inlet datum, with
    the equilibrium populations M_k of that datum at the step's kinetic speed;
  - outlet column i = nx - 1, rows 1 .. ny - 2: the state of column nx - 2 of
    the same row;
  - rows j = 0 and ny - 1, columns 1 .. nx - 1: the state of rows 1 and
    ny - 2 of the same column, so the outlet corners carry the diagonal
    interior nodes (nx - 2, 1) and (nx - 2, ny - 2);
  - every boundary node carries the equilibria of its own new state;
  - the interior update does not read the populations stored on boundary
    nodes (their equilibria stand in for them).
The state is rough in every row and column, so a copy from the wrong row or
column (rows 2 / ny - 3, column nx - 3) fails the equalities below.
"""

import numpy as np

from oracle import oracle as O
from tests import inputs

NX, NY = 23, 13
GAMMA = 5.0 / 3.0


def euler_flux(u, gamma=GAMMA):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (gamma - 1) * (E - 0.5 * rho * (v1 ** 2 + v2 ** 2))
    f = np.stack([m1, m1 * v1 + p, m1 * v2, (E + p) * v1])
    g = np.stack([m2, m1 * v2, m2 * v2 + p, (E + p) * v2])
    return f, g


def equilibria(u, a, alpha=0.0):
    """M_1..M_4 of Eqs. (maxwellians12), (maxwellians34): c1 u +- f / 2a, c1 u +- g / 2a."""
    f, g = euler_flux(u)
    c1 = (1.0 - alpha) / 4.0
    return np.concatenate([c1 * u + f / (2 * a), c1 * u - f / (2 * a), c1 * u + g / (2 * a), c1 * u - g / (2 * a)])


def setup(limiter=2, seed=3):
    grid = O.Grid(NX, NY)
    params = O.Params(limiter=limiter, bc=O.BC_JET)
    u, pops = inputs.random_state(seed, NX, NY, rough=0.3)
    inl = inputs.random_state(seed + 100, 1, NY, rough=0.3)[0][:, :, 0]  # any admissible column [4, ny]
    a = 3.0 * O.kinetic_speed(grid, params, u)
    return grid, params, u, pops, inl, a


def test_rough_state_distinguishes_rows_and_columns():
    grid, params, u, pops, inl, a = setup()
    un, _, _ = O.step(grid, params, a, u, pops, inl)
    assert np.abs(un[:, 1, 1:] - un[:, 2, 1:]).min() > 0
    assert np.abs(un[:, NY - 2, 1:] - un[:, NY - 3, 1:]).min() > 0
    assert np.abs(un[:, 1:-1, NX - 2] - un[:, 1:-1, NX - 3]).min() > 0


def test_inlet_column_is_dirichlet_with_equilibria():
    for limiter in (0, 2):
        grid, params, u, pops, inl, a = setup(limiter)
        un, pn, _ = O.step(grid, params, a, u, pops, inl)
        assert np.array_equal(un[:, :, 0], inl)
        assert np.allclose(pn[:, :, 0], equilibria(inl, a), rtol=1e-14, atol=1e-14 * np.abs(inl).max())


def test_outlet_column_copies_column_nx_minus_2():
    grid, params, u, pops, inl, a = setup()
    un, _, _ = O.step(grid, params, a, u, pops, inl)
    assert np.array_equal(un[:, 1:NY - 1, NX - 1], un[:, 1:NY - 1, NX - 2])


def test_first_and_last_rows_copy_their_neighbours_and_corners_are_diagonal():
    grid, params, u, pops, inl, a = setup()
    un, _, _ = O.step(grid, params, a, u, pops, inl)
    assert np.array_equal(un[:, 0, 1:NX - 1], un[:, 1, 1:NX - 1])
    assert np.array_equal(un[:, NY - 1, 1:NX - 1], un[:, NY - 2, 1:NX - 1])
    # outlet corners: the diagonal interior nodes (x copy first, then y)
    assert np.array_equal(un[:, 0, NX - 1], un[:, 1, NX - 2])
    assert np.array_equal(un[:, NY - 1, NX - 1], un[:, NY - 2, NX - 2])
    # inlet corners stay Dirichlet
    assert np.array_equal(un[:, 0, 0], inl[:, 0]) and np.array_equal(un[:, NY - 1, 0], inl[:, NY - 1])


def test_boundary_nodes_carry_equilibria_of_their_state():
    grid, params, u, pops, inl, a = setup()
    un, pn, _ = O.step(grid, params, a, u, pops, inl)
    mask = np.zeros((NY, NX), bool)
    mask[0, :] = mask[-1, :] = mask[:, 0] = mask[:, -1] = True
    eq = equilibria(un, a)
    scale = np.abs(un).max(axis=(1, 2))
    for c in range(16):
        err = np.abs(pn[c][mask] - eq[c][mask]).max()
        assert err <= 1e-13 * scale[c % 4], (c, err)


def test_interior_ignores_populations_stored_on_boundary_nodes():
    grid, params, u, pops, inl, a = setup()
    un, pn, _ = O.step(grid, params, a, u, pops, inl)
    rng = np.random.default_rng(7)
    pops2 = pops.copy()
    mask = np.zeros((NY, NX), bool)
    mask[0, :] = mask[-1, :] = mask[:, 0] = mask[:, -1] = True
    pops2[:, mask] *= 1.0 + 0.3 * rng.uniform(-1, 1, pops2[:, mask].shape)
    un2, pn2, _ = O.step(grid, params, a, u, pops2, inl)
    assert np.array_equal(un, un2) and np.array_equal(pn, pn2)
