"""Initialisation from given KL coefficients (vlbm_init_ensemble_samples).

The coefficients of realization m drawn by the oracle's Philox4x32-10
(Sec. 2.3, Eq. (karhunenExp)) reproduce the seeded initialisation bit for bit,
whether they come from pageable host memory, pinned host memory or the
device; other coefficients change the inlet as Eq. (rho_inlet_def) says.
"""

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_25282_gb300 import vlbm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

LEVELS = [(64, 32), (128, 64)]


def oracle_xi(seed, M, K=10):
    rows = []
    for m in range(M):
        Y, Z = O.kl_coefficients(seed, m, K)
        rows.append(np.concatenate([Y, Z]))
    return np.array(rows)


def states(ens):
    ens.sync()
    return [H.to_np(ens.get_state(l)[0]) for l in range(len(LEVELS))]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("where", ["numpy", "pinned", "device"])
def test_oracle_draws_reproduce_seeded_init(precision, where):
    seed, M = 7, 3
    a = vlbm.Ensemble(LEVELS, precision=precision)
    a.init(seed, M)
    xi = oracle_xi(seed, M)
    if where == "pinned":
        xi = torch.from_numpy(xi).pin_memory()
    elif where == "device":
        xi = torch.from_numpy(xi).cuda()
    b = vlbm.Ensemble(LEVELS, precision=precision)
    b.init_samples(xi)
    for sa, sb in zip(states(a), states(b)):
        assert np.array_equal(sa, sb)
    a.step(6)
    b.step(6)
    for sa, sb in zip(states(a), states(b)):
        assert np.array_equal(sa, sb)


def test_given_coefficients_set_the_inlet_density():
    # Y_1 = 1, everything else 0: rho = rho_jet (1 + A cos(pi ybar) W(ybar)) in the jet rows
    M, K = 2, 10
    xi = np.zeros((M, 2 * K))
    xi[0, 0] = 1.0
    ens = vlbm.Ensemble([(64, 32)], precision="fp64")
    ens.init_samples(xi)
    rho = H.to_np(ens.moments(0)["rho"])[:, :, 0]
    g = O.Grid(64, 32)
    jet = O.Jet()
    for j in range(32):
        y = g.y0 + (j + 0.5) * g.dx
        if abs(y) <= jet.r_jet:
            Y = np.zeros(K)
            Y[0] = 1.0
            want = O.kl_density(y / jet.r_jet, Y, np.zeros(K), jet)
            assert abs(rho[0, j] - want) <= 1e-14 * want
            assert rho[1, j] == jet.rho_jet
        else:
            assert rho[0, j] == jet.rho_amb and rho[1, j] == jet.rho_amb
