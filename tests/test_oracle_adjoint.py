"""Pins of the reference adjoint (oracle/vlbm_torch.py).

The torch restatement of the jet step must compute what the C oracle computes
(forward parity), and its autograd gradient of an ensemble observable with
respect to the per-mode amplitudes of Eq. (karhunenExp) must equal central
finite differences of the C oracle itself.  Over a short window the
discrete map is smooth almost everywhere, so the two agree to the
finite-difference error.
"""

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import vlbm_torch as T


@pytest.mark.parametrize("limiter", [2, 0, 1])
def test_torch_restatement_equals_c_oracle(limiter):
    g, P, J = O.Grid(40, 20), O.Params(limiter=limiter), O.Jet()
    amp = torch.tensor(J.amplitudes())
    # the unlimited scheme (theta = 1) loses positivity on the jet after a few steps
    cases = ((0, 0), (1, 3), (2, 12)) if limiter != 1 else ((0, 0), (1, 1))
    for m, n in cases:
        ref = O.run_jet(g, P, J, 0, m, 1, n)["u"][0]
        got = T.run_jet(g, P, J, 0, m, n, amp).detach().numpy()
        assert np.allclose(got, ref, rtol=1e-13, atol=0.0), (m, n, np.abs(got - ref).max())


def _fd_axial(g, P, seed, M, n, amp0, w, h):
    def J(a):
        jet = O.Jet()
        jet.amp = a
        acc = 0.0
        for m in range(M):
            u = O.run_jet(g, P, jet, seed, m, 1, n, want_pops=False)["u"][0]
            acc = acc + 0.5 * (u[0, g.ny // 2 - 1] + u[0, g.ny // 2])
        return float((w * acc / M).sum())

    out = []
    for k in range(len(amp0)):
        ap, am = amp0.copy(), amp0.copy()
        ap[k] += h
        am[k] -= h
        out.append((J(ap) - J(am)) / (2 * h))
    return np.array(out)


def test_autograd_gradient_equals_central_differences_of_c_oracle():
    g, P, jet = O.Grid(48, 24), O.Params(), O.Jet()
    M, n = 2, 10
    w = np.random.default_rng(0).uniform(0.5, 1.5, g.nx)
    amp0 = jet.amplitudes().copy()
    amp = torch.tensor(amp0, requires_grad=True)
    obs = T.axial_mean_density(g, P, jet, 0, M, n, amp)
    (torch.from_numpy(w) * obs).sum().backward()
    fd = _fd_axial(g, P, 0, M, n, amp0, w, 1e-6)
    grad = amp.grad.numpy()
    assert np.abs(grad - fd).max() <= 1e-8 * np.abs(fd).max(), (grad, fd)
    # every mode moves the observable
    assert np.all(np.abs(fd) > 1e-3 * np.abs(fd).max())


def test_reference_adjoint_growth_with_and_without_the_limiter():
    # With theta = 0 the map is smooth (but for lambda's argmax): the adjoint
    # equals central differences over 120 steps.  With R-theta it does over
    # 20 steps; beyond a few tens of steps the exact derivative of the
    # piecewise-smooth map grows by orders of magnitude past any secant.
    g, jet = O.Grid(64, 32), O.Jet()
    w = np.ones(g.nx)
    amp0 = jet.amplitudes().copy()

    def adjoint(P, n):
        amp = torch.tensor(amp0, requires_grad=True)
        (torch.from_numpy(w) * T.axial_mean_density(g, P, jet, 0, 1, n, amp)).sum().backward()
        return amp.grad.numpy()[:2]

    def fd(P, n, h=1e-6):
        out = []
        for k in range(2):
            vals = []
            for s in (1, -1):
                a = amp0.copy()
                a[k] += s * h
                j = O.Jet()
                j.amp = a
                u = O.run_jet(g, P, j, 0, 0, 1, n, want_pops=False)["u"][0]
                vals.append(float((w * 0.5 * (u[0, g.ny // 2 - 1] + u[0, g.ny // 2])).sum()))
            out.append((vals[0] - vals[1]) / (2 * h))
        return np.array(out)

    lf = O.Params(limiter=0)
    assert np.allclose(adjoint(lf, 120), fd(lf, 120), rtol=1e-6)
    rt = O.Params()
    assert np.allclose(adjoint(rt, 20), fd(rt, 20), rtol=1e-6)
    assert np.abs(adjoint(rt, 80)).max() > 1e3 * np.abs(fd(rt, 80)).max()
