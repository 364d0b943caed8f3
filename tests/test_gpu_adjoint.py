"""The discrete adjoint of the FP64 step (vlbm_grad_amplitudes) against the
reference adjoint of the oracle (oracle/vlbm_torch.py: torch.autograd of the
oracle's step, itself pinned to central differences of the C oracle) and
against central differences of the GPU's own FP64 path at the full
configuration (512 x 256, M = 16, 200 steps, checkpoints every 20) with the
Lax-Friedrichs limiter.  With R-theta the discrete derivatives grow without
bound within tens of steps (a property of the map, shared by the reference
adjoint, not of the adjoint code), so the full-size grid is checked against
the reference adjoint over a short window instead."""

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import vlbm_torch as T
from paper_2605_25282_gb300 import vlbm

pytestmark = pytest.mark.gpu


def gpu_grad(nx, ny, M, n, g, every, amp=None, limiter=2, seed=0):
    ens = vlbm.Ensemble([(nx, ny)], precision="fp64", relax=vlbm.RelaxParams(limiter=limiter))
    pert = vlbm.PerturbParams() if amp is None else vlbm.PerturbParams(amp=list(amp))
    ens.init(seed, M, pert)
    J, grad = ens.grad_amplitudes(n, vlbm.axial_weights(ny, nx, torch.from_numpy(g)), every)
    # the context is left at step n
    t, s = ens.time(0)
    assert np.all(s == n)
    ens.close()
    return J, grad


@pytest.mark.parametrize("limiter", [2, 0])
def test_adjoint_matches_oracle_autograd(limiter):
    nx, ny, M, n = 48, 24, 2, 10
    g = np.random.default_rng(1).uniform(0.5, 1.5, nx)
    J, grad = gpu_grad(nx, ny, M, n, g, every=4, limiter=limiter)
    jet, P = O.Jet(), O.Params(limiter=limiter)
    amp = torch.tensor(jet.amplitudes(), requires_grad=True)
    obs = T.axial_mean_density(O.Grid(nx, ny), P, jet, 0, M, n, amp)
    L = (torch.from_numpy(g) * obs).sum()
    L.backward()
    ref = amp.grad.numpy()
    assert abs(J - float(L.detach())) <= 1e-13 * abs(float(L.detach()))
    assert np.abs(grad - ref).max() <= 1e-9 * np.abs(ref).max(), (grad, ref)


def test_adjoint_checkpoint_interval_does_not_change_the_gradient():
    nx, ny, M, n = 64, 32, 3, 12
    g = np.ones(nx)
    a = gpu_grad(nx, ny, M, n, g, every=1)
    b = gpu_grad(nx, ny, M, n, g, every=5)
    c = gpu_grad(nx, ny, M, n, g, every=50)
    assert a[0] == b[0] == c[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[1], c[1])


def test_adjoint_zero_steps_is_the_initial_state():
    # after 0 steps only the inlet column carries the amplitudes; the axis rows
    # are ambient except in column 0
    nx, ny = 32, 16
    g = np.zeros(nx)
    g[0] = 1.0
    J, grad = gpu_grad(nx, ny, 2, 0, g, every=3)
    jet, P = O.Jet(), O.Params()
    amp = torch.tensor(jet.amplitudes(), requires_grad=True)
    obs = T.axial_mean_density(O.Grid(nx, ny), P, jet, 0, 2, 0, amp)
    (torch.from_numpy(g) * obs).sum().backward()
    assert np.abs(grad - amp.grad.numpy()).max() <= 1e-12 * np.abs(amp.grad.numpy()).max()


def test_adjoint_full_config_lax_friedrichs_matches_central_differences():
    # 512 x 256, M = 16, 200 steps, checkpoints every 20; 8 perturbed
    # amplitudes, a_9 and a_10 held.  With the Lax-Friedrichs limiter the
    # discrete map is smooth but for the argmax of lambda, and the adjoint of
    # the full window equals central differences.
    nx, ny, M, n = 512, 256, 16, 200
    g = np.ones(nx)
    amp0 = O.Jet().amplitudes().copy()
    J0, grad = gpu_grad(nx, ny, M, n, g, every=20, amp=amp0, limiter=0)
    h = 1e-6
    fd = []
    for k in range(8):
        ap, am = amp0.copy(), amp0.copy()
        ap[k] += h
        am[k] -= h
        fd.append((axial_j(nx, ny, M, n, ap, g, 0) - axial_j(nx, ny, M, n, am, g, 0)) / (2 * h))
    fd = np.array(fd)
    print("adjoint", grad[:8], "\nFD     ", fd)
    assert np.abs(grad[:8] - fd).max() <= 1e-5 * np.abs(fd).max(), (grad[:8], fd)


@pytest.mark.parametrize("n,every", [(3, 2), (20, 5)])
def test_adjoint_full_grid_r_theta_matches_reference_adjoint(n, every):
    # With R-theta the map's derivatives grow without bound at the limiter's
    # kinks within tens of steps (central differences stop meaning the
    # derivative), so the full-size grid is checked against the reference
    # adjoint itself: 512 x 256, M = 2, over 3 steps and over the first
    # checkpoint window of the configuration (20 steps, checkpoints every 5).
    nx, ny, M = 512, 256, 2
    g = np.linspace(0.5, 1.5, nx)
    amp0 = O.Jet().amplitudes().copy()
    J, grad = gpu_grad(nx, ny, M, n, g, every=every, amp=amp0)
    amp = torch.tensor(amp0, requires_grad=True)
    obs = T.axial_mean_density(O.Grid(nx, ny), O.Params(), O.Jet(), 0, M, n, amp)
    (torch.from_numpy(g) * obs).sum().backward()
    ref = amp.grad.numpy()
    assert np.abs(grad - ref).max() <= 1e-9 * np.abs(ref).max(), (grad, ref)


def axial_j(nx, ny, M, n, amp, g, limiter=2):
    ens = vlbm.Ensemble([(nx, ny)], precision="fp64", relax=vlbm.RelaxParams(limiter=limiter))
    ens.init(0, M, vlbm.PerturbParams(amp=list(amp)))
    ens.step(n)
    rho = ens.density(0, f32=False)
    ax = 0.5 * (rho[:, ny // 2 - 1] + rho[:, ny // 2]).mean(0)
    J = float((ax.cpu() * torch.from_numpy(g)).sum())
    ens.close()
    return J


def test_autograd_function_backward_equals_adjoint():
    nx, ny, M, n = 48, 24, 2, 8
    amp = torch.tensor(O.Jet().amplitudes(), requires_grad=True)
    ax = vlbm.AxialMeanDensity.apply(amp, (nx, ny), M, n, 0, 4)
    gvec = torch.linspace(0.5, 1.5, nx, dtype=torch.float64)
    (ax.cpu() * gvec).sum().backward()
    _, grad = gpu_grad(nx, ny, M, n, gvec.numpy(), every=4, amp=amp.detach().numpy())
    assert np.array_equal(amp.grad.numpy(), grad)
