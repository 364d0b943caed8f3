"""Shared helpers of the GPU parity tests: oracle runs and the comparison norms.

Norms (the oracle is FP64; the paper fixes no precision):
  - conserved rho and E: |x_gpu - x_orc| <= rtol |x_orc| per cell;
  - momentum components: |m_gpu - m_orc| <= rtol sqrt(2 rho E) (|m| is bounded
    by sqrt(2 rho E) since the kinetic energy never exceeds E);
  - pressure: |p_gpu - p_orc| <= rtol (|p| + rho |v|^2 / 2): p = (gamma - 1)(E - K)
    is a difference of two numbers ~E, so 1 ulp of E is ~5e-10 p at Mach 2000;
  - populations: component c of every population scaled like component c of u.
"""

from __future__ import annotations

import numpy as np
import torch

from oracle import oracle as O
from paper_2605_25282_gb300 import vlbm


def oracle_params(limiter=2, alpha=0.0, kappa=1.0):
    return O.Params(gamma=5.0 / 3.0, alpha=alpha, kappa=kappa, limiter=limiter)


def relax(limiter=2, alpha=0.0, kappa=1.0):
    return vlbm.RelaxParams(alpha=alpha, kappa=kappa, limiter=limiter)


def cons_scales(u):
    rho, E = np.abs(u[..., 0, :, :]), np.abs(u[..., 3, :, :])
    ms = np.sqrt(2.0 * rho * E)
    return np.stack([rho, ms, ms, E], axis=-3)


def rel_err_cons(u_gpu, u_ref):
    return np.abs(u_gpu - u_ref) / cons_scales(u_ref)


def pressure(u, gamma=5.0 / 3.0):
    rho, m1, m2, E = (u[..., c, :, :] for c in range(4))
    v1, v2 = m1 / rho, m2 / rho
    K = 0.5 * rho * (v1 * v1 + v2 * v2)
    return (gamma - 1.0) * (E - K), K


def rel_err_pressure(u_gpu, u_ref, gamma=5.0 / 3.0):
    pg, _ = pressure(u_gpu, gamma)
    pr, K = pressure(u_ref, gamma)
    return np.abs(pg - pr) / (np.abs(pr) + K)


def rel_err_pops(p_gpu, p_ref, u_ref):
    s = cons_scales(u_ref)
    sc = np.concatenate([s, s, s, s], axis=-3)
    return np.abs(p_gpu - p_ref) / sc


def oracle_jet(nx, ny, M, nsteps, seed=0, limiter=2, t_end=None, m0=0):
    g = O.Grid(nx, ny)
    return O.run_jet(g, oracle_params(limiter), O.Jet(), seed, m0, M, nsteps, t_end=t_end)


def gpu_jet(levels, M, precision="fp64", limiter=2, seed=0):
    ens = vlbm.Ensemble(levels, precision=precision, relax=relax(limiter))
    ens.init(seed, M)
    return ens


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()
