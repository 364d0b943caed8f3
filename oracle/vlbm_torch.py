"""Differentiable FP64 CPU restatement of the jet step: the reference for the
gradients of ensemble observables with respect to the perturbation amplitudes.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import this module; the library never does.

It restates, with plain PyTorch CPU tensor operations, exactly what
vlbm_oracle.c computes for the jet (BC_JET): the KL inlet of Sec. 2.3,
Eq. (karhunenExp) with per-mode amplitudes, the initial state of Eq. (u0_def)
with equilibrium populations, the kinetic speed a_n = kappa 2 lambda / (1 - alpha)
(Sec. 2.1), the blended update of Eqs. (vlbm1)-(vlbm5) with the R-theta
limiter, and the boundaries (inlet Dirichlet, zero-gradient copies).  Every
branch of the C code is a torch.where on the same comparison in the same
order, so that torch.autograd gives the discrete adjoint of the oracle's
arithmetic: the argmax of lambda, the minima and maxima of the limiter and its
branches are differentiated as the piecewise-smooth functions they are, with
the branch the C code takes (first minimum / maximum in its scan order, tR on
a tie of theta_L and theta_R).  Denominators of branches that are not taken are
replaced by 1 so that no infinity enters the backward pass.

Layouts: u [4, ny, nx] conserved state, pops [16, ny, nx] (population k,
component c at 4 k + c), inlet [4, ny].
"""

from __future__ import annotations

import math

import torch

from . import oracle as O

DT = torch.float64


def _prim(q, gamma):
    v1 = q[1] / q[0]
    v2 = q[2] / q[0]
    p = (gamma - 1.0) * (q[3] - 0.5 * q[0] * (v1 * v1 + v2 * v2))
    return v1, v2, p


def _maxwellian(q, gamma, alpha, inv2a, k):
    """M_k(q; a), k = 0..3 (Eqs. (maxwellians12), (maxwellians34)); q [4, ...]."""
    v1, v2, p = _prim(q, gamma)
    if k < 2:
        F = (q[1], q[1] * v1 + p, q[1] * v2, (q[3] + p) * v1)
    else:
        F = (q[2], q[1] * v2, q[2] * v2 + p, (q[3] + p) * v2)
    c1 = (1.0 - alpha) / 4.0
    sgn = 1.0 if k % 2 == 0 else -1.0
    return torch.stack([c1 * q[c] + sgn * (F[c] * inv2a) for c in range(4)])


def kl_inlet(grid: O.Grid, jet: O.Jet, gamma: float, amp: torch.Tensor, Y, Z) -> torch.Tensor:
    """Inlet state per row [4, ny] (Eqs. (inletBC), (rho_inlet_def), (karhunenExp))."""
    ny = grid.ny
    pi = 3.14159265358979323846
    rows = []
    for j in range(ny):
        y = grid.y0 + (j + 0.5) * grid.dx
        if abs(y) <= jet.r_jet:
            yb = y / jet.r_jet
            s = torch.zeros((), dtype=DT)
            for k in range(1, jet.K + 1):
                arg = k * pi * yb
                s = s + amp[k - 1] * (Y[k - 1] * math.cos(arg) + Z[k - 1] * math.sin(arg))
            cw = math.cos(0.5 * pi * yb)
            rho = jet.rho_jet * (1.0 + s * (cw * cw))
            v1 = jet.v_jet
        else:
            rho = torch.tensor(jet.rho_amb, dtype=DT)
            v1 = 0.0
        q = torch.stack([rho * 1.0, rho * v1, rho * 0.0,
                         jet.p_amb / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + 0.0 * 0.0)])
        rows.append(q)
    return torch.stack(rows, 1)


def kinetic_speed(params: O.Params, u: torch.Tensor) -> torch.Tensor:
    """a_n = kappa 2 lambda / (1 - alpha); lambda at the first maximum in row-major order."""
    v1, v2, p = _prim(u, params.gamma)
    c = torch.sqrt(params.gamma * p / u[0])
    a1, a2 = v1.abs(), v2.abs()
    l = torch.where(a1 > a2, a1, a2) + c
    flat = l.reshape(-1)
    lam = flat[torch.argmax(flat)]
    return params.kappa * 2.0 * lam / (1.0 - params.alpha)


def init_state(params: O.Params, grid: O.Grid, jet: O.Jet, inlet: torch.Tensor):
    ny, nx = grid.ny, grid.nx
    qa = torch.tensor([jet.rho_amb, 0.0, 0.0, jet.p_amb / (params.gamma - 1.0) + 0.5 * jet.rho_amb * 0.0],
                      dtype=DT)
    amb = qa.view(4, 1, 1).expand(4, ny, nx - 1)
    u = torch.cat([inlet.view(4, ny, 1), amb], 2)
    a = kinetic_speed(params, u)
    inv2a = 0.5 / a
    pops = torch.cat([_maxwellian(u, params.gamma, params.alpha, inv2a, k) for k in range(4)], 0)
    return u, pops, a


def theta_star(U0, D, lo_b, hi_b, eps_r, eps_p, gamma):
    """Vectorised R-theta limiter: the C branches as masks (tensors [4, ...] / [...])."""
    one = torch.ones_like(U0[0])
    th = one
    lower = torch.where(eps_r > lo_b, eps_r, lo_b)
    neg, pos = D[0] < 0.0, D[0] > 0.0
    lim_n = (U0[0] - lower) / torch.where(neg, -D[0], one)
    lim_p = (hi_b - U0[0]) / torch.where(pos, D[0], one)
    lim = torch.where(neg, lim_n, lim_p)
    th = torch.where((neg | pos) & (lim < th), lim, th)
    th = torch.where(th < 0.0, torch.zeros_like(th), th)
    kk = eps_p / (gamma - 1.0)
    C = U0[0] * U0[3] - 0.5 * (U0[1] * U0[1] + U0[2] * U0[2]) - kk * U0[0]
    B = U0[0] * D[3] + D[0] * U0[3] - (U0[1] * D[1] + U0[2] * D[2]) - kk * D[0]
    A = D[0] * D[3] - 0.5 * (D[1] * D[1] + D[2] * D[2])
    qth = C + th * (B + th * A)
    done_th = qth >= 0.0
    done_zero = (~done_th) & (C <= 0.0)
    # the root branch
    a0 = A == 0.0
    r_lin = -C / torch.where(a0 & (B != 0.0), B, one)
    disc = B * B - 4.0 * A * C
    disc = torch.where(disc < 0.0, torch.zeros_like(disc), disc)
    sq = torch.sqrt(torch.where(disc > 0.0, disc, one)) * (disc > 0.0)
    Q = -0.5 * (B + torch.where(B >= 0.0, sq, -sq))
    q0 = Q == 0.0
    r1 = Q / torch.where(a0, one, A)
    r2 = C / torch.where(q0, one, Q)
    r = -one
    r = torch.where(r1 > 0.0, r1, r)
    r = torch.where((r2 > 0.0) & ((r < 0.0) | (r2 < r)), r2, r)
    root_zero = (~a0) & (q0 | (r < 0.0))
    r = torch.where(a0, r_lin, r)
    r = torch.where(r > th, th, r)
    r = torch.where(r < 0.0, torch.zeros_like(r), r)
    zero = torch.zeros_like(th)
    out = torch.where(done_th, th, torch.where(done_zero | root_zero, zero, r))
    return out


def _interior_mask(ny, nx):
    m = torch.zeros((ny, nx), dtype=torch.bool)
    m[1:ny - 1, 1:nx - 1] = True
    return m


def step(params: O.Params, grid: O.Grid, a, inlet: torch.Tensor, u: torch.Tensor, pops: torch.Tensor):
    """One step of every node (the C oracle's orc_step for BC_JET)."""
    ny, nx = grid.ny, grid.nx
    gamma, alpha = params.gamma, params.alpha
    inv2a = 0.5 / a
    M = [_maxwellian(u, gamma, alpha, inv2a, k) for k in range(4)]  # [4, ny, nx] each
    inner = _interior_mask(ny, nx)
    bnd = ~inner
    # populations as read: boundary nodes carry their equilibria
    P = [torch.where(bnd, M[k], pops[4 * k: 4 * k + 4]) for k in range(4)]
    # Step 3: U_LF and the bounds of interior nodes (full-size arrays, used on the interior)
    sl = (slice(None), slice(1, ny - 1), slice(1, nx - 1))
    qc = u[sl]
    qW, qE = u[:, 1:ny - 1, 0:nx - 2], u[:, 1:ny - 1, 2:nx]
    qS, qN = u[:, 0:ny - 2, 1:nx - 1], u[:, 2:ny, 1:nx - 1]
    M1W, M2E = M[0][:, 1:ny - 1, 0:nx - 2], M[1][:, 1:ny - 1, 2:nx]
    M3S, M4N = M[2][:, 0:ny - 2, 1:nx - 1], M[3][:, 2:ny, 1:nx - 1]
    Ui = alpha * qc + M1W + M2E + M3S + M4N
    lo, hi = qc[0], qc[0]
    for r in (qW[0], qE[0], qS[0], qN[0], Ui[0]):
        lo = torch.where(r < lo, r, lo)
        hi = torch.where(r > hi, r, hi)
    delta = params.rlmp_rel * (hi - lo) + params.rlmp_abs
    _, _, pLF = _prim(Ui, gamma)
    eps = torch.full_like(lo, params.eps_pos)
    bi = torch.stack([lo - delta, hi + delta, torch.where(eps < Ui[0], eps, Ui[0]), torch.where(eps < pLF, eps, pLF)])
    # embed into full arrays; boundary entries are safe placeholders (never selected)
    Ufull = torch.cat([torch.ones(1, ny, nx, dtype=DT), torch.zeros(2, ny, nx, dtype=DT),
                       torch.ones(1, ny, nx, dtype=DT)], 0)
    Ufull = torch.where(inner.expand(4, ny, nx), _pad(Ui, ny, nx, 1.0), Ufull)
    Bfull = torch.where(inner.expand(4, ny, nx), _pad(bi, ny, nx, 1.0), torch.ones(4, ny, nx, dtype=DT))
    # Step 4: faces
    thx, thy = _faces(params, u, M, P, Ufull, Bfull, inner, 0), _faces(params, u, M, P, Ufull, Bfull, inner, 1)
    # Step 5: interior update
    th_w = thx[1:ny - 1, 0:nx - 2]
    th_e = thx[1:ny - 1, 1:nx - 1]
    th_s = thy[0:ny - 2, 1:nx - 1]
    th_n = thy[1:ny - 1, 1:nx - 1]
    p1W = P[0][:, 1:ny - 1, 0:nx - 2]
    p2E = P[1][:, 1:ny - 1, 2:nx]
    p3S = P[2][:, 0:ny - 2, 1:nx - 1]
    p4N = P[3][:, 2:ny, 1:nx - 1]
    Mc = [M[k][sl] for k in range(4)]
    pc = [pops[4 * k: 4 * k + 4][sl] for k in range(4)]
    n1 = M1W + th_w * (M1W - p1W)
    n2 = M2E + th_e * (M2E - p2E)
    n3 = M3S + th_s * (M3S - p3S)
    n4 = M4N + th_n * (M4N - p4N)
    un = (n1 + n2 + n3 + n4 + alpha * qc - th_w * (Mc[1] - pc[1]) - th_e * (Mc[0] - pc[0])
          - th_s * (Mc[3] - pc[3]) - th_n * (Mc[2] - pc[2]))
    # Step 6: boundaries
    u_new = _pad(un, ny, nx, 0.0)
    u_new = torch.cat([inlet.view(4, ny, 1), u_new[:, :, 1:]], 2)
    rows = u_new[:, 1:ny - 1]
    rows = torch.cat([rows[:, :, :nx - 1], rows[:, :, nx - 2:nx - 1]], 2)
    u_new = torch.cat([u_new[:, 0:1], rows, u_new[:, ny - 1:ny]], 1)
    top = torch.cat([u_new[:, 0:1, 0:1], u_new[:, 1:2, 1:]], 2)
    bot = torch.cat([u_new[:, ny - 1:ny, 0:1], u_new[:, ny - 2:ny - 1, 1:]], 2)
    u_new = torch.cat([top, u_new[:, 1:ny - 1], bot], 1)
    newpops = torch.cat([n1, n2, n3, n4], 0)
    Mn = torch.cat([_maxwellian(u_new, gamma, alpha, inv2a, k) for k in range(4)], 0)
    pops_new = torch.where(inner.expand(16, ny, nx), _pad(newpops, ny, nx, 0.0), Mn)
    return u_new, pops_new


def _pad(x, ny, nx, fill):
    """Interior block [C, ny-2, nx-2] -> full [C, ny, nx] with fill on the boundary ring."""
    C = x.shape[0]
    col = torch.full((C, ny - 2, 1), fill, dtype=DT)
    mid = torch.cat([col, x, col], 2)
    row = torch.full((C, 1, nx), fill, dtype=DT)
    return torch.cat([row, mid, row], 1)


def _faces(params, u, M, P, Ufull, Bfull, inner, direction):
    """theta_f of every face (i+1/2, j) (direction 0) or (i, j+1/2) (direction 1),
    stored at its left / lower node; zero where the face does not exist."""
    ny, nx = u.shape[1], u.shape[2]
    if direction == 0:
        L = (slice(None), slice(None), slice(0, nx - 1))
        R = (slice(None), slice(None), slice(1, nx))
        kout, kin = 0, 1
    else:
        L = (slice(None), slice(0, ny - 1), slice(None))
        R = (slice(None), slice(1, ny), slice(None))
        kout, kin = 2, 3
    Mo, Mi = M[kout][L], M[kin][R]
    pL, pR = P[kout][L], P[kin][R]
    d = (Mo - pL) - (Mi - pR)
    bL, bR = ~inner[L[1:]], ~inner[R[1:]]
    lim = params.limiter
    if lim == 0:
        th = torch.zeros_like(d[0])
    elif lim == 1:
        th = torch.where(bL & bR, torch.zeros_like(d[0]), torch.ones_like(d[0]))
    else:
        g = params.gamma
        BL, BR = Bfull[L], Bfull[R]
        tL = theta_star(Ufull[L], -4.0 * d, BL[0], BL[1], BL[2], BL[3], g)
        tR = theta_star(Ufull[R], 4.0 * d, BR[0], BR[1], BR[2], BR[3], g)
        one = torch.ones_like(tL)
        tL = torch.where(bL, one, tL)
        tR = torch.where(bR, one, tR)
        th = torch.where(tL < tR, tL, tR)
        th = torch.where(bL & bR, torch.zeros_like(th), th)
    if direction == 0:
        return torch.cat([th, torch.zeros(ny, 1, dtype=DT)], 1)
    return torch.cat([th, torch.zeros(1, nx, dtype=DT)], 0)


def run_jet(grid: O.Grid, params: O.Params, jet: O.Jet, seed: int, m: int, nsteps: int, amp: torch.Tensor):
    """Realization m after nsteps fixed steps; amp [K] are the per-mode amplitudes."""
    Y, Z = O.kl_coefficients(seed, m, jet.K)
    inlet = kl_inlet(grid, jet, params.gamma, amp, Y, Z)
    u, pops, _ = init_state(params, grid, jet, inlet)
    for _ in range(nsteps):
        a = kinetic_speed(params, u)
        u, pops = step(params, grid, a, inlet, u, pops)
    return u


def axial_mean_density(grid: O.Grid, params: O.Params, jet: O.Jet, seed: int, M: int, nsteps: int,
                       amp: torch.Tensor) -> torch.Tensor:
    """Ensemble mean over realizations 0..M-1 of the density on the jet axis
    (the mean of rows ny/2 - 1 and ny/2) after nsteps: a vector over x."""
    ny = grid.ny
    acc = None
    for m in range(M):
        u = run_jet(grid, params, jet, seed, m, nsteps, amp)
        ax = 0.5 * (u[0, ny // 2 - 1] + u[0, ny // 2])
        acc = ax if acc is None else acc + ax
    return acc / M
