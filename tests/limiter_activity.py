"""How much work the R-theta limiter's general case is on the jet: an analysis
of the oracle's state (not a test; run it as a script).

One realization of the jet on one level is advanced by the oracle to a time t
(landing rule).  For every interior side of every face, the script evaluates
the limiter's theta = 1 test (Sec. 2.1, the convex split V = U_LF + 4 s d_f
inside the relaxed density bounds and with non-negative q(1)) from the
oracle's conserved state and raw populations, and reports:
  - the fraction of interior sides whose theta = 1 test fails (they need the
    general case of the limiter);
  - of those, the fraction limited by the pressure quadratic (density-limited
    theta still leaves q < 0), i.e. that need the quadratic's root;
  - for the warp march of the mixed kernel (30 columns per warp, one row per
    march step, the north and east face of every lane), the share of lanes
    busy while a warp runs the general case, and the share of warp-face
    evaluations in which some lane needs the root.

    python tests/limiter_activity.py [nx ny t]     (default 400 200 0.002)
"""

from __future__ import annotations

import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import oracle as O  # noqa: E402

STRIP = 30  # columns updated per warp in the march


def advance(nx: int, ny: int, t_end: float):
    grid, prm, jet = O.Grid(nx, ny), O.Params(), O.Jet()
    inl = O.inlet(grid, prm, jet, 0, 0)
    u, pops, _ = O.init_state(grid, prm, jet, inl)
    t = 0.0
    while t < t_end:
        a = max(O.kinetic_speed(grid, prm, u), grid.dx / (t_end - t))
        landing = t + grid.dx / a >= t_end * (1.0 - 1e-15)
        u, pops, _ = O.step(grid, prm, a, u, pops, inl)
        t = t_end if landing else t + grid.dx / a
    return grid, prm, u, pops, O.kinetic_speed(grid, prm, u)


def euler_fluxes(q, gamma):
    r = q[..., 0]
    v1, v2 = q[..., 1] / r, q[..., 2] / r
    p = (gamma - 1.0) * (q[..., 3] - 0.5 * r * (v1 * v1 + v2 * v2))
    f = np.stack([q[..., 1], q[..., 1] * v1 + p, q[..., 1] * v2, (q[..., 3] + p) * v1], -1)
    g = np.stack([q[..., 2], q[..., 1] * v2, q[..., 2] * v2 + p, (q[..., 3] + p) * v2], -1)
    return f, g, p


def analyse(nx: int = 400, ny: int = 200, t_end: float = 0.002) -> dict:
    grid, prm, u, pops, a = advance(nx, ny, t_end)
    gamma = prm.gamma
    U = np.moveaxis(u, 0, -1)
    pk = [np.moveaxis(pops[4 * k:4 * k + 4], 0, -1) for k in range(4)]
    f, g, _ = euler_fluxes(U, gamma)
    h, c1 = 1.0 / (2.0 * a), (1.0 - prm.alpha) / 4.0
    M = [c1 * U + h * f, c1 * U - h * f, c1 * U + h * g, c1 * U - h * g]  # Eqs. (maxwellians12), (maxwellians34)
    neq = [M[k] - pk[k] for k in range(4)]  # M_k(u) - u_k
    interior = np.zeros((ny, nx), bool)
    interior[1:-1, 1:-1] = True
    ULF = np.ones_like(U)
    ULF[1:-1, 1:-1] = M[0][1:-1, :-2] + M[1][1:-1, 2:] + M[2][:-2, 1:-1] + M[3][2:, 1:-1]
    rho = U[..., 0]
    st = np.stack([rho[1:-1, 1:-1], rho[1:-1, :-2], rho[1:-1, 2:], rho[:-2, 1:-1], rho[2:, 1:-1],
                   ULF[1:-1, 1:-1, 0]])
    lo, hi = np.ones_like(rho), np.ones_like(rho)
    lo[1:-1, 1:-1], hi[1:-1, 1:-1] = st.min(0), st.max(0)
    delta = prm.rlmp_rel * (hi - lo) + prm.rlmp_abs
    _, _, p_lf = euler_fluxes(ULF, gamma)
    eps_r, eps_p = np.minimum(prm.eps_pos, ULF[..., 0]), np.minimum(prm.eps_pos, p_lf)
    lower, upper = np.maximum(eps_r, lo - delta), hi + delta
    kk = eps_p / (gamma - 1.0)

    def q_of(V0, D, th, j, i):
        r0, dr = V0[..., 0], D[..., 0]
        C = r0 * V0[..., 3] - 0.5 * (V0[..., 1] ** 2 + V0[..., 2] ** 2) - kk[j, i] * r0
        B = r0 * D[..., 3] + dr * V0[..., 3] - (V0[..., 1] * D[..., 1] + V0[..., 2] * D[..., 2]) - kk[j, i] * dr
        A = dr * D[..., 3] - 0.5 * (D[..., 1] ** 2 + D[..., 2] ** 2)
        return C + th * (B + th * A)

    def side(V0, D, j, i):
        """(theta = 1 fails, the density-limited theta leaves q < 0)"""
        vx = V0[..., 0] + D[..., 0]
        fail1 = (vx < lower[j, i]) | (vx > upper[j, i]) | (q_of(V0, D, 1.0, j, i) < 0)
        below, above = vx < lower[j, i], vx > upper[j, i]
        th = np.ones_like(vx)
        th = np.where(below, (V0[..., 0] - lower[j, i]) / np.where(below, -D[..., 0], 1.0), th)
        th = np.where(above, (upper[j, i] - V0[..., 0]) / np.where(above, D[..., 0], 1.0), th)
        th = np.clip(th, 0.0, 1.0)
        return fail1, fail1 & (q_of(V0, D, th, j, i) < 0)

    out = {"nx": nx, "ny": ny, "t": t_end, "sides": 0, "general": 0, "root": 0,
           "warp_lane_passes": 0, "warp_passes": 0, "warp_faces": 0, "warp_faces_root": 0}
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for axis, (kout, kin) in ((0, (0, 1)), (1, (2, 3))):
        sl_L = (slice(None), slice(0, -1)) if axis == 0 else (slice(0, -1), slice(None))
        sl_R = (slice(None), slice(1, None)) if axis == 0 else (slice(1, None), slice(None))
        d = neq[kout][sl_L] - neq[kin][sl_R]  # d_f = [M_out(u_L) - u_out,L] - [M_in(u_R) - u_in,R]
        JL, IL, JR, IR = J[sl_L], I[sl_L], J[sl_R], I[sl_R]
        inL, inR = interior[JL, IL], interior[JR, IR]
        gL, rL = side(ULF[JL, IL], -4.0 * d, JL, IL)
        gR, rR = side(ULF[JR, IR], 4.0 * d, JR, IR)
        gL, rL, gR, rR = gL & inL, rL & inL, gR & inR, rR & inR
        out["sides"] += int(inL.sum() + inR.sum())
        out["general"] += int(gL.sum() + gR.sum())
        out["root"] += int(rL.sum() + rR.sum())
        passes = gL.astype(int) + gR.astype(int)
        root = rL | rR
        for q in range(1, min(ny - 1, passes.shape[0])):
            for s0 in range(1, nx - 1, STRIP):
                seg = slice(s0, min(s0 + STRIP, nx - 1))
                out["warp_lane_passes"] += int(passes[q, seg].sum())
                out["warp_passes"] += int(passes[q, seg].max())
                out["warp_faces"] += 1
                out["warp_faces_root"] += int(root[q, seg].any())
    out["general_frac"] = out["general"] / out["sides"]
    out["root_frac_of_general"] = out["root"] / max(1, out["general"])
    out["lane_efficiency"] = out["warp_lane_passes"] / max(1, 32 * out["warp_passes"])
    out["warp_faces_root_frac"] = out["warp_faces_root"] / out["warp_faces"]
    return out


if __name__ == "__main__":
    args = sys.argv[1:]
    nx, ny, t = (int(args[0]), int(args[1]), float(args[2])) if len(args) == 3 else (400, 200, 0.002)
    r = analyse(nx, ny, t)
    print(f"{nx}x{ny}, t = {t}: theta = 1 fails at {100 * r['general_frac']:.1f} % of interior sides; "
          f"{100 * r['root_frac_of_general']:.1f} % of those need the pressure root; lanes busy in a warp's "
          f"general-case pass {100 * r['lane_efficiency']:.1f} %; warp-face evaluations with a root "
          f"{100 * r['warp_faces_root_frac']:.1f} %")
