"""Exact solution of the 1-D Riemann problem for the ideal-gas Euler equations.

Written from the mathematics (two nonlinear waves separated by a contact; the
star pressure is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
Rankine-Hugoniot branch for p > p_K and the isentropic branch for p <= p_K).
Used only as an independent pin of the VLBM oracle (Sod shock tube).
"""

from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        sq = math.sqrt(A / (p + B))
        return (p - pk) * sq, sq * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    f = 2.0 * a / (gamma - 1.0) * ((p / pk) ** e - 1.0)
    df = 1.0 / (rho * a) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma):
    rl, ul, pl = left
    rr, ur, pr = right
    p = 0.5 * (pl + pr)
    for _ in range(200):
        fl, dfl = _f_and_df(p, rl, pl, gamma)
        fr, dfr = _f_and_df(p, rr, pr, gamma)
        g = fl + fr + (ur - ul)
        dp = g / (dfl + dfr)
        pn = max(p - dp, 1e-12)
        if abs(pn - p) <= 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, gamma)
    fr, _ = _f_and_df(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, gamma, xi):
    """Primitive state (rho, u, p) at similarity coordinate xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    al = math.sqrt(gamma * pl / rl)
    ar = math.sqrt(gamma * pr / rr)
    gm = (gamma - 1.0) / (gamma + 1.0)
    out = np.zeros((len(xi), 3))
    for n, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rls = rl * ((ps / pl + gm) / (gm * ps / pl + 1.0))
                sl = ul - al * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + (gamma - 1.0) / (2.0 * gamma))
                out[n] = (rl, ul, pl) if s < sl else (rls, us, ps)
            else:  # left rarefaction
                rls = rl * (ps / pl) ** (1.0 / gamma)
                als = al * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
                sh, st = ul - al, us - als
                if s < sh:
                    out[n] = (rl, ul, pl)
                elif s > st:
                    out[n] = (rls, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) + gm / al * (ul - s)
                    out[n] = (rl * c ** (2.0 / (gamma - 1.0)),
                              2.0 / (gamma + 1.0) * (al + (gamma - 1.0) / 2.0 * ul + s),
                              pl * c ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rrs = rr * ((ps / pr + gm) / (gm * ps / pr + 1.0))
                sr = ur + ar * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + (gamma - 1.0) / (2.0 * gamma))
                out[n] = (rr, ur, pr) if s > sr else (rrs, us, ps)
            else:  # right rarefaction
                rrs = rr * (ps / pr) ** (1.0 / gamma)
                ars = ar * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
                sh, st = ur + ar, us + ars
                if s > sh:
                    out[n] = (rr, ur, pr)
                elif s < st:
                    out[n] = (rrs, us, ps)
                else:
                    c = 2.0 / (gamma + 1.0) - gm / ar * (ur - s)
                    out[n] = (rr * c ** (2.0 / (gamma - 1.0)),
                              2.0 / (gamma + 1.0) * (-ar + (gamma - 1.0) / 2.0 * ur + s),
                              pr * c ** (2.0 * gamma / (gamma - 1.0)))
    return out
