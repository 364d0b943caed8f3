"""Plain FP64 CPU oracle of the probabilistic VLBM (ctypes wrapper + numpy statistics).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import this module.  It shares no
code with the CUDA library in ``paper_2605_25282_gb300``; the step itself lives in
``vlbm_oracle.c`` (plain C, FP64, built with ``-O2 -ffp-contract=off``).

Statistics follow the paper's Sec. 3.2 (restriction by block averaging onto the
coarse grid) and Sec. 3.4, Eqs. (mean), (std) (population variance, 1/M) and
(w1disc) (one-point W1 as the mean absolute difference of the ascending order
statistics).  Reading: each realization's fine field is restricted first, then
every statistic is taken on the common grid.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlbm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liborc.so")

BC_JET, BC_PERIODIC, BC_NEUMANN, BC_TUBE = 0, 1, 2, 3
ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ENONPOSITIVE, ORC_ENONFINITE = 0, 1, 2, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, no fast-math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("y_min", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("alpha", ctypes.c_double), ("kappa", ctypes.c_double),
                ("limiter", ctypes.c_int), ("rlmp_rel", ctypes.c_double),
                ("rlmp_abs", ctypes.c_double), ("eps_pos", ctypes.c_double), ("bc", ctypes.c_int)]


class _Prim(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("v1", ctypes.c_double), ("v2", ctypes.c_double),
                ("p", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.orc_philox4x32_10.argtypes = [p, p, p]
        _lib.orc_kl_coefficients.argtypes = [ctypes.c_uint64, i, i, p, p]
        _lib.orc_kl_density.argtypes = [d, d, i, p, p, p]
        _lib.orc_kl_density.restype = d
        _lib.orc_inlet.argtypes = [p, d, p, p, d, i, p, ctypes.c_uint64, i, p]
        _lib.orc_kinetic_speed.argtypes = [p, p, p, p]
        _lib.orc_init_state.argtypes = [p, p, p, p, p, p, p]
        _lib.orc_step.argtypes = [p, p, d, p, p, p, p, p]
        _lib.orc_moments.argtypes = [p, d, p, p, p, p, p]
        _lib.orc_run_jet.argtypes = [p, p, p, p, d, i, p, ctypes.c_uint64, i, i, i, d, p, p, p, p]
        _lib.orc_theta_star_export.argtypes = [p, p, d, d, d, d, d]
        _lib.orc_theta_star_export.restype = d
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------- #
# Problem description (Sec. 2.2 constants by default).                         #
# --------------------------------------------------------------------------- #


@dataclass
class Grid:
    nx: int
    ny: int
    x_max: float = 2.5
    y_min: float | None = None  # default: centred, y in [-ny dx / 2, ny dx / 2]
    cell: float | None = None  # explicit cell size (a sub-domain of a larger grid)

    @property
    def dx(self) -> float:
        return self.x_max / self.nx if self.cell is None else self.cell

    @property
    def y0(self) -> float:
        return -0.5 * self.ny * self.dx if self.y_min is None else self.y_min

    def c(self):
        return _Grid(self.nx, self.ny, self.dx, self.y0)


@dataclass
class Params:
    gamma: float = 5.0 / 3.0
    alpha: float = 0.0
    kappa: float = 1.0
    limiter: int = 2
    rlmp_rel: float = 0.1
    rlmp_abs: float = 0.0
    eps_pos: float = 1e-13
    bc: int = BC_JET

    def c(self):
        return _Params(self.gamma, self.alpha, self.kappa, self.limiter, self.rlmp_rel, self.rlmp_abs,
                       self.eps_pos, self.bc)


@dataclass
class Jet:
    rho_jet: float = 5.0
    v_jet: float = 800.0
    p_amb: float = 0.4127
    rho_amb: float = 0.5
    r_jet: float = 0.05
    A: float = 0.1
    p_decay: float = 2.0
    K: int = 10
    amp: np.ndarray | None = None  # per-mode amplitudes; default A k^-p

    def amplitudes(self) -> np.ndarray:
        if self.amp is not None:
            return np.ascontiguousarray(self.amp, dtype=np.float64)
        k = np.arange(1, self.K + 1, dtype=np.float64)
        return self.A * k ** (-self.p_decay)


# --------------------------------------------------------------------------- #
# Thin wrappers.                                                              #
# --------------------------------------------------------------------------- #


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def kl_coefficients(seed: int, m: int, K: int = 10):
    Y = np.zeros(K)
    Z = np.zeros(K)
    lib().orc_kl_coefficients(ctypes.c_uint64(seed), m, K, _ptr(Y), _ptr(Z))
    return Y, Z


def kl_density(ybar: float, Y, Z, jet: Jet = Jet()) -> float:
    amp = jet.amplitudes()
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    return lib().orc_kl_density(float(ybar), jet.rho_jet, jet.K, _ptr(amp), _ptr(Y), _ptr(Z))


def _prims(jet: Jet):
    return (_Prim(jet.rho_jet, jet.v_jet, 0.0, jet.p_amb), _Prim(jet.rho_amb, 0.0, 0.0, jet.p_amb))


def inlet(grid: Grid, params: Params, jet: Jet, seed: int, m: int) -> np.ndarray:
    out = np.zeros((4, grid.ny))
    pj, pa = _prims(jet)
    amp = jet.amplitudes()
    g = grid.c()
    st = lib().orc_inlet(ctypes.byref(g), params.gamma, ctypes.byref(pj), ctypes.byref(pa), jet.r_jet,
                         jet.K, _ptr(amp), ctypes.c_uint64(seed), m, _ptr(out))
    if st:
        raise RuntimeError(f"orc_inlet failed: {st}")
    return out


def kinetic_speed(grid: Grid, params: Params, u: np.ndarray) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    a = ctypes.c_double(0.0)
    g, P = grid.c(), params.c()
    st = lib().orc_kinetic_speed(ctypes.byref(g), ctypes.byref(P), _ptr(u), ctypes.byref(a))
    if st:
        raise RuntimeError(f"orc_kinetic_speed failed: {st}")
    return a.value


def init_state(grid: Grid, params: Params, jet: Jet, inl: np.ndarray):
    u = np.zeros((4, grid.ny, grid.nx))
    pops = np.zeros((16, grid.ny, grid.nx))
    a = ctypes.c_double(0.0)
    _, pa = _prims(jet)
    g, P = grid.c(), params.c()
    inl = np.ascontiguousarray(inl, dtype=np.float64)
    st = lib().orc_init_state(ctypes.byref(g), ctypes.byref(P), _ptr(inl), ctypes.byref(pa), _ptr(u),
                              _ptr(pops), ctypes.byref(a))
    if st:
        raise RuntimeError(f"orc_init_state failed: {st}")
    return u, pops, a.value


def step(grid: Grid, params: Params, a: float, u: np.ndarray, pops: np.ndarray,
         inl: np.ndarray | None = None, check: bool = True):
    """One VLBM step with kinetic speed ``a``; returns (u_new, pops_new, status)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    pops = np.ascontiguousarray(pops, dtype=np.float64)
    un = np.zeros_like(u)
    pn = np.zeros_like(pops)
    g, P = grid.c(), params.c()
    ip = _ptr(np.ascontiguousarray(inl, dtype=np.float64)) if inl is not None else None
    if params.bc == BC_JET and inl is None:
        raise ValueError("jet boundary needs the inlet table")
    st = lib().orc_step(ctypes.byref(g), ctypes.byref(P), float(a), ip, _ptr(u), _ptr(pops), _ptr(un),
                        _ptr(pn))
    if check and st:
        raise RuntimeError(f"orc_step failed: {st}")
    return un, pn, st


def theta_star(U0, D, lo_b, hi_b, eps_r, eps_p, gamma=5.0 / 3.0) -> float:
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    return lib().orc_theta_star_export(_ptr(U0), _ptr(D), lo_b, hi_b, eps_r, eps_p, gamma)


def moments(grid: Grid, params: Params, u: np.ndarray):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = [np.zeros((grid.ny, grid.nx)) for _ in range(4)]
    g = grid.c()
    lib().orc_moments(ctypes.byref(g), params.gamma, _ptr(u), *[_ptr(o) for o in out])
    return tuple(out)


def run_jet(grid: Grid, params: Params, jet: Jet, seed: int, m0: int, count: int, nsteps: int,
            t_end: float | None = None, want_pops: bool = True):
    """Realizations m0..m0+count-1 from t = 0: ``nsteps`` steps, or to ``t_end``
    with the landing rule (``nsteps`` is then a cap)."""
    n = grid.nx * grid.ny
    u = np.zeros((count, 4, grid.ny, grid.nx))
    pops = np.zeros((count, 16, grid.ny, grid.nx)) if want_pops else None
    t = np.zeros(count)
    s = np.zeros(count, dtype=np.int64)
    pj, pa = _prims(jet)
    amp = jet.amplitudes()
    g, P = grid.c(), params.c()
    st = lib().orc_run_jet(ctypes.byref(g), ctypes.byref(P), ctypes.byref(pj), ctypes.byref(pa),
                           jet.r_jet, jet.K, _ptr(amp), ctypes.c_uint64(seed), m0, count, nsteps,
                           -1.0 if t_end is None else float(t_end), _ptr(u),
                           _ptr(pops) if pops is not None else None, _ptr(t), _ptr(s))
    if st:
        raise RuntimeError(f"orc_run_jet failed: {st}")
    del n
    return {"u": u, "pops": pops, "t": t, "steps": s}


# --------------------------------------------------------------------------- #
# Ensemble statistics (Sec. 3.2 and Sec. 3.4).                                 #
# --------------------------------------------------------------------------- #


def restrict(fine: np.ndarray, r: int) -> np.ndarray:
    """Block average of the last two axes by r x r blocks (Sec. 3.2, operator R)."""
    *lead, nyf, nxf = fine.shape
    if nyf % r or nxf % r:
        raise ValueError("fine grid is not an r-multiple of the coarse grid")
    out = np.zeros((*lead, nyf // r, nxf // r))
    for a in range(r):
        for b in range(r):
            out += fine[..., a::r, b::r]
    return out / (r * r)


def ensemble_stats(ens_a: np.ndarray, ens_b: np.ndarray):
    """Per-cell mean, population std of both ensembles and one-point W1 between
    them (Eqs. mean, std, w1disc).  ens_* has shape [M, ...cells] on one grid."""
    ens_a = np.asarray(ens_a, dtype=np.float64)
    ens_b = np.asarray(ens_b, dtype=np.float64)
    M = ens_a.shape[0]
    if ens_b.shape != ens_a.shape:
        raise ValueError("both ensembles must hold M samples on the same grid")
    mean_a = ens_a.sum(axis=0) / M
    mean_b = ens_b.sum(axis=0) / M
    std_a = np.sqrt(((ens_a - mean_a) ** 2).sum(axis=0) / M)
    std_b = np.sqrt(((ens_b - mean_b) ** 2).sum(axis=0) / M)
    sa = np.sort(ens_a, axis=0)
    sb = np.sort(ens_b, axis=0)
    w1 = np.abs(sa - sb).sum(axis=0) / M
    return mean_a, std_a, mean_b, std_b, w1


def stats_w1_mean_std(ens_a: np.ndarray, ens_b: np.ndarray):
    """Statistics between a coarse ensemble [M, ny, nx] and a fine ensemble
    [M, r ny, r nx], the fine one restricted onto the coarse grid first."""
    r = ens_b.shape[-1] // ens_a.shape[-1]
    if r < 1 or ens_b.shape[-1] != r * ens_a.shape[-1] or ens_b.shape[-2] != r * ens_a.shape[-2]:
        raise ValueError("fine grid must be an integer refinement of the coarse grid")
    b = restrict(ens_b, r) if r > 1 else np.asarray(ens_b, dtype=np.float64)
    return ensemble_stats(ens_a, b)


# --------------------------------------------------------------------------- #
# Error functionals and diagnostics (Sec. 3.3-3.4, Sec. 4.3).                  #
# --------------------------------------------------------------------------- #


def error_functionals(ens_a: np.ndarray, ens_b: np.ndarray):
    """(E_mean, E_std, W_11, E_strong) between a coarse ensemble [M, ny, nx]
    and a fine one [M, r ny, r nx] restricted onto it (Eqs. mean, std,
    w1disc, strongError): cell averages of |mean_a - mean_b|, |std_a - std_b|
    and of the one-point W1, and the realization average of the relative L1
    distance ||a_m - R b_m||_1 / ||R b_m||_1 (the L1 norms as sums over the
    common grid: the cell size cancels)."""
    ens_a = np.asarray(ens_a, dtype=np.float64)
    r = ens_b.shape[-1] // ens_a.shape[-1]
    b = restrict(ens_b, r) if r > 1 else np.asarray(ens_b, dtype=np.float64)
    mean_a, std_a, mean_b, std_b, w1 = ensemble_stats(ens_a, b)
    n = mean_a.size
    e_mean = np.abs(mean_a - mean_b).sum() / n
    e_std = np.abs(std_a - std_b).sum() / n
    w11 = w1.sum() / n
    M = ens_a.shape[0]
    strong = 0.0
    for m in range(M):
        strong += np.abs(ens_a[m] - b[m]).sum() / np.abs(b[m]).sum()
    return e_mean, e_std, w11, strong / M


def w1_points_2d(a: np.ndarray, b: np.ndarray) -> float:
    """First Wasserstein distance between the uniform empirical measures of the
    M points a [M, 2] and b [M, 2] on R^2 with Euclidean ground cost: the
    optimal assignment (scipy's linear_sum_assignment on the cost matrix),
    (1/M) min over permutations sigma of sum_i |a_i - b_sigma(i)|."""
    from scipy.optimize import linear_sum_assignment

    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    dx = a[:, None, 0] - b[None, :, 0]
    dy = a[:, None, 1] - b[None, :, 1]
    C = np.sqrt(dx * dx + dy * dy)
    r, c = linear_sum_assignment(C)
    return float(C[r, c].sum() / a.shape[0])


def two_point_points(nx: int, ny: int, npd: int):
    """The npd x npd subsample of a grid: the centre cell of each of npd equal
    strips per direction, as (i, j) in row-major order (j outer)."""
    xs = [((2 * k + 1) * nx) // (2 * npd) for k in range(npd)]
    ys = [((2 * k + 1) * ny) // (2 * npd) for k in range(npd)]
    return [(i, j) for j in ys for i in xs]


def w1_two_point(ens_a: np.ndarray, ens_b: np.ndarray, npd: int = 10):
    """Two-point Wasserstein distance W_{1,2} (Sec. 3.4, Eq. (w2)) between a
    coarse ensemble [M, ny, nx] and a fine one [M, r ny, r nx] restricted onto
    it: for every ordered pair (x_k, x_k') of the npd x npd subsample, the W1
    on R^2 between the empirical joint laws of (rho(x_k), rho(x_k')) of the two
    ensembles; returns (the mean over the P = npd^4 pairs, the per-pair values
    in pair order k * npd^2 + k')."""
    ens_a = np.asarray(ens_a, dtype=np.float64)
    r = ens_b.shape[-1] // ens_a.shape[-1]
    b = restrict(ens_b, r) if r > 1 else np.asarray(ens_b, dtype=np.float64)
    M, ny, nx = ens_a.shape
    pts = two_point_points(nx, ny, npd)
    out = np.zeros(len(pts) * len(pts))
    for k, (i, j) in enumerate(pts):
        for k2, (i2, j2) in enumerate(pts):
            A = np.stack([ens_a[:, j, i], ens_a[:, j2, i2]], 1)
            B = np.stack([b[:, j, i], b[:, j2, i2]], 1)
            out[k * len(pts) + k2] = w1_points_2d(A, B)
    return float(out.mean()), out


def quantile(samples: np.ndarray, alpha: float) -> np.ndarray:
    """Empirical alpha-quantile per cell, Eq. (empcdf):
    p_alpha = inf{xi : F(xi) >= alpha} = the ceil(alpha M)-th smallest sample."""
    s = np.sort(np.asarray(samples, dtype=np.float64), axis=0)
    M = s.shape[0]
    k = int(np.ceil(alpha * M))
    k = min(max(k, 1), M)
    return s[k - 1]


def width_ratio(samples: np.ndarray) -> np.ndarray:
    """Quantile width ratio Q = (p95 - p5) / (p84 - p16), Eq. (widthratio)."""
    return (quantile(samples, 0.95) - quantile(samples, 0.05)) / (quantile(samples, 0.84) - quantile(samples, 0.16))


def histogram(samples: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """Per-cell histogram density on bins [edges[j], edges[j+1]), Eq. (hist):
    f = count / (M |B_j|); samples outside [edges[0], edges[-1]) are not
    counted.  samples [M, ...cells] -> [nbins, ...cells]."""
    s = np.asarray(samples, dtype=np.float64)
    M = s.shape[0]
    nb = len(edges) - 1
    out = np.zeros((nb,) + s.shape[1:])
    for j in range(nb):
        inside = (s >= edges[j]) & (s < edges[j + 1])
        out[j] = inside.sum(axis=0) / (M * (edges[j + 1] - edges[j]))
    return out


def rate_fit(dx, err):
    """Least-squares slope and intercept of log(err) against log(dx), Eq. (ratefit)."""
    x = np.log(np.asarray(dx, dtype=np.float64))
    y = np.log(np.asarray(err, dtype=np.float64))
    A = np.stack([x, np.ones_like(x)], axis=1)
    (r, c), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(r), float(c)
