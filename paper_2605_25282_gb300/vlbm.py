"""Python binding of libvlbm (ctypes; argument marshalling only).

Every step of the method runs in the CUDA library; PyTorch provides device
memory (its caching allocator backs the library's state) and the stream.  The
binding never falls back to a CPU path: it raises if the library or a GPU is
missing.

Names follow the C ABI in include/vlbm.h: ``Ensemble`` wraps a ``vlbm_ctx``
(vlbm_create / vlbm_init_ensemble / vlbm_step / vlbm_advance_to / vlbm_moments
...), and ``stats_w1_mean_std`` wraps the statistics call.

Streams: every call is ordered after the work the caller has queued on its
current stream, and the caller's current stream after the call, whichever
stream the call itself runs on (an Ensemble's own, or a statistics call's
``stream`` argument).
"""

from __future__ import annotations

import contextlib
import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

VLBM_FP64, VLBM_MIXED = 0, 1
LIMITER_NONE, LIMITER_UNLIMITED, LIMITER_RTHETA = 0, 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONPOSITIVE", 5: "ENONFINITE", 6: "ETIMEOUT",
          7: "ESTATE"}

EXPORTED = [
    "vlbm_default_relax", "vlbm_default_perturb", "vlbm_create", "vlbm_init_ensemble",
    "vlbm_init_ensemble_block", "vlbm_init_ensemble_samples", "vlbm_kernel_launches", "vlbm_step",
    "vlbm_advance_to", "vlbm_moments", "vlbm_density", "vlbm_time", "vlbm_sync", "vlbm_get_state",
    "vlbm_set_state", "stats_w1_mean_std", "stats_error_functionals", "stats_error_functionals_noalloc",
    "stats_quantiles", "stats_histogram", "stats_restrict", "stats_w1_two_point",
    "vlbm_save", "vlbm_load", "vlbm_last_error", "vlbm_step_design", "vlbm_step_rows", "vlbm_grad_amplitudes",
    "vlbm_amplitudes",
    "vlbm_check_bounded_wait", "vlbm_destroy",
]


class VlbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x_max", ctypes.c_double),
                ("y_min", ctypes.c_double), ("y_max", ctypes.c_double)]


class Prim(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("u", ctypes.c_double), ("v", ctypes.c_double),
                ("p", ctypes.c_double)]


class Relax(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("kappa", ctypes.c_double), ("limiter", ctypes.c_int),
                ("rlmp_rel", ctypes.c_double), ("rlmp_abs", ctypes.c_double), ("eps_pos", ctypes.c_double)]


class Perturb(ctypes.Structure):
    _fields_ = [("r_jet", ctypes.c_double), ("A", ctypes.c_double), ("p_decay", ctypes.c_double),
                ("K", ctypes.c_int), ("amp", ctypes.c_double * 16), ("use_amp", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libvlbm.so (building it with nvcc when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libvlbm not built: {_build.LIB} is missing (run paper_2605_25282_gb300/build.py)")
    lib = ctypes.CDLL(_build.LIB)
    p, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    sig = {
        "vlbm_default_relax": ([p], None),
        "vlbm_default_perturb": ([p], None),
        "vlbm_create": ([p, i, d, p, p, p, i, p, ALLOC_FN, FREE_FN, p, ctypes.POINTER(p)], i),
        "vlbm_init_ensemble": ([p, u64, i, p], i),
        "vlbm_init_ensemble_block": ([p, u64, i, i, p], i),
        "vlbm_init_ensemble_samples": ([p, p, i, p], i),
        "vlbm_kernel_launches": ([], ctypes.c_ulonglong),
        "vlbm_step": ([p, i], i),
        "vlbm_advance_to": ([p, d], i),
        "vlbm_moments": ([p, i, i, i, p, p, p, p], i),
        "vlbm_density": ([p, i, i, i, p, i], i),
        "vlbm_time": ([p, i, p, p], i),
        "vlbm_sync": ([p], i),
        "vlbm_get_state": ([p, i, i, i, p, p], i),
        "vlbm_set_state": ([p, i, i, i, p, p], i),
        "stats_w1_mean_std": ([p, i, i, i, p, i, i, i, i, p, p, p, p, p, p], i),
        "stats_error_functionals": ([p, i, i, i, p, i, i, i, i, p, p], i),
        "stats_error_functionals_noalloc": ([p, i, i, i, p, i, i, i, i, p, p], i),
        "stats_quantiles": ([p, i, i, i, i, p, i, p, p], i),
        "stats_histogram": ([p, i, i, i, i, p, i, p, p], i),
        "stats_restrict": ([p, i, i, i, i, i, p, i, p], i),
        "stats_w1_two_point": ([p, i, i, i, p, i, i, i, i, i, p, p, p], i),
        "vlbm_save": ([p, p, ctypes.POINTER(ctypes.c_size_t)], i),
        "vlbm_load": ([p, p, ctypes.c_size_t], i),
        "vlbm_last_error": ([p], ctypes.c_char_p),
        "vlbm_step_design": ([p, p, ctypes.POINTER(ctypes.c_char_p), p], i),
        "vlbm_step_rows": ([p, p], i),
        "vlbm_grad_amplitudes": ([p, i, i, p, p, p], i),
        "vlbm_amplitudes": ([p, p, p], i),
        "vlbm_check_bounded_wait": ([d], i),
        "vlbm_destroy": ([p], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(code: int, ctx=None):
    if code != 0:
        msg = load_library().vlbm_last_error(ctx).decode()
        raise VlbmError(code, msg)


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libvlbm needs a CUDA GPU; no CPU fallback exists")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def jet_grid(nx: int, ny: int, x_max: float = 2.5) -> Grid:
    """Square cells of size x_max / nx on [0, x_max] x [-ny dx / 2, ny dx / 2]."""
    dx = x_max / nx
    return Grid(nx, ny, x_max, -0.5 * ny * dx, 0.5 * ny * dx)


@dataclass(frozen=True)
class JetProblem:
    """Sec. 2.2 constants of the Mach 2000 jet."""
    gamma: float = 5.0 / 3.0
    rho_jet: float = 5.0
    v_jet: float = 800.0
    p_amb: float = 0.4127
    rho_amb: float = 0.5


@dataclass(frozen=True)
class PerturbParams:
    """Sec. 2.3, Eq. (karhunenExp)."""
    r_jet: float = 0.05
    A: float = 0.1
    p_decay: float = 2.0
    K: int = 10
    amp: list | None = None

    def c(self) -> Perturb:
        p = Perturb()
        p.r_jet, p.A, p.p_decay, p.K = self.r_jet, self.A, self.p_decay, self.K
        if self.amp is not None:
            for k, a in enumerate(self.amp):
                p.amp[k] = float(a)
            p.use_amp = 1
        return p


@dataclass(frozen=True)
class RelaxParams:
    alpha: float = 0.0
    kappa: float = 1.0
    limiter: int = LIMITER_RTHETA
    rlmp_rel: float = 0.1
    rlmp_abs: float = 0.0
    eps_pos: float = 1e-13

    def c(self) -> Relax:
        return Relax(self.alpha, self.kappa, self.limiter, self.rlmp_rel, self.rlmp_abs, self.eps_pos)


class Ensemble:
    """A Monte-Carlo ensemble of jet realizations on one or more grid levels."""

    def __init__(self, levels, precision: str = "fp64", problem: JetProblem = JetProblem(),
                 relax: RelaxParams = RelaxParams(), stream: torch.cuda.Stream | None = None,
                 device: int | None = None):
        _require_cuda()
        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.grids = [lv if isinstance(lv, Grid) else jet_grid(*lv) for lv in levels]
        self.precision = {"fp64": VLBM_FP64, "mixed": VLBM_MIXED}[precision]
        self.problem = problem
        # The context needs a real stream: PyTorch's default stream has handle 0,
        # which the C ABI would read as "create a private stream".
        if stream is None or stream.cuda_stream == 0:
            stream = torch.cuda.Stream(self.device)
        self.stream = stream
        blocks = {}
        self._blocks = blocks
        dev_index, alloc_stream = self.device.index, self.stream

        # The callbacks hold no reference to self, so the ensemble is freed as
        # soon as it is unreachable (no reference cycle through ctypes).
        def _alloc(nbytes, _user):
            with torch.cuda.device(dev_index):
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), dev_index, alloc_stream)
            blocks[ptr] = nbytes
            return ptr

        def _free(ptr, _user):
            if ptr in blocks:
                del blocks[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        arr = (Grid * len(self.grids))(*self.grids)
        jet = Prim(problem.rho_jet, problem.v_jet, 0.0, problem.p_amb)
        amb = Prim(problem.rho_amb, 0.0, 0.0, problem.p_amb)
        rel = relax.c()
        ctx = ctypes.c_void_p()
        _check(self.lib.vlbm_create(arr, len(self.grids), problem.gamma, ctypes.byref(jet), ctypes.byref(amb),
                                    ctypes.byref(rel), self.precision, ctypes.c_void_p(self.stream.cuda_stream),
                                    self._alloc_cb, self._free_cb, None, ctypes.byref(ctx)))
        self.ctx = ctx
        self.M = 0

    def _enter(self):
        """Orders the context's stream after work already queued by the caller."""
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)

    def _leave(self):
        """Orders the caller's current stream after the context's work."""
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    def _call(self, fn, *args):
        self._enter()
        code = fn(self.ctx, *args)
        self._leave()
        _check(code, self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.vlbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, level: int):
        g = self.grids[level]
        return g.ny, g.nx

    def init(self, seed: int, M: int, perturb: PerturbParams = PerturbParams(), m_begin: int = 0):
        p = perturb.c()
        self._call(self.lib.vlbm_init_ensemble_block, seed, m_begin, M, ctypes.byref(p))
        self.M = M

    def init_samples(self, xi, perturb: PerturbParams = PerturbParams()):
        """Initialises M = xi.shape[0] realizations from given KL coefficients:
        row r holds Y_1..Y_K, Z_1..Z_K in [-1, 1].  xi is a float64 numpy
        array, or a CPU (pinned or pageable) or CUDA torch tensor."""
        if isinstance(xi, np.ndarray):
            xi = torch.from_numpy(np.ascontiguousarray(xi, dtype=np.float64))
        if xi.dtype != torch.float64 or not xi.is_contiguous() or xi.dim() != 2:
            raise ValueError("xi must be a contiguous float64 matrix [M, 2K]")
        p = perturb.c()
        if xi.shape[1] != 2 * p.K:
            raise ValueError(f"xi has {xi.shape[1]} columns; 2K = {2 * p.K}")
        self._xi_keep = xi  # a pinned host buffer is read asynchronously
        self._call(self.lib.vlbm_init_ensemble_samples, _ptr(xi), int(xi.shape[0]), ctypes.byref(p))
        self.M = int(xi.shape[0])

    def step(self, n: int = 1):
        self._call(self.lib.vlbm_step, n)

    def advance_to(self, t: float):
        self._call(self.lib.vlbm_advance_to, float(t))

    def _count(self, m0, count):
        return self.M - m0 if count is None else count

    def moments(self, level: int = 0, m0: int = 0, count: int | None = None):
        count = self._count(m0, count)
        ny, nx = self.shape(level)
        out = [torch.empty((count, ny, nx), dtype=torch.float64, device=self.device) for _ in range(4)]
        self._call(self.lib.vlbm_moments, level, m0, count, *[_ptr(o) for o in out])
        return dict(zip(("rho", "u", "v", "p"), out))

    def density(self, level: int = 0, m0: int = 0, count: int | None = None, f32: bool = True,
                out: torch.Tensor | None = None):
        count = self._count(m0, count)
        ny, nx = self.shape(level)
        if out is None:
            out = torch.empty((count, ny, nx), dtype=torch.float32 if f32 else torch.float64, device=self.device)
        self._call(self.lib.vlbm_density, level, m0, count, _ptr(out), int(out.dtype == torch.float32))
        return out

    def time(self, level: int = 0):
        t = np.zeros(self.M)
        s = np.zeros(self.M, dtype=np.int64)
        self._call(self.lib.vlbm_time, level, t.ctypes.data_as(ctypes.c_void_p), s.ctypes.data_as(ctypes.c_void_p))
        return t, s

    def sync(self):
        self._call(self.lib.vlbm_sync)

    def amplitudes(self) -> np.ndarray:
        """Per-mode amplitudes of the last initialisation (Eq. (karhunenExp))."""
        K = ctypes.c_int(0)
        _check(self.lib.vlbm_amplitudes(self.ctx, None, ctypes.byref(K)), self.ctx)
        amp = np.zeros(K.value)
        _check(self.lib.vlbm_amplitudes(self.ctx, amp.ctypes.data_as(ctypes.c_void_p), None), self.ctx)
        return amp

    def grad_amplitudes(self, nsteps: int, w: torch.Tensor, checkpoint_every: int = 20):
        """(J, dJ/da) for J = (1/M) sum_m sum w rho_m after nsteps FP64 steps from the
        initial state of the last initialisation (hand-written discrete adjoint,
        checkpoint-and-recompute every checkpoint_every steps).  w [ny, nx]."""
        ny, nx = self.shape(0)
        w = w.to(self.device, torch.float64).contiguous()
        if tuple(w.shape) != (ny, nx):
            raise ValueError(f"w must be [{ny}, {nx}]")
        grad = np.zeros(len(self.amplitudes()))
        J = ctypes.c_double(0.0)
        self._call(self.lib.vlbm_grad_amplitudes, int(nsteps), int(checkpoint_every), _ptr(w), ctypes.byref(J),
                   grad.ctypes.data_as(ctypes.c_void_p))
        return J.value, grad

    def step_design(self):
        """(index, name, count) of the step kernel's launch design (mixed or
        FP64); index -1 before the first step."""
        idx, cnt, name = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_char_p()
        _check(self.lib.vlbm_step_design(self.ctx, ctypes.byref(idx), ctypes.byref(name), ctypes.byref(cnt)), self.ctx)
        return idx.value, name.value.decode(), cnt.value

    def step_rows(self) -> int:
        """Rows per warp of the mixed warp-march design in use (0 for the
        other designs, for FP64 and before the first step)."""
        rows = ctypes.c_int(0)
        _check(self.lib.vlbm_step_rows(self.ctx, ctypes.byref(rows)), self.ctx)
        return rows.value

    def get_state(self, level: int = 0, m0: int = 0, count: int | None = None, pops: bool = True):
        count = self._count(m0, count)
        ny, nx = self.shape(level)
        u = torch.empty((count, 4, ny, nx), dtype=torch.float64, device=self.device)
        f = torch.empty((count, 16, ny, nx), dtype=torch.float64, device=self.device) if pops else None
        self._call(self.lib.vlbm_get_state, level, m0, count, _ptr(u), _ptr(f))
        return u, f

    def set_state(self, u: torch.Tensor, pops: torch.Tensor, level: int = 0, m0: int = 0):
        u = u.to(self.device, torch.float64).contiguous()
        pops = pops.to(self.device, torch.float64).contiguous()
        count = u.shape[0]
        self._call(self.lib.vlbm_set_state, level, m0, count, _ptr(u), _ptr(pops))
        self._keep = (u, pops)

    def save(self) -> bytes:
        n = ctypes.c_size_t(0)
        self._call(self.lib.vlbm_save, None, ctypes.byref(n))
        buf = (ctypes.c_ubyte * n.value)()
        self._call(self.lib.vlbm_save, buf, ctypes.byref(n))
        return bytes(buf)

    def load(self, blob: bytes):
        buf = (ctypes.c_ubyte * len(blob)).from_buffer_copy(blob)
        self._call(self.lib.vlbm_load, buf, len(blob))


def check_bounded_wait(limit_s: float = 0.05) -> int:
    """Status of one device wait that nothing completes, bounded by limit_s
    (VLBM_ETIMEOUT = 6 is the designed outcome)."""
    _require_cuda()
    return int(load_library().vlbm_check_bounded_wait(float(limit_s)))


def kernel_launches() -> int:
    """Kernels enqueued by libvlbm in this process so far."""
    return int(load_library().vlbm_kernel_launches())


@contextlib.contextmanager
def _on_stream(stream: torch.cuda.Stream | None, device):
    """The stream a statistics call runs on (`stream`, else the caller's
    current one), ordered after the work the caller has queued on its current
    stream; on exit the caller's current stream is ordered after the call, so
    its inputs and outputs are used in order wherever the caller goes on."""
    cur = torch.cuda.current_stream(device)
    s = stream if stream is not None else cur
    other = s.cuda_stream != cur.cuda_stream
    if other:
        s.wait_stream(cur)
    yield s
    if other:
        cur.wait_stream(s)


def stats_w1_mean_std(ens_a: torch.Tensor, ens_b: torch.Tensor, stream: torch.cuda.Stream | None = None):
    """Per-cell mean/std of both ensembles and one-point W1 (b restricted onto a's grid)."""
    _require_cuda()
    lib = load_library()
    if ens_a.dim() != 3 or ens_b.dim() != 3 or ens_a.shape[0] != ens_b.shape[0]:
        raise ValueError("ensembles must be [M, ny, nx] with equal M")
    ens_a = ens_a.contiguous()
    ens_b = ens_b.contiguous()
    M, nya, nxa = ens_a.shape
    _, nyb, nxb = ens_b.shape
    dev = ens_a.device
    out = [torch.empty((nya, nxa), dtype=torch.float64, device=dev) for _ in range(5)]
    with _on_stream(stream, dev) as s:
        _check(lib.stats_w1_mean_std(_ptr(ens_a), int(ens_a.dtype == torch.float32), nxa, nya, _ptr(ens_b),
                                     int(ens_b.dtype == torch.float32), nxb, nyb, M, *[_ptr(o) for o in out],
                                     ctypes.c_void_p(s.cuda_stream)))
    return dict(zip(("mean_a", "std_a", "mean_b", "std_b", "w1"), out))


def stats_restrict(ens: torch.Tensor, r: int, f32: bool = False, stream: torch.cuda.Stream | None = None):
    """Block average of every field of ens [M, ny, nx] onto [M, ny / r, nx / r] (Sec. 3.3)."""
    _require_cuda()
    lib = load_library()
    if ens.dim() != 3:
        raise ValueError("ens must be [M, ny, nx]")
    ens = ens.contiguous()
    M, ny, nx = ens.shape
    out = torch.empty((M, ny // r, nx // r), dtype=torch.float32 if f32 else torch.float64, device=ens.device)
    with _on_stream(stream, ens.device) as s:
        _check(lib.stats_restrict(_ptr(ens), int(ens.dtype == torch.float32), nx, ny, M, r, _ptr(out), int(f32),
                                  ctypes.c_void_p(s.cuda_stream)))
    return out


def stats_w1_two_point(ens_a: torch.Tensor, ens_b: torch.Tensor, npd: int = 10,
                       stream: torch.cuda.Stream | None = None):
    """Two-point Wasserstein distance W_{1,2} (Sec. 3.4) between [M, ny, nx] and
    [M, r ny, r nx] on the npd x npd subsample: (mean as a 0-d device tensor,
    per-pair values [npd^4])."""
    _require_cuda()
    lib = load_library()
    ens_a, ens_b = ens_a.contiguous(), ens_b.contiguous()
    M, nya, nxa = ens_a.shape
    _, nyb, nxb = ens_b.shape
    w = torch.empty((), dtype=torch.float64, device=ens_a.device)
    pairs = torch.empty(npd ** 4, dtype=torch.float64, device=ens_a.device)
    with _on_stream(stream, ens_a.device) as s:
        _check(lib.stats_w1_two_point(_ptr(ens_a), int(ens_a.dtype == torch.float32), nxa, nya, _ptr(ens_b),
                                      int(ens_b.dtype == torch.float32), nxb, nyb, M, npd, _ptr(w), _ptr(pairs),
                                      ctypes.c_void_p(s.cuda_stream)))
    return w, pairs


def stats_error_functionals(ens_a: torch.Tensor, ens_b: torch.Tensor, stream: torch.cuda.Stream | None = None):
    """(E_mean, E_std, W_11, E_strong) between ensembles [M, ny, nx] and [M, r ny, r nx] (device tensor [4])."""
    _require_cuda()
    lib = load_library()
    ens_a, ens_b = ens_a.contiguous(), ens_b.contiguous()
    M, nya, nxa = ens_a.shape
    _, nyb, nxb = ens_b.shape
    out = torch.empty(4, dtype=torch.float64, device=ens_a.device)
    with _on_stream(stream, ens_a.device) as s:
        _check(lib.stats_error_functionals(_ptr(ens_a), int(ens_a.dtype == torch.float32), nxa, nya, _ptr(ens_b),
                                           int(ens_b.dtype == torch.float32), nxb, nyb, M, _ptr(out),
                                           ctypes.c_void_p(s.cuda_stream)))
    return out


def stats_error_functionals_noalloc(ens_a: torch.Tensor, ens_b: torch.Tensor, out: torch.Tensor,
                                    stream: torch.cuda.Stream | None = None):
    """stats_error_functionals writing into a caller-owned device tensor out[4], with no
    device allocation by the library (scratch in a fixed device array, M <= 4096)."""
    _require_cuda()
    lib = load_library()
    if not (ens_a.is_cuda and ens_b.is_cuda and out.is_cuda):
        raise ValueError("ensembles and out must be CUDA tensors")
    if not (ens_a.device == ens_b.device == out.device):
        raise ValueError("ensembles and out must be on one device")
    if not (ens_a.is_contiguous() and ens_b.is_contiguous() and out.is_contiguous()):
        raise ValueError("ensembles and out must be contiguous device tensors")
    if out.dtype != torch.float64 or out.numel() < 4:
        raise ValueError("out must be a float64 device tensor with 4 elements")
    M, nya, nxa = ens_a.shape
    _, nyb, nxb = ens_b.shape
    # the scratch array is resolved for the current device: make it the tensors' one
    with torch.cuda.device(ens_a.device):
        with _on_stream(stream, ens_a.device) as s:
            _check(lib.stats_error_functionals_noalloc(_ptr(ens_a), int(ens_a.dtype == torch.float32), nxa, nya,
                                                       _ptr(ens_b), int(ens_b.dtype == torch.float32), nxb, nyb, M,
                                                       _ptr(out), ctypes.c_void_p(s.cuda_stream)))
    return out


def stats_quantiles(ens: torch.Tensor, probs, stream: torch.cuda.Stream | None = None):
    """Per-cell empirical quantiles p_alpha of an ensemble [M, ny, nx] -> [len(probs), ny, nx]."""
    _require_cuda()
    lib = load_library()
    ens = ens.contiguous()
    M, ny, nx = ens.shape
    pr = np.ascontiguousarray(probs, dtype=np.float64)
    out = torch.empty((len(pr), ny, nx), dtype=torch.float64, device=ens.device)
    with _on_stream(stream, ens.device) as s:
        _check(lib.stats_quantiles(_ptr(ens), int(ens.dtype == torch.float32), nx, ny, M,
                                   pr.ctypes.data_as(ctypes.c_void_p), len(pr), _ptr(out),
                                   ctypes.c_void_p(s.cuda_stream)))
    return out


def stats_histogram(ens: torch.Tensor, edges: torch.Tensor, stream: torch.cuda.Stream | None = None):
    """Per-cell histogram density of an ensemble [M, ny, nx] on the bins of `edges` -> [nbins, ny, nx]."""
    _require_cuda()
    lib = load_library()
    ens = ens.contiguous()
    M, ny, nx = ens.shape
    e = edges.to(ens.device, torch.float64).contiguous()
    out = torch.empty((e.numel() - 1, ny, nx), dtype=torch.float64, device=ens.device)
    with _on_stream(stream, ens.device) as s:
        _check(lib.stats_histogram(_ptr(ens), int(ens.dtype == torch.float32), nx, ny, M, _ptr(e), e.numel() - 1,
                                   _ptr(out), ctypes.c_void_p(s.cuda_stream)))
    return out


def axial_weights(ny: int, nx: int, g: torch.Tensor | None = None) -> torch.Tensor:
    """w [ny, nx] of the axial density: 1/2 on rows ny/2 - 1 and ny/2 (the two
    rows next to y = 0), times the column weights g [nx] (ones by default)."""
    w = torch.zeros((ny, nx), dtype=torch.float64)
    g = torch.ones(nx, dtype=torch.float64) if g is None else g.detach().to("cpu", torch.float64)
    w[ny // 2 - 1] = 0.5 * g
    w[ny // 2] = 0.5 * g
    return w


class AxialMeanDensity(torch.autograd.Function):
    """Axial ensemble-mean density after nsteps FP64 steps as a differentiable
    function of the K per-mode KL amplitudes (Sec. 2.3, Eq. (karhunenExp)).

    forward(amp [K], grid (nx, ny), M, nsteps, seed, checkpoint_every) -> [nx]
    backward runs the library's adjoint (vlbm_grad_amplitudes) with the
    incoming gradient as column weights.  Valid over windows shorter than the
    pathwise-divergence time of the realizations."""

    @staticmethod
    def forward(ctx, amp, grid, M, nsteps, seed=0, checkpoint_every=20):
        nx, ny = grid
        a = amp.detach().to("cpu", torch.float64)
        ens = Ensemble([(nx, ny)], precision="fp64")
        ens.init(seed, M, PerturbParams(K=len(a), amp=[float(x) for x in a]))
        ens.step(nsteps)
        rho = ens.density(0, f32=False)
        axial = 0.5 * (rho[:, ny // 2 - 1] + rho[:, ny // 2]).mean(0)
        ctx.ens, ctx.nsteps, ctx.every = ens, nsteps, checkpoint_every
        return axial.to(amp.device, amp.dtype)

    @staticmethod
    def backward(ctx, g):
        ens = ctx.ens
        ny, nx = ens.shape(0)
        _, grad = ens.grad_amplitudes(ctx.nsteps, axial_weights(ny, nx, g), ctx.every)
        ens.close()
        ctx.ens = None
        return torch.from_numpy(grad).to(g.device, g.dtype), None, None, None, None, None
