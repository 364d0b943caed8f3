"""The C-ABI library builds, loads and exports every call include/vlbm.h
declares; host-side validation rejects bad arguments before any device work.
These tests make no compute call and need no GPU."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2605_25282_gb300 import vlbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = "\n".join(l for l in src.splitlines() if "typedef" not in l)
    names = re.findall(r"\b((?:vlbm|stats)_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declarations_are_exported():
    names = declared_functions()
    assert "vlbm_create" in names and "stats_w1_mean_std" in names
    assert sorted(vlbm.EXPORTED) == names
    lib = vlbm.load_library()
    out = subprocess.run(["nm", "-D", "--defined-only", vlbm.library_path()], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for n in names:
        assert n in syms, n
        assert getattr(lib, n) is not None


def _create(levels, gamma=5 / 3, jet=None, amb=None, relax=None, precision=0):
    lib = vlbm.load_library()
    arr = (vlbm.Grid * max(1, len(levels)))(*levels) if levels else None
    jet = jet or vlbm.Prim(5.0, 800.0, 0.0, 0.4127)
    amb = amb or vlbm.Prim(0.5, 0.0, 0.0, 0.4127)
    ctx = ctypes.c_void_p()
    rel = ctypes.byref(relax) if relax is not None else None
    code = lib.vlbm_create(arr, len(levels), gamma, ctypes.byref(jet), ctypes.byref(amb), rel, precision, None,
                           vlbm.ALLOC_FN(0), vlbm.FREE_FN(0), None, ctypes.byref(ctx))
    return code, lib.vlbm_last_error(None).decode()


@pytest.mark.parametrize("case, expect", [
    (dict(levels=[]), "1..8 grid levels"),
    (dict(levels=[vlbm.Grid(2, 100, 2.5, -0.625, 0.625)]), "nx, ny >= 3"),
    (dict(levels=[vlbm.Grid(200, 100, 2.5, -0.5, 0.5)]), "square"),
    (dict(levels=[vlbm.jet_grid(200, 100)], gamma=1.0), "gamma"),
    (dict(levels=[vlbm.jet_grid(200, 100)], jet=vlbm.Prim(-5.0, 800.0, 0.0, 0.4127)), "rho > 0"),
    (dict(levels=[vlbm.jet_grid(200, 100)], amb=vlbm.Prim(float("inf"), 0.0, 0.0, 0.4127)), "finite"),
    (dict(levels=[vlbm.jet_grid(200, 100)], jet=vlbm.Prim(5.0, float("nan"), 0.0, 0.4127)), "finite"),
    (dict(levels=[vlbm.jet_grid(200, 100)], precision=7), "precision"),
    (dict(levels=[vlbm.jet_grid(200, 100)], relax=vlbm.Relax(1.0, 1.0, 2, 0.1, 0.0, 1e-13)), "alpha"),
    (dict(levels=[vlbm.jet_grid(200, 100)], relax=vlbm.Relax(0.0, 0.5, 2, 0.1, 0.0, 1e-13)), "kappa"),
    (dict(levels=[vlbm.jet_grid(200, 100)], relax=vlbm.Relax(0.0, 1.0, 5, 0.1, 0.0, 1e-13)), "limiter"),
    (dict(levels=[vlbm.jet_grid(200, 100)], relax=vlbm.Relax(0.0, float("inf"), 2, 0.1, 0.0, 1e-13)), "finite"),
    (dict(levels=[vlbm.jet_grid(200, 100)], relax=vlbm.Relax(0.0, 1.0, 2, float("inf"), 0.0, 1e-13)), "finite"),
    (dict(levels=[vlbm.Grid(200, 100, float("inf"), -0.625, 0.625)]), "finite"),
])
def test_create_rejects_invalid_problems(case, expect):
    code, msg = _create(**case)
    assert code == 1, (code, msg)
    assert expect in msg


def test_stats_rejects_bad_shapes_without_launching():
    lib = vlbm.load_library()
    dummy = ctypes.c_void_p(16)
    # b is not an integer refinement of a
    code = lib.stats_w1_mean_std(dummy, 0, 10, 10, dummy, 0, 15, 15, 4, None, None, None, None, None, None)
    assert code == 1 and "refinement" in lib.vlbm_last_error(None).decode()
    code = lib.stats_w1_mean_std(dummy, 0, 10, 10, dummy, 0, 20, 30, 4, None, None, None, None, None, None)
    assert code == 1
    code = lib.stats_w1_mean_std(dummy, 0, 10, 10, dummy, 0, 10, 10, 5000, None, None, None, None, None, None)
    assert code == 1 and "M" in lib.vlbm_last_error(None).decode()
    code = lib.stats_w1_mean_std(None, 0, 10, 10, dummy, 0, 10, 10, 4, None, None, None, None, None, None)
    assert code == 1
    # an empty fine level (refinement factor 0) and a coarse grid beyond one launch
    code = lib.stats_w1_mean_std(dummy, 0, 10, 10, dummy, 0, 0, 0, 4, None, None, None, None, None, None)
    assert code == 1 and "refinement" in lib.vlbm_last_error(None).decode()
    code = lib.stats_w1_mean_std(dummy, 0, 65536, 65536, dummy, 0, 65536, 65536, 4, None, None, None, None, None,
                                 None)
    assert code == 1 and "2^31" in lib.vlbm_last_error(None).decode()


def test_null_context_calls_fail_cleanly():
    lib = vlbm.load_library()
    assert lib.vlbm_step(None, 1) == 1
    assert lib.vlbm_advance_to(None, 0.1) == 1
    assert lib.vlbm_sync(None) == 1
    rows = ctypes.c_int(5)
    assert lib.vlbm_step_rows(None, ctypes.byref(rows)) == 1 and rows.value == 5
    assert lib.vlbm_last_error(None)
    lib.vlbm_destroy(None)


def test_init_samples_rejects_out_of_range_host_values_before_device_work():
    lib = vlbm.load_library()
    arr = (vlbm.Grid * 1)(vlbm.jet_grid(16, 8))
    jet, amb = vlbm.Prim(5.0, 800.0, 0.0, 0.4127), vlbm.Prim(0.5, 0.0, 0.0, 0.4127)
    ctx = ctypes.c_void_p()
    code = lib.vlbm_create(arr, 1, 5 / 3, ctypes.byref(jet), ctypes.byref(amb), None, 1, None,
                           vlbm.ALLOC_FN(0), vlbm.FREE_FN(0), None, ctypes.byref(ctx))
    assert code == 0, lib.vlbm_last_error(None)
    try:
        p = vlbm.PerturbParams(K=3).c()
        for bad in (1.5, float("nan"), -1.0000001):
            xi = np.zeros((2, 6))
            xi[1, 4] = bad
            code = lib.vlbm_init_ensemble_samples(ctx, xi.ctypes.data_as(ctypes.c_void_p), 2, ctypes.byref(p))
            assert code == 1 and "xi[10]" in lib.vlbm_last_error(ctx).decode(), bad
        assert lib.vlbm_init_ensemble_samples(ctx, None, 2, ctypes.byref(p)) == 1
        idx, name, cnt = ctypes.c_int(7), ctypes.c_char_p(), ctypes.c_int(0)
        assert lib.vlbm_step_design(ctx, ctypes.byref(idx), ctypes.byref(name), ctypes.byref(cnt)) == 0
        assert idx.value == -1 and name.value == b"none" and cnt.value >= 5
        rows = ctypes.c_int(7)
        assert lib.vlbm_step_rows(ctx, ctypes.byref(rows)) == 0 and rows.value == 0
        assert lib.vlbm_step_rows(ctx, None) == 1
    finally:
        lib.vlbm_destroy(ctx)


def test_allocation_failure_is_reported_without_device_work():
    # host-side fault injection: an allocator that refuses every request
    lib = vlbm.load_library()
    arr = (vlbm.Grid * 1)(vlbm.jet_grid(16, 8))
    jet, amb = vlbm.Prim(5.0, 800.0, 0.0, 0.4127), vlbm.Prim(0.5, 0.0, 0.0, 0.4127)
    calls = []

    def refuse(nbytes, user):
        calls.append(nbytes)
        return None

    def release(ptr, user):
        pass

    alloc_cb, free_cb = vlbm.ALLOC_FN(refuse), vlbm.FREE_FN(release)
    ctx = ctypes.c_void_p()
    # stream handle 1 is the legacy default stream: valid everywhere, no work enqueued here
    code = lib.vlbm_create(arr, 1, 5 / 3, ctypes.byref(jet), ctypes.byref(amb), None, 1, ctypes.c_void_p(1),
                           alloc_cb, free_cb, None, ctypes.byref(ctx))
    assert code == 0, lib.vlbm_last_error(None)
    try:
        code = lib.vlbm_init_ensemble(ctx, 0, 4, None)
        assert code == 2, (code, lib.vlbm_last_error(ctx))  # VLBM_ENOMEM
        assert "allocation" in lib.vlbm_last_error(ctx).decode() and calls
        # the context is still usable for calls that need no state
        assert lib.vlbm_step(ctx, 1) == 7  # VLBM_ESTATE: nothing initialised
    finally:
        lib.vlbm_destroy(ctx)


@pytest.mark.parametrize("field, value, expect", [
    ("A", float("inf"), "finite"),
    ("p_decay", float("nan"), "finite"),
    ("r_jet", float("inf"), "r_jet"),
    ("r_jet", 0.0, "r_jet"),
    ("amp", float("nan"), "amp[2]"),
])
def test_init_rejects_invalid_perturbations_before_device_work(field, value, expect):
    lib = vlbm.load_library()
    arr = (vlbm.Grid * 1)(vlbm.jet_grid(16, 8))
    jet, amb = vlbm.Prim(5.0, 800.0, 0.0, 0.4127), vlbm.Prim(0.5, 0.0, 0.0, 0.4127)
    calls = []

    def refuse(nbytes, user):
        calls.append(nbytes)
        return None

    alloc_cb, free_cb = vlbm.ALLOC_FN(refuse), vlbm.FREE_FN(lambda ptr, user: None)
    ctx = ctypes.c_void_p()
    # stream handle 1 is the legacy default stream: valid everywhere, no work enqueued here
    assert lib.vlbm_create(arr, 1, 5 / 3, ctypes.byref(jet), ctypes.byref(amb), None, 1, ctypes.c_void_p(1),
                           alloc_cb, free_cb, None, ctypes.byref(ctx)) == 0
    try:
        p = vlbm.PerturbParams(K=4).c()
        if field == "amp":
            p.use_amp = 1
            for k in range(4):
                p.amp[k] = 0.01
            p.amp[2] = value
        else:
            setattr(p, field, value)
        code = lib.vlbm_init_ensemble(ctx, 0, 2, ctypes.byref(p))
        assert code == 1 and expect in lib.vlbm_last_error(ctx).decode(), (code, lib.vlbm_last_error(ctx))
        assert calls == []  # rejected before any allocation
    finally:
        lib.vlbm_destroy(ctx)
