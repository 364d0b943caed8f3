"""The allocation-free error functionals (stats_error_functionals_noalloc)
against the allocating entry point, through the C ABI.

It serves callers that cannot allocate device memory while they run (a host
whose pool allocator owns the whole GPU, a real-time loop that cannot afford
an allocation's latency or failure).  The scratch lives in a fixed device
array shared by all calls, so the test makes two calls in a row, with
different inputs, and checks both against the allocating call: a second call
must not see anything left by the first.  This file is collected last; it
passes alone in a fresh process and after the other tests.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2605_25282_gb300 import vlbm
from tests import inputs

pytestmark = pytest.mark.gpu


def _noalloc(lib, a, b, out, stream):
    M, nya, nxa = a.shape
    _, nyb, nxb = b.shape
    return lib.stats_error_functionals_noalloc(
        ctypes.c_void_p(a.data_ptr()), int(a.dtype == torch.float32), nxa, nya, ctypes.c_void_p(b.data_ptr()),
        int(b.dtype == torch.float32), nxb, nyb, M, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_allocating_call_twice_in_a_row():
    lib = vlbm.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(inputs.random_samples(31, 300, 20, 30), inputs.random_samples(32, 300, 40, 60)),
             (inputs.random_samples(33, 57, 7, 5), inputs.random_samples(34, 57, 7, 5))]
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for a_np, b_np in cases:
        a = torch.tensor(a_np, dtype=torch.float32, device="cuda")
        b = torch.tensor(b_np, dtype=torch.float32, device="cuda")
        ref = vlbm.stats_error_functionals(a, b)
        assert _noalloc(lib, a, b, out, stream) == 0, lib.vlbm_last_error(None).decode()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=0), (got, want)


def test_noalloc_rejects_ensembles_beyond_its_scratch():
    lib = vlbm.load_library()
    a = torch.zeros((4097, 1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, a, a, out, 0) == 1
    assert "4096" in lib.vlbm_last_error(None).decode()
