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


class _Pool:
    """The device's default stream-ordered memory pool (where cudaMallocAsync
    allocates), through the CUDA runtime the library itself is linked to."""

    USED_CURRENT, USED_HIGH = 7, 8  # cudaMemPoolAttrUsedMemCurrent / UsedMemHigh

    def __init__(self):
        self.rt = ctypes.CDLL("libcudart.so.13")
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), torch.cuda.current_device()) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(zero)) == 0


def test_noalloc_matches_allocating_call_twice_in_a_row():
    lib = vlbm.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(inputs.random_samples(31, 300, 20, 30), inputs.random_samples(32, 300, 40, 60)),
             (inputs.random_samples(33, 57, 7, 5), inputs.random_samples(34, 57, 7, 5))]
    tensors = [(torch.tensor(a, dtype=torch.float32, device="cuda"), torch.tensor(b, dtype=torch.float32, device="cuda"))
               for a, b in cases]
    refs = [vlbm.stats_error_functionals(a, b) for a, b in tensors]
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, *tensors[0], out, stream) == 0, lib.vlbm_last_error(None).decode()  # address lookup
    torch.cuda.synchronize()
    pool = _Pool()
    pool.reset_high()
    used0, free0 = pool.get(pool.USED_CURRENT), torch.cuda.mem_get_info()[0]
    for (a, b), ref in zip(tensors, refs):
        assert _noalloc(lib, a, b, out, stream) == 0, lib.vlbm_last_error(None).decode()
        torch.cuda.synchronize()
        # the same kernels in the same order: identical to the allocating call
        assert torch.equal(out, ref), (out, ref)
    # nothing was allocated: the pool never grew and the device's free memory is unchanged
    assert pool.get(pool.USED_HIGH) == used0
    assert torch.cuda.mem_get_info()[0] == free0
    # (the check sees the allocating call's scratch)
    vlbm.stats_error_functionals(*tensors[0])
    torch.cuda.synchronize()
    assert pool.get(pool.USED_HIGH) > used0


def test_noalloc_rejects_ensembles_beyond_its_scratch():
    lib = vlbm.load_library()
    a = torch.zeros((4097, 1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, a, a, out, 0) == 1
    assert "4096" in lib.vlbm_last_error(None).decode()
