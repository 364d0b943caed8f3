"""Failure detection without a GPU fault: a device wait that nothing
completes gives up after its bound and reports VLBM_ETIMEOUT, and the GPU
and the contexts stay usable afterwards."""

import numpy as np
import pytest

from paper_2605_25282_gb300 import vlbm
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    ens = H.gpu_jet([(64, 32)], 2, precision="mixed")
    ens.step(3)
    before = H.to_np(ens.density(0))
    assert vlbm.check_bounded_wait(0.02) == 6  # VLBM_ETIMEOUT
    assert "gave up" in vlbm.load_library().vlbm_last_error(None).decode()
    ens.step(2)
    ens.sync()
    after = H.to_np(ens.density(0))
    assert np.isfinite(after).all() and not np.array_equal(before, after)
    t, s = ens.time(0)
    assert np.all(s == 5)


def test_bounded_wait_rejects_bad_limits():
    assert vlbm.check_bounded_wait(0.0) == 1
    assert vlbm.check_bounded_wait(11.0) == 1
