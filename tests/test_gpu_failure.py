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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_finite_state_is_reported_and_isolated(precision):
    # host-side fault injection: a NaN written into one realization's state
    ens = H.gpu_jet([(48, 24)], 2, precision=precision)
    ens.step(2)
    u, pops = ens.get_state(0)
    u[1, 0, 12, 20] = float("nan")
    ens.set_state(u, pops, 0)
    ens.step(3)
    with pytest.raises(vlbm.VlbmError) as err:
        ens.sync()
    assert err.value.code == 5 and "realization 1" in str(err.value)  # VLBM_ENONFINITE
    # the other realization is untouched
    d = H.to_np(ens.density(0, 0, 1))
    assert np.isfinite(d).all()
