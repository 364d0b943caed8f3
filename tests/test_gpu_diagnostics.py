"""GPU error functionals, quantiles and histograms (through the C ABI) against
the oracle (Sec. 3.3-3.4, Sec. 4.3-4.4).  Quantiles and histogram counts are
order statistics and integer counts: bit-exact.  Functionals are sums of
O(cells) terms in a different order: 1e-12 relative."""

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_25282_gb300 import vlbm
from tests import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,r,f32", [(1, 1, False), (7, 2, False), (64, 2, True), (1000, 2, False), (4096, 1, True)])
def test_error_functionals_match_oracle(M, r, f32):
    ny, nx = (9, 13) if M <= 1000 else (3, 4)
    a = inputs.random_samples(10 + M, M, ny, nx)
    b = inputs.random_samples(20 + M, M, r * ny, r * nx)
    dt = torch.float32 if f32 else torch.float64
    ta, tb = torch.tensor(a, dtype=dt, device="cuda"), torch.tensor(b, dtype=dt, device="cuda")
    got = vlbm.stats_error_functionals(ta, tb).cpu().numpy()
    ref = O.error_functionals(ta.double().cpu().numpy(), tb.double().cpu().numpy())
    assert np.allclose(got, ref, rtol=1e-12, atol=0), (got, ref)
    # reproducible bit for bit
    again = vlbm.stats_error_functionals(ta, tb).cpu().numpy()
    assert np.array_equal(got, again)


def test_quantiles_bit_exact():
    s = inputs.random_samples(3, 101, 6, 7, "ties")
    probs = [0.05, 0.16, 0.5, 0.84, 0.95, 1.0]
    got = vlbm.stats_quantiles(torch.tensor(s, device="cuda"), probs).cpu().numpy()
    for i, p in enumerate(probs):
        assert np.array_equal(got[i], O.quantile(s, p))


def test_histogram_bit_exact():
    s = inputs.random_samples(4, 333, 5, 6)
    edges = np.linspace(0.0, 30.0, 61)
    got = vlbm.stats_histogram(torch.tensor(s, device="cuda"), torch.tensor(edges)).cpu().numpy()
    assert np.array_equal(got, O.histogram(s, edges))
