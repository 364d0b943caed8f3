"""Every launch design of the mixed kernel (tile shapes, persistent CTAs, warps
marching up column strips) computes bit-identical results, so the autotuner's
choice never changes a realization (and nested prefixes stay exact)."""

import os
import subprocess
import sys

import numpy as np
import pytest

from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from tests import gpu_helpers as H
ens = H.gpu_jet([(67, 29), (150, 60), (96, 230)], 3, precision="mixed")
ens.step(12)
idx, name, count = ens.step_design()
assert idx == {v}, (idx, name)
np.save({out!r}, np.concatenate([ens.get_state(l)[0].cpu().numpy().ravel() for l in range(3)]))
"""


def test_all_mixed_variants_agree_bitwise(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    probe = H.gpu_jet([(16, 8)], 1, precision="mixed")
    probe.step(1)
    chosen, name, count = probe.step_design()
    assert 0 <= chosen < count and count >= 5, (chosen, name, count)
    probe.close()
    outs = []
    for v in range(count):
        out = str(tmp_path / f"v{v}.npy")
        env = dict(os.environ, VLBM_MIXED_VARIANT=str(v))
        subprocess.run([sys.executable, "-c", SCRIPT.format(root=root, out=out, v=v)], env=env, check=True)
        outs.append(np.load(out))
    for v in range(1, count):
        assert np.array_equal(outs[0], outs[v]), v
