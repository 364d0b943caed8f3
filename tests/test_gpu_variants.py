"""Every launch design of the mixed kernel (tile shape, one tile per CTA or
persistent) computes bit-identical results, so the autotuner's choice never
changes a realization (and nested prefixes stay exact)."""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCRIPT = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from tests import gpu_helpers as H
ens = H.gpu_jet([(67, 29), (150, 60)], 3, precision="mixed")
ens.step(12)
np.save({out!r}, np.concatenate([ens.get_state(l)[0].cpu().numpy().ravel() for l in range(2)]))
"""


def test_all_mixed_variants_agree_bitwise(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for v in range(3):
        out = str(tmp_path / f"v{v}.npy")
        env = dict(os.environ, VLBM_MIXED_VARIANT=str(v))
        subprocess.run([sys.executable, "-c", SCRIPT.format(root=root, out=out)], env=env, check=True)
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
