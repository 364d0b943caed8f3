"""Every launch design of the mixed kernel (tile shapes, persistent CTAs, warps
marching up column strips) computes bit-identical results, so the autotuner's
choice never changes a realization (and nested prefixes stay exact); the two
designs of the FP64 kernel (tiles, warp march) compute identical results."""

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
levels = [(67, 29), (150, 60), (96, 230), (3, 3), (5, 7)]
ens = H.gpu_jet(levels, 3, precision="mixed")
ens.step(12)
idx, name, count = ens.step_design()
assert idx == {v}, (idx, name)
np.save({out!r}, np.concatenate([ens.get_state(l)[0].cpu().numpy().ravel() for l in range(len(levels))]))
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


SCRIPT64 = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from tests import gpu_helpers as H
levels = [(67, 29), (150, 60), (96, 230), (9, 3), (31, 5), (3, 3), (3, 7)]
for limiter in (2, 0, 1):
    ens = H.gpu_jet(levels, 3, precision="fp64", limiter=limiter)
    ens.step(12 if limiter != 1 else 3)
    idx, name, count = ens.step_design()
    assert idx == {v} and count == 2, (idx, name, count)
    np.save({out!r}.replace(".npy", f"_{{limiter}}.npy"),
            np.concatenate([x.cpu().numpy().ravel() for l in range(len(levels)) for x in ens.get_state(l)]))
"""


def test_fp64_designs_agree_bitwise(tmp_path):
    # ragged strips and row chunks, a level with a single interior row, three limiters
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for v in (0, 1):
        out = str(tmp_path / f"f{v}.npy")
        env = dict(os.environ, VLBM_F64_VARIANT=str(v))
        subprocess.run([sys.executable, "-c", SCRIPT64.format(root=root, out=out, v=v)], env=env, check=True)
    for limiter in (2, 0, 1):
        a = np.load(str(tmp_path / f"f0_{limiter}.npy"))
        b = np.load(str(tmp_path / f"f1_{limiter}.npy"))
        assert np.array_equal(a, b, equal_nan=True), limiter
