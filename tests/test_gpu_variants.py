"""Every launch design of the mixed kernel (tile shapes, persistent CTAs, warps
marching up column strips) computes bit-identical results, so the autotuner's
choice never changes a realization (and nested prefixes stay exact); the two
designs of the FP64 kernel (tiles, warp march) compute identical results.
The mixed runs cover single launches, a replayed graph of steps and landings
on an output time, and compare the times and step counts as well."""

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
ens.step(40)
t_mid = max(float(ens.time(l)[0].max()) for l in range(len(levels)))
ens.advance_to(1.5 * t_mid)
idx, name, count = ens.step_design()
assert idx == {v}, (idx, name)
parts = []
for l in range(len(levels)):
    t, n = ens.time(l)
    assert np.all(t == 1.5 * t_mid), (l, t)
    parts += [ens.get_state(l)[0].cpu().numpy().ravel(), t, n.astype(np.float64)]
np.save({out!r}, np.concatenate(parts))
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


SCRIPT_ROWS = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
from tests import gpu_helpers as H
levels = [(67, 29), (150, 60), (96, 230), (3, 3), (5, 7)]
ens = H.gpu_jet(levels, 2, precision="mixed")
ens.step(12)
ens.step(40)
assert ens.step_rows() == {rows}, ens.step_rows()
parts = []
for l in range(len(levels)):
    t, n = ens.time(l)
    parts += [ens.get_state(l)[0].cpu().numpy().ravel(), t, n.astype(np.float64)]
np.save({out!r}, np.concatenate(parts))
"""


@pytest.mark.parametrize("variant", [3, 5])
def test_march_row_counts_agree_bitwise(tmp_path, variant):
    # the rows per warp of a march (tuned on small launches) change no result:
    # one row per warp (every warp a warm-up and one row), 2, 3 and 25
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for rows in (25, 1, 2, 3):
        out = str(tmp_path / f"r{rows}.npy")
        env = dict(os.environ, VLBM_MIXED_VARIANT=str(variant), VLBM_MARCH_ROWS=str(rows))
        subprocess.run([sys.executable, "-c", SCRIPT_ROWS.format(root=root, out=out, rows=rows)], env=env,
                       check=True)
        outs.append(np.load(out))
    for k in range(1, len(outs)):
        assert np.array_equal(outs[0], outs[k]), k


def test_small_launch_tunes_march_rows():
    # a single small grid: the context times row counts for a winning march
    ens = H.gpu_jet([(400, 200)], 1, precision="mixed")
    ens.step(2)
    idx, name, count = ens.step_design()
    rows = ens.step_rows()
    print("400 x 200, M = 1:", name, rows, "rows per warp")
    if name.startswith("march"):
        assert rows in (1, 2, 3, 4, 6, 8, 12, 16), rows
    else:
        assert rows == 0
    ens.close()
