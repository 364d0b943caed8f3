"""The oracle's rate fit (Eq. (ratefit)) against the paper's own error tables
(Sec. 4, Tables tab:err-t0p0005 ... tab:err-t0p0035, `tests/golden/error_tables.txt`).

Every table prints, for both protocols of Eqs. (cauchy) and (ref), the three
per-pair L1 errors of five observables and the fitted rates.  Fed the printed
errors, with each error attached to the mesh width of the coarser member of
its pair (Dx = 2.5 / Nx, the paper's reading), the oracle's fit must give the
printed rates: 70 rates, each within what the errors' 4 printed digits allow.
A fit against the finer member's width, or of log(Dx) against log(error),
fails it.
"""

import os

import numpy as np

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "error_tables.txt")
OBS = ("W_11", "W_12", "E_mean", "E_std", "E_strong")


def _tables():
    blocks = {}
    with open(GOLDEN) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t, proto, kind, a, b, *vals = line.split()
            blk = blocks.setdefault((t, proto), {"pairs": [], "rates": None})
            if kind == "pair":
                blk["pairs"].append((int(a), int(b), [float(v) for v in vals]))
            else:
                blk["rates"] = [float(v) for v in vals]
    return blocks


def _max_rounding_effect(dx, err):
    # the slope moves by at most sum |d slope / d log e_l| x (half a unit of the
    # 4th printed digit, relative)
    x = np.log(dx)
    w = (x - x.mean()) / ((x - x.mean()) ** 2).sum()
    rel = np.array([0.5e-3 / float(f"{e:.3e}".split("e")[0]) for e in err])
    return float(np.abs(w) @ rel)


def test_rate_fit_reproduces_the_papers_tables():
    blocks = _tables()
    assert len(blocks) == 14
    checked = 0
    for (t, proto), blk in sorted(blocks.items()):
        assert len(blk["pairs"]) == 3 and blk["rates"] is not None
        dx = np.array([2.5 / coarse for coarse, _, _ in blk["pairs"]])
        for k, name in enumerate(OBS):
            err = np.array([e[k] for _, _, e in blk["pairs"]])
            r, _ = O.rate_fit(dx, err)
            tol = _max_rounding_effect(dx, err) + 0.5e-3  # + the rate's own printed rounding
            assert abs(r - blk["rates"][k]) <= tol, (t, proto, name, r, blk["rates"][k])
            checked += 1
    assert checked == 70


def test_the_pairing_is_the_coarser_member():
    # the same errors attached to the finer member's width give other rates in
    # the Cauchy protocol (its pairs step by 2 in both members: the slope is
    # unchanged) but not in the reference protocol (all finer members are 4000)
    blocks = _tables()
    blk = blocks[("0.0035", "reference")]
    err = np.array([e[0] for _, _, e in blk["pairs"]])
    dx_fine = np.array([2.5 / fine for _, fine, _ in blk["pairs"]])
    assert np.ptp(np.log(dx_fine)) == 0.0  # no fit possible: the reading must be the coarser member
    dx = np.array([2.5 / c for c, _, _ in blk["pairs"]])
    assert abs(O.rate_fit(dx, err)[0] - blk["rates"][0]) < 2e-3
