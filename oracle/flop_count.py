"""Builds and runs ``flop_count.cpp``: the FP64 operation count of the
oracle's step per cell-update (test infrastructure; an analysis of the
oracle, see the C++ file's header).

    python -m oracle.flop_count [nx ny t1 t2 ...]     (default 400 200 1e-5 3e-4 2e-3 3.5e-3)
"""

from __future__ import annotations

import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flop_count.cpp")
_EXE = os.path.join(_HERE, "_build", "flop_count")


def build(force: bool = False) -> str:
    """Compile with g++ (the oracle source unchanged, no FMA contraction)."""
    os.makedirs(os.path.dirname(_EXE), exist_ok=True)
    deps = (_SRC, os.path.join(_HERE, "vlbm_oracle.c"))
    if force or not os.path.exists(_EXE) or any(os.path.getmtime(_EXE) < os.path.getmtime(d) for d in deps):
        tmp = _EXE + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fpermissive",
                               "-w", "-I", _HERE, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _EXE)
    return _EXE


def run(nx: int = 400, ny: int = 200, times=(1e-5, 3e-4, 2e-3, 3.5e-3)) -> list[dict]:
    exe = build()
    out = subprocess.run([exe, str(nx), str(ny), *map(str, times)], capture_output=True, text=True, check=True)
    rows = []
    for line in out.stdout.splitlines():
        f = line.split()
        rec = {"nx": int(f[0]), "ny": int(f[1]), "t": float(f[2])}
        for k in range(3, len(f), 2):
            rec[f[k]] = float(f[k + 1])
        rec["arith"] = rec["add"] + rec["mul"] + rec["div"] + rec["sqrt"]
        rows.append(rec)
    return rows


if __name__ == "__main__":
    a = sys.argv[1:]
    rows = run(int(a[0]), int(a[1]), [float(x) for x in a[2:]]) if len(a) >= 3 else run()
    for r in rows:
        print(f"{r['nx']}x{r['ny']} t = {r['t']:g}: {r['arith']:.1f} FP64 arithmetic operations per cell-update "
              f"(add {r['add']:.1f}, mul {r['mul']:.1f}, div {r['div']:.1f}, sqrt {r['sqrt']:.2f}), "
              f"compare {r['cmp']:.1f}, abs {r['abs']:.1f}")
