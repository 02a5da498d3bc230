"""Build the CPU oracle (test infrastructure only).

Compiles ``dog_oracle.c`` twice with gcc: the FP32 mirror (``liboracle_f32.so``, IEEE
binary32 with contraction off) and the FP64 mode (``liboracle_f64.so``).  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` load them.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dog_oracle.c")
TARGETS = {
    "f32": (os.path.join(HERE, "liboracle_f32.so"), ["-DORACLE_F32"]),
    "f64": (os.path.join(HERE, "liboracle_f64.so"), []),
}
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-Wall", "-Wextra"]


def build(force: bool = False) -> dict:
    out = {}
    for mode, (path, defs) in TARGETS.items():
        stale = (not os.path.exists(path)) or os.path.getmtime(path) < os.path.getmtime(SRC)
        if force or stale:
            cmd = ["gcc", *CFLAGS, *defs, "-o", path, SRC, "-lm"]
            subprocess.run(cmd, check=True)
        out[mode] = path
    return out


if __name__ == "__main__":
    for k, v in build(force=True).items():
        print(k, v)
