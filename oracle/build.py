"""Compile the C oracle (test infrastructure) into ``oracle/_build``.

``build(mutant=0)`` returns the path of the shared library; mutants plant one
known mistake each (see ``rk_oracle.c``) and exist only for the tests that
show the oracle's pins catch such mistakes.
"""

from __future__ import annotations

import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rk_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
_lock = threading.Lock()
# -O3 without -march=native: the library is built on x86-64 here and on
# AArch64 hosts, and must compute the same on both with portable code.
CFLAGS = ["-O3", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra"]


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mut{mutant}.so"
    return os.path.join(OUT_DIR, name)


def build(mutant: int = 0, force: bool = False) -> str:
    out = lib_path(mutant)
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= max(os.path.getmtime(SRC), os.path.getmtime(__file__))):
            return out
        os.makedirs(OUT_DIR, exist_ok=True)
        tmp = f"{out}.{os.getpid()}.tmp"
        cmd = ["gcc", *CFLAGS, f"-DORACLE_MUTANT={int(mutant)}", SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
