"""Compile the CPU oracle (``aes_oracle.c``) into a shared library with gcc.

Test infrastructure: the tests, ``__graft_entry__`` and the benchmark's CPU
baseline leg are the only users.  ``mutant=n`` builds the variant with the
deliberate mistake number ``n`` planted (see ``aes_oracle.c``); the tests use
those variants to show that the oracle's pins catch each mistake.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "aes_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(out_path: str | None = None, mutant: int = 0, force: bool = False) -> str:
    out = out_path or LIB
    if (not force and mutant == 0 and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Wextra", "-shared", "-fPIC", "-pthread",
           f"-DORC_MUTANT={int(mutant)}", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)  # atomic: a concurrent loader never sees a half-written file
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
