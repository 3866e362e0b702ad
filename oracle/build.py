"""Compile the C part of the oracle (test infrastructure only).

``python -m oracle.build`` or ``build_oracle()`` writes ``oracle/_lib/liboracle_kpm.so``
with gcc (OpenMP when the compiler supports it).  Plain portable C: it builds the
same on x86_64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "liboracle_kpm.so")
SOURCES = [os.path.join(HERE, "kpm_oracle.c")]


def build_oracle(force: bool = False) -> str:
    if (not force and os.path.exists(LIB_PATH)
            and all(os.path.getmtime(LIB_PATH) >= os.path.getmtime(s) for s in SOURCES)):
        return LIB_PATH
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp] + SOURCES + ["-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
