"""Builds the oracle's shared library with the host C compiler (test infrastructure)."""
from __future__ import annotations

import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")


def library_path() -> str:
    """Path of the oracle library; WD_ORACLE_LIB names a prebuilt variant
    (the mutation tests point it at deliberately broken copies)."""
    return os.environ.get("WD_ORACLE_LIB") or os.path.join(_HERE, "_build", "liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile wilson_oracle.c into oracle/_build/liboracle.so if it is missing or stale."""
    if os.environ.get("WD_ORACLE_LIB"):
        return os.environ["WD_ORACLE_LIB"]
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [os.environ.get("CC", "gcc"), "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
