"""Builds the oracle's shared library (test infrastructure; plain gcc, no CUDA)."""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path(wide: bool = False) -> str:
    """libmpo.so holds mantissas up to 1024 bits; libmpo_wide.so (the same
    source built with 256-word mantissas) up to 8192 bits."""
    return os.path.join(_HERE, "libmpo_wide.so" if wide else "libmpo.so")


def _build_one(out: str, defs, force: bool) -> str:
    src = os.path.join(_HERE, "mpo.c")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)
            and os.path.getmtime(out) >= os.path.getmtime(os.path.join(_HERE, "mpo.h"))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-fPIC", "-shared", *defs, src, "-o",
           tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_oracle(force: bool = False) -> str:
    _build_one(lib_path(True), ["-DWMAX=256"], force)
    return _build_one(lib_path(False), [], force)


if __name__ == "__main__":
    print(build_oracle(force=True))
